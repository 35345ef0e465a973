"""ctypes binding of libdgcurved.so (include/dgcurved.h), same names as the
C ABI.  Argument marshalling only: every step of the computation runs in the
library.  Loading fails loudly when the library is missing; there is no
fallback.
"""
import ctypes as C
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdgcurved.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONFINITE, DG_ETIMEOUT, DG_EBUSY, DG_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
DG_FP32, DG_TF32, DG_BF16X3, DG_FP64_DEBUG = 0, 1, 2, 3
DG_BC_INTERIOR, DG_BC_WALL, DG_BC_FARFIELD = 0, 1, 2
PREC = {"fp32": DG_FP32, "tf32": DG_TF32, "bf16x3": DG_BF16X3, "fp64": DG_FP64_DEBUG}


class DgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dgcurved status %d: %s" % (status, msg))
        self.status = status


class dg_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("flux", C.c_int32), ("av_on", C.c_int32),
                ("kappa", C.c_double), ("eps0", C.c_double), ("s0", C.c_double),
                ("u_inf", C.c_double * 5), ("prec", C.c_int32), ("cub_q", C.c_int32)]


FLUX = {"llf": 0, "hllc": 1}


def make_params(gamma=1.4, av_on=False, kappa=4.0, eps0=0.3, s0=None, u_inf=(1.0, 0.0, 0.0, 2.5),
                prec="fp32", cub_q=0, flux="llf"):
    p = dg_params()
    p.gamma = gamma
    p.flux = FLUX[flux] if isinstance(flux, str) else int(flux)
    p.av_on = int(bool(av_on))
    p.kappa, p.eps0 = kappa, eps0
    p.s0 = math.nan if s0 is None else float(s0)
    for i in range(len(u_inf)):      # four values on triangles, five on tetrahedra
        p.u_inf[i] = float(u_inf[i])
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    p.cub_q = cub_q
    return p


_lib = None


def load():
    """Load the library (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdgcurved.so not built at %s: run __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    dp = C.POINTER(C.c_double)
    sig = {
        "dg_create": (I, [C.POINTER(P), I, P]),
        "dg_destroy": (I, [P]),
        "dg_set_host_io": (I, [P, I]),
        "dg_host_io": (I, [P, C.POINTER(C.c_int32)]),
        "dg_reference_nodes": (I, [I, dp]),
        "dg_sizes": (I, [I, I, C.POINTER(C.c_int32)]),
        "dg_mesh_upload": (I, [P, I, I64, P, P, P, dp, C.POINTER(dg_params), C.POINTER(C.c_int32)]),
        "dg_mesh_free": (I, [P, C.c_int32]),
        "dg_mesh_prepare": (I, [I, I64, P, P, P, dp, C.POINTER(dg_params), C.POINTER(P)]),
        "dg_mesh_upload_prepared": (I, [P, P, C.POINTER(C.c_int32)]),
        "dg_prepared_free": (I, [P]),
        "dg_batch_residual": (I, [P, I, C.POINTER(C.c_int32), dp]),
        "dg_mesh_bytes": (I, [P, C.c_int32, C.POINTER(I64)]),
        "dg_set_state": (I, [P, C.c_int32, dp]),
        "dg_get_state": (I, [P, C.c_int32, dp]),
        "dg_set_state_device": (I, [P, C.c_int32, P]),
        "dg_get_state_device": (I, [P, C.c_int32, P]),
        "dg_eval_rhs": (I, [P, C.c_int32, dp]),
        "dg_step": (I, [P, C.c_int32, D, I]),
        "dg_residual": (I, [P, C.c_int32, dp, dp]),
        "dg_batch_step": (I, [P, I, C.POINTER(C.c_int32), dp, I]),
        "dg_sync": (I, [P, D]),
        "dg_selftest_bounded_wait": (I, [P, C.c_uint32, I, C.POINTER(C.c_int32)]),
        "dg_set_profiling": (I, [P, C.c_int32, I]),
        "dg_residual_norms_noalloc": (I, [P, I64, C.c_int32, P, P]),
        "dg_kernel_times": (I, [P, C.c_int32, dp]),
        "dg_prolong": (I, [P, C.c_int32, C.c_int32]),
        "dg_step_lserk": (I, [P, C.c_int32, D, I]),
        "dg_autotune": (I, [P, C.c_int32, I, C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp,
                            C.POINTER(C.c_int32)]),
        "dg_set_tc_config": (I, [P, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "dg_tet_reference_nodes": (I, [I, dp]),
        "dg_tet_sizes": (I, [I, C.POINTER(C.c_int32)]),
        "dg_tet_mesh_upload": (I, [P, I, I64, P, P, dp, C.POINTER(dg_params), C.POINTER(C.c_int32)]),
        "dg_mesh_info": (I, [P, C.c_int32, C.POINTER(I64)]),
        "dg_av_count": (I, [P, C.c_int32, C.POINTER(I64)]),
        "dg_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != DG_OK:
        msg = load().dg_last_error(ctx)
        raise DgError(status, msg.decode() if msg else "")
    return status


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------- calls
def dg_create(device=0, stream=None):
    ctx = C.c_void_p()
    _check(load().dg_create(C.byref(ctx), device, stream), None)
    return ctx


def dg_destroy(ctx):
    return _check(load().dg_destroy(ctx), None)


HOST_IO = {"auto": 0, "staged": 1, "device": 2}


def dg_set_host_io(ctx, mode):
    """How dg_set_state / dg_get_state / dg_eval_rhs move host FP64 state:
    "staged" (host threads and one copy; also "auto"), or "device" (a kernel
    on the caller's rows through coherent host-memory access)."""
    return _check(load().dg_set_host_io(ctx, HOST_IO[mode] if isinstance(mode, str) else int(mode)), ctx)


def dg_host_io(ctx):
    """The host I/O mode in effect: "staged" or "device"."""
    out = C.c_int32()
    _check(load().dg_host_io(ctx, C.byref(out)), ctx)
    return {v: k for k, v in HOST_IO.items()}[out.value]


def dg_reference_nodes(N):
    np_ = (N + 1) * (N + 2) // 2
    out = np.zeros((np_, 2))
    _check(load().dg_reference_nodes(N, _dptr(out)), None)
    return out[:, 0].copy(), out[:, 1].copy()


def dg_sizes(N, cub_q=0):
    out = (C.c_int32 * 4)()
    _check(load().dg_sizes(N, cub_q, out), None)
    return tuple(out)


def dg_mesh_upload(ctx, N, EToE, EToF, bc, node_xy, params):
    EToE = np.ascontiguousarray(EToE, dtype=np.int32)
    EToF = np.ascontiguousarray(EToF, dtype=np.int8)
    bc = np.ascontiguousarray(bc, dtype=np.int8)
    node_xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    K = EToE.shape[0]
    h = C.c_int32()
    _check(load().dg_mesh_upload(ctx, N, K, EToE.ctypes.data, EToF.ctypes.data, bc.ctypes.data,
                                 _dptr(node_xy), C.byref(params), C.byref(h)), ctx)
    return h.value


def dg_mesh_prepare(N, EToE, EToF, bc, node_xy, params):
    """Host half of dg_mesh_upload (no context; may run on a worker thread:
    ctypes releases the interpreter lock during the call).  Returns an
    opaque handle for dg_mesh_upload_prepared or dg_prepared_free."""
    EToE = np.ascontiguousarray(EToE, dtype=np.int32)
    EToF = np.ascontiguousarray(EToF, dtype=np.int8)
    bc = np.ascontiguousarray(bc, dtype=np.int8)
    node_xy = np.ascontiguousarray(node_xy, dtype=np.float64)
    out = C.c_void_p()
    _check(load().dg_mesh_prepare(N, EToE.shape[0], EToE.ctypes.data, EToF.ctypes.data, bc.ctypes.data,
                                  _dptr(node_xy), C.byref(params), C.byref(out)))
    return out.value


def dg_mesh_upload_prepared(ctx, prep):
    h = C.c_int32()
    _check(load().dg_mesh_upload_prepared(ctx, C.c_void_p(prep), C.byref(h)), ctx)
    return h.value


def dg_prepared_free(prep):
    _check(load().dg_prepared_free(C.c_void_p(prep)))


def dg_batch_residual(ctx, meshes, allow_nonfinite=False):
    """(linf [n, 4], l2 [n, 4]) of n triangle meshes with one synchronisation."""
    n = len(meshes)
    hs = (C.c_int32 * n)(*meshes)
    out = np.zeros((n, 10))
    st = load().dg_batch_residual(ctx, n, hs, _dptr(out))
    if not (allow_nonfinite and st == DG_ENONFINITE):
        _check(st, ctx)
    return out[:, :4].copy(), out[:, 5:9].copy()


def dg_mesh_info(ctx, m):
    out = (C.c_int64 * 6)()
    _check(load().dg_mesh_info(ctx, m, out), ctx)
    return dict(zip(("dim", "nvar", "N", "Np", "K", "curved"), (int(v) for v in out)))


def _state_shape(ctx, m, K, Np):
    info = dg_mesh_info(ctx, m)
    if (K is not None and K != info["K"]) or (Np is not None and Np != info["Np"]):
        raise ValueError("K / Np do not match the mesh (%d, %d)" % (info["K"], info["Np"]))
    return (info["K"], info["nvar"], info["Np"])


def dg_tet_reference_nodes(N):
    np_ = (N + 1) * (N + 2) * (N + 3) // 6
    out = np.zeros((np_, 3))
    _check(load().dg_tet_reference_nodes(N, _dptr(out)), None)
    return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy()


def dg_tet_sizes(N):
    out = (C.c_int32 * 4)()
    _check(load().dg_tet_sizes(N, out), None)
    return tuple(out)


def dg_tet_mesh_upload(ctx, N, EToV, bc, node_xyz, params):
    EToV = np.ascontiguousarray(EToV, dtype=np.int64)
    bc = np.ascontiguousarray(bc, dtype=np.int8)
    node_xyz = np.ascontiguousarray(node_xyz, dtype=np.float64)
    K = EToV.shape[0]
    h = C.c_int32()
    _check(load().dg_tet_mesh_upload(ctx, N, K, EToV.ctypes.data, bc.ctypes.data, _dptr(node_xyz),
                                     C.byref(params), C.byref(h)), ctx)
    return h.value


def dg_av_count(ctx, m):
    """Elements with eps > 0 for the current state."""
    out = C.c_int64()
    _check(load().dg_av_count(ctx, m, C.byref(out)), ctx)
    return int(out.value)


def dg_mesh_free(ctx, m):
    return _check(load().dg_mesh_free(ctx, m), ctx)


def dg_mesh_bytes(ctx, m):
    out = C.c_int64()
    _check(load().dg_mesh_bytes(ctx, m, C.byref(out)), ctx)
    return out.value


def dg_set_state(ctx, m, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return _check(load().dg_set_state(ctx, m, _dptr(U)), ctx)


def dg_get_state(ctx, m, K=None, Np=None):
    out = np.zeros(_state_shape(ctx, m, K, Np))
    _check(load().dg_get_state(ctx, m, _dptr(out)), ctx)
    return out


def dg_set_state_device(ctx, m, dev_ptr):
    return _check(load().dg_set_state_device(ctx, m, C.c_void_p(dev_ptr)), ctx)


def dg_get_state_device(ctx, m, dev_ptr):
    return _check(load().dg_get_state_device(ctx, m, C.c_void_p(dev_ptr)), ctx)


def dg_eval_rhs(ctx, m, K=None, Np=None):
    out = np.zeros(_state_shape(ctx, m, K, Np))
    _check(load().dg_eval_rhs(ctx, m, _dptr(out)), ctx)
    return out


def dg_step(ctx, m, dt, nsteps):
    return _check(load().dg_step(ctx, m, float(dt), int(nsteps)), ctx)


def dg_residual(ctx, m, allow_nonfinite=False):
    nv = dg_mesh_info(ctx, m)["nvar"]
    linf = np.zeros(nv)
    l2 = np.zeros(nv)
    st = load().dg_residual(ctx, m, _dptr(linf), _dptr(l2))
    if not (allow_nonfinite and st == DG_ENONFINITE):
        _check(st, ctx)
    return linf, l2


def dg_batch_step(ctx, meshes, dts, nsteps):
    ms = (C.c_int32 * len(meshes))(*meshes)
    d = np.ascontiguousarray(dts, dtype=np.float64)
    return _check(load().dg_batch_step(ctx, len(meshes), ms, _dptr(d), int(nsteps)), ctx)


def dg_sync(ctx, timeout_s=0.0):
    return _check(load().dg_sync(ctx, float(timeout_s)), ctx)


def dg_selftest_bounded_wait(ctx, limit, arrive):
    """1 if a bounded device wait with nothing arriving ran out, 0 if it completed."""
    out = C.c_int32(-1)
    _check(load().dg_selftest_bounded_wait(ctx, C.c_uint32(int(limit)), int(arrive), C.byref(out)), ctx)
    return out.value


def dg_residual_norms_noalloc(values_dev_ptr, K, Np, out8_dev_ptr, stream=None):
    """FP64 residual norms of a device float[K][4][Np] into a device
    double[8], without any allocation (see include/dgcurved.h)."""
    st = load().dg_residual_norms_noalloc(C.c_void_p(values_dev_ptr), int(K), int(Np), C.c_void_p(out8_dev_ptr),
                                          None if stream is None else C.c_void_p(stream))
    return _check(st, None)


def dg_set_profiling(ctx, m, on):
    return _check(load().dg_set_profiling(ctx, m, int(on)), ctx)


def dg_step_lserk(ctx, m, dt, nsteps):
    """nsteps steps of the five-stage fourth-order low-storage RK."""
    return _check(load().dg_step_lserk(ctx, m, float(dt), int(nsteps)), ctx)


def dg_prolong(ctx, m_from, m_to):
    """Embed the state of m_from exactly into m_to (same mesh, degree >=)."""
    return _check(load().dg_prolong(ctx, m_from, m_to), ctx)


def dg_autotune(ctx, m, nsteps=5):
    """The autotuner: returns (elements per tile, {candidate: ms per step},
    chosen candidate).  CUDA-core paths: the candidates are tile sizes and
    the chosen one is the tile size; the tensor-core path on triangles: the
    tiles are 32 elements and the candidates are the stage kernel's
    tile-pipeline configurations 10 C + P (C CTAs per SM of P pipelines)."""
    best = C.c_int32(0)
    cand = (C.c_int32 * 8)()
    ms = np.zeros(8)
    n = C.c_int32(0)
    _check(load().dg_autotune(ctx, m, int(nsteps), C.byref(best), cand, _dptr(ms), C.byref(n)), ctx)
    table = {int(cand[i]): float(ms[i]) for i in range(n.value)}
    return int(best.value), table, (min(table, key=table.get) if table else int(best.value))


def dg_set_tc_config(ctx, m, cfg=0):
    """Set a tensor-core mesh's tile-pipeline configuration (0: the default);
    returns the codes that fit its kernel."""
    cand = (C.c_int32 * 4)()
    n = C.c_int32(0)
    _check(load().dg_set_tc_config(ctx, m, int(cfg), cand, C.byref(n)), ctx)
    return [int(cand[i]) for i in range(n.value)]


def dg_kernel_times(ctx, m):
    """(sensor_ms, gradient_ms, stage_ms, kernels_per_step) of the last step."""
    out = np.zeros(4)
    _check(load().dg_kernel_times(ctx, m, _dptr(out)), ctx)
    return out


def dg_last_error(ctx=None):
    msg = load().dg_last_error(ctx)
    return msg.decode() if msg else ""

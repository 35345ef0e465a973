"""Tensor-core (tcgen05) path, DG_TF32 and DG_BF16X3, against the FP64
oracle and against the FP32 CUDA-core path.

Tolerances (from the arithmetic of the products):
  * BF16 x3: each operand is split into a BF16 high and low part and three
    products are summed; the dropped low x low term and the BF16 rounding of
    the low parts leave ~2^-16 relative error per product, applied to the
    deviation from the element-mean state -> right-hand side within 1e-5 of
    the volume-term norm (as the FP32 path), states after 100 steps within
    1e-5 relative L2.
  * TF32: 10-bit mantissa (2^-11 relative per operand), again on the
    deviations only -> right-hand side within 2e-3 of the volume-term norm,
    states after 100 vortex steps within 1e-4 relative L2.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg import Oracle
from paper_1208_4772_gb300.inputs import meshes, states
from cases import make_case, rel_l2_per_var

pytestmark = pytest.mark.gpu

RHS_TOL = {"tf32": 2e-3, "bf16x3": 1e-5}
STEP_TOL = {"tf32": 1e-4, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def B():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def upload(B, ctx, case, prec, U=None):
    m = case["mesh"]
    p = B.make_params(u_inf=case["u_inf"], av_on=case["av"], prec=prec)
    h = B.dg_mesh_upload(ctx, case["N"], m.EToE, m.EToF, m.bc, case["xy"], p)
    B.dg_set_state(ctx, h, case["U"] if U is None else U)
    return h


def oracle_of(case):
    m = case["mesh"]
    return Oracle(case["N"], m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=case["av"])


def term_scale(o, U):
    _, vol, _ = o.rhs(U, parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry(None).Minv, vol)
    return np.linalg.norm(V.transpose(1, 0, 2).reshape(4, -1), axis=1)


def rel_err(L, Lo, scale):
    return np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(4, -1), axis=1) / scale


CASES = [("vortex", N, False) for N in (2, 3, 4, 5, 6)] + \
        [("naca", 4, False), ("naca", 4, True), ("cyl", 6, False), ("cyl", 3, True), ("vortex", 5, True)]


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("kind,N,av", CASES)
def test_tc_rhs_matches_oracle(B, ctx, kind, N, av, prec):
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    case["U"] = case["U"].astype(np.float32).astype(np.float64)
    h = upload(B, ctx, case, prec)
    L = B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
    B.dg_mesh_free(ctx, h)
    o = oracle_of(case)
    Lo = o.rhs(case["U"])
    err = rel_err(L, Lo, term_scale(o, case["U"]))
    tol = RHS_TOL[prec] * (10 if av else 1)
    assert np.all(err <= tol), err


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tc_vortex_100_steps(B, ctx, prec):
    N = 2
    r, s = B.dg_reference_nodes(N)
    m = meshes.periodic_square(16, length=10.0, jitter=0.1, seed=1000)
    xy = meshes.straight_nodes(m.verts, r, s)
    U0 = states.vortex_state(xy, period=(10.0, 10.0))
    dt = states.time_step(m.verts, U0, N, cfl=0.3)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy)
    Uo = U0.copy()
    for _ in range(100):
        Uo = o.ssp_rk3_step(Uo, dt)
    case = dict(mesh=m, xy=xy, u_inf=states.freestream(0.5), U=U0, av=False, N=N)
    h = upload(B, ctx, case, prec)
    B.dg_step(ctx, h, dt, 100)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    err = rel_l2_per_var(Ug, Uo)
    assert np.all(err <= STEP_TOL[prec]), err


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tc_ragged_and_mixed_tiles(B, ctx, prec):
    """K below one tile, K not a multiple of 32, and a mesh whose curved
    tiles run the CUDA-core body inside the tensor-core launch."""
    for kind, N, size in (("vortex", 3, 3), ("vortex", 4, 5), ("naca", 2, "tiny"), ("cyl", 4, "small")):
        r, s = B.dg_reference_nodes(N)
        case = make_case(kind, N, r, s, size=size)
        case["U"] = case["U"].astype(np.float32).astype(np.float64)
        h = upload(B, ctx, case, prec)
        L = B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
        B.dg_mesh_free(ctx, h)
        o = oracle_of(case)
        err = rel_err(L, o.rhs(case["U"]), term_scale(o, case["U"]))
        assert np.all(err <= RHS_TOL[prec]), (kind, N, size, err)


def test_profiling_times_and_later_calls(B, ctx):
    """Kernel timing nodes in the step graph; calls made afterwards outside
    the graph (residual, state reads) are unaffected."""
    N = 4
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, av=True)
    h = upload(B, ctx, case, "tf32")
    B.dg_set_profiling(ctx, h, 1)
    dt = 0.1 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3)
    B.dg_step(ctx, h, dt, 2)
    B.dg_sync(ctx, 30.0)
    t = B.dg_kernel_times(ctx, h)
    # tensor-core path with AV: gradient and stage kernels per stage (the
    # stage kernel computes the next stage's sensor in its epilogue)
    assert t[3] == 6 and t[0] == 0 and np.all(t[1:3] > 0)
    B.dg_residual(ctx, h)
    B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
    B.dg_set_profiling(ctx, h, 0)
    B.dg_step(ctx, h, dt, 1)
    B.dg_sync(ctx, 30.0)
    with pytest.raises(B.DgError):
        B.dg_kernel_times(ctx, h)
    B.dg_mesh_free(ctx, h)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tc_batch_equals_single(B, ctx, prec):
    """The tensor-core batched stage (one persistent launch per stage for
    degrees 2..5, a second one for degree 6; curved tiles on the CUDA-core
    body) gives the same states as each mesh stepped alone: same tiles, same
    tile body.  The mix switches degree between items, so the operator
    tables are reloaded inside a CTA."""
    cases = []
    for i, (kind, N) in enumerate((("naca", 2), ("cyl", 3), ("vortex", 4), ("naca", 5), ("cyl", 6),
                                   ("vortex", 2), ("naca", 4))):
        r, s = B.dg_reference_nodes(N)
        cases.append(make_case(kind, N, r, s, seed=i))
    dts = [0.3 * states.time_step(c["mesh"].verts, c["U"], c["N"]) for c in cases]
    single = []
    for c, dt in zip(cases, dts):
        h = upload(B, ctx, c, prec)
        B.dg_step(ctx, h, dt, 3)
        single.append(B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2]))
        B.dg_mesh_free(ctx, h)
    hs = [upload(B, ctx, c, prec) for c in cases]
    B.dg_batch_step(ctx, hs, dts, 3)
    for h, c, Us in zip(hs, cases, single):
        Ub = B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2])
        assert np.array_equal(Ub, Us), (c["N"], np.abs(Ub - Us).max())
    for h in hs:
        B.dg_mesh_free(ctx, h)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tc_av_steps_match_fp32_path(B, ctx, prec):
    """With artificial viscosity the tensor-core path computes each stage's
    eps in the previous stage kernel's epilogue (three eps buffers in
    rotation; a sensor launch only when the state was set from outside).
    Twenty steps agree with the FP32 CUDA-core path, which runs the sensor
    kernel every stage, within the products' tolerance; a state set in
    between is picked up (its eps is recomputed), bitwise as on a fresh mesh."""
    N = 4
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, av=True)
    K, Np = case["mesh"].K, len(r)
    dt = 0.2 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3)
    out = {}
    for pr in ("fp32", prec):
        h = upload(B, ctx, case, pr)
        B.dg_step(ctx, h, dt, 10)
        B.dg_step(ctx, h, dt, 10)
        out[pr] = B.dg_get_state(ctx, h, K, Np)
        B.dg_mesh_free(ctx, h)
    err = rel_l2_per_var(out[prec], out["fp32"])
    assert np.all(err <= STEP_TOL[prec]), err
    # a state set from outside between steps
    h = upload(B, ctx, case, prec)
    B.dg_step(ctx, h, dt, 3)
    U1 = case["U"] * (1.0 + 1e-3 * np.cos(case["xy"][..., 0]))[:, None, :]
    B.dg_set_state(ctx, h, U1)
    B.dg_step(ctx, h, dt, 3)
    Ua = B.dg_get_state(ctx, h, K, Np)
    B.dg_mesh_free(ctx, h)
    h = upload(B, ctx, case, prec, U=U1)
    B.dg_step(ctx, h, dt, 3)
    Ub = B.dg_get_state(ctx, h, K, Np)
    B.dg_mesh_free(ctx, h)
    assert np.array_equal(Ua, Ub)


@pytest.mark.parametrize("prec", ["tf32"])
def test_av_viscous_switching_matches_fp32_path(B, ctx, prec):
    """Tiles with eps = 0 skip the gradient (their q is multiplied by
    sqrt(eps) = 0 wherever it enters), and a launch with no viscous tile at
    all does nothing; the count of viscous tiles travels with eps from
    kernel to kernel.  States that switch between inviscid (smooth) and
    viscous (noisy) between steps give the FP32 path's result each time,
    and LSERK steps and right-hand-side evaluations in between do not
    disturb the counts."""
    N = 4
    r, s = B.dg_reference_nodes(N)
    noisy = make_case("naca", N, r, s, av=True)
    smooth = make_case("naca", N, r, s, av=True, perturb=0.0)
    K, Np = noisy["mesh"].K, len(r)
    dt = 0.2 * states.time_step(noisy["mesh"].verts, noisy["U"], N, eps0=0.3)
    seq = [smooth["U"], noisy["U"], smooth["U"], noisy["U"]]
    out = {}
    for pr in ("fp32", prec):
        h = upload(B, ctx, noisy, pr, U=seq[0])
        res = []
        for i, U in enumerate(seq):
            B.dg_set_state(ctx, h, U)
            B.dg_step(ctx, h, dt, 4)
            if i == 1:
                B.dg_eval_rhs(ctx, h, K, Np)
                B.dg_step_lserk(ctx, h, dt, 1)
                B.dg_step(ctx, h, dt, 2)
            res.append(B.dg_get_state(ctx, h, K, Np))
        out[pr] = res
        B.dg_mesh_free(ctx, h)
    for a, b in zip(out[prec], out["fp32"]):
        err = rel_l2_per_var(a, b)
        assert np.all(err <= STEP_TOL[prec]), err


def test_av_count_matches_oracle_sensor(B, ctx):
    """dg_av_count = the number of elements the oracle's sensor gives eps > 0."""
    from oracle.dg import Oracle
    N = 4
    r, s = B.dg_reference_nodes(N)
    for perturb in (0.0, 0.02):
        case = make_case("naca", N, r, s, av=True, perturb=perturb)
        m = case["mesh"]
        U = case["U"].astype(np.float32).astype(np.float64)
        h = upload(B, ctx, case, "fp64", U=U)
        n = B.dg_av_count(ctx, h)
        B.dg_mesh_free(ctx, h)
        eps = Oracle(N, m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=True).sensor(U)
        assert n == int(np.sum(eps > 0)), (perturb, n, int(np.sum(eps > 0)))
        assert (n == 0) == (perturb == 0.0)


def _vortex_error_gpu(B, ctx, N, n, prec, T=0.2, length=10.0):
    from oracle import basis
    from oracle.operators import ReferenceElement
    ref = ReferenceElement(N)
    r, s = B.dg_reference_nodes(N)
    # interpolation to the cubature points from the library's own nodes
    Icub = ref.Vq @ np.linalg.inv(basis.vandermonde(N, r, s))
    m = meshes.periodic_square(n, length=length, seed=7)
    xy = meshes.straight_nodes(m.verts, r, s)
    U = states.vortex_state(xy, period=(length, length))
    dt0 = states.time_step(m.verts, U, N, cfl=0.3)
    nst = int(np.ceil(T / dt0))
    h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, xy, B.make_params(u_inf=states.freestream(0.5, 45.0), prec=prec))
    B.dg_set_state(ctx, h, U)
    B.dg_step(ctx, h, T / nst, nst)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    Ue = states.vortex_state(xy, t=T, period=(length, length))
    e = (Ug - Ue)[:, 0, :] @ Icub.T
    # affine elements: J is the constant area ratio
    v = m.verts
    J = 0.25 * np.abs((v[:, 1, 0] - v[:, 0, 0]) * (v[:, 2, 1] - v[:, 0, 1])
                      - (v[:, 2, 0] - v[:, 0, 0]) * (v[:, 1, 1] - v[:, 0, 1]))
    return np.sqrt(np.sum(J[:, None] * ref.wq[None, :] * e * e))


@pytest.mark.parametrize("N,n1", [(2, 16), (3, 8)])
def test_mixed_precision_keeps_convergence_order(B, ctx, N, n1):
    """The isentropic vortex at T = 0.2 on n and 2n periodic meshes (the
    oracle's convergence pin, run through the library): the density L2
    error falls at order >= N + 1/2 with TF32 and BF16 x3 products as with
    FP32, and the mixed-precision errors stay within 10% of the FP32 ones."""
    errs = {}
    for prec in ("fp32", "tf32", "bf16x3"):
        e1, e2 = _vortex_error_gpu(B, ctx, N, n1, prec), _vortex_error_gpu(B, ctx, N, 2 * n1, prec)
        errs[prec] = (e1, e2)
        assert np.log2(e1 / e2) >= N + 0.5, (prec, e1, e2)
    for prec in ("tf32", "bf16x3"):
        assert errs[prec][1] <= 1.1 * errs["fp32"][1], errs


@pytest.mark.parametrize("kind,N,av", [("naca", 4, True), ("cyl", 4, False), ("vortex", 6, False)])
def test_tc_autotune_times_pipeline_configurations(B, ctx, kind, N, av):
    """The autotuner on the tensor-core path times the stage kernel's
    tile-pipeline configurations that fit (10 C + P: C CTAs per SM of P
    pipelines), leaves the state as it was, and the chosen configuration
    steps bitwise like the default one (each tile's arithmetic does not
    depend on which pipeline runs it); a later mesh of the same kind
    inherits the choice."""
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    case["U"] = case["U"].astype(np.float32).astype(np.float64)
    dt = 0.2 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3 if av else None)
    K, Np = case["mesh"].K, len(r)
    c2 = B.dg_create(0)
    try:
        h = upload(B, c2, case, "tf32")
        B.dg_step(c2, h, dt, 2)
        Ud = B.dg_get_state(c2, h, K, Np)           # default configuration
        B.dg_set_state(c2, h, case["U"])
        tile, table, cfg = B.dg_autotune(c2, h, 3)
        assert tile == 32 and len(table) >= 1 and cfg in table and all(t > 0 for t in table.values()), table
        assert set(table) <= {11, 12, 13, 21, 113}
        assert np.array_equal(B.dg_get_state(c2, h, K, Np), case["U"])
        # the chosen configuration steps like the default one
        B.dg_step(c2, h, dt, 2)
        assert np.array_equal(B.dg_get_state(c2, h, K, Np), Ud)
        h2 = upload(B, c2, case, "tf32")             # inherits the tuned configuration
        B.dg_step(c2, h2, dt, 2)
        assert np.array_equal(B.dg_get_state(c2, h2, K, Np), Ud)
    finally:
        B.dg_destroy(c2)


@pytest.mark.parametrize("kind,N,av", [("cyl", 6, False), ("naca", 5, False), ("cyl", 4, False),
                                       ("naca", 4, True), ("vortex", 3, False)])
def test_tc_every_pipeline_configuration_steps_alike(B, ctx, kind, N, av):
    """Every tile-pipeline configuration that fits (set by hand), the lean
    three-pipeline layout (113: one operand buffer for the flux products,
    D2 in D1's face columns) among them, steps bitwise like the default
    one; a code that does not fit is refused."""
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    case["U"] = case["U"].astype(np.float32).astype(np.float64)
    dt = 0.2 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3 if av else None)
    K, Np = case["mesh"].K, len(r)
    c2 = B.dg_create(0)
    try:
        h = upload(B, c2, case, "tf32")
        cands = B.dg_set_tc_config(c2, h, 0)
        B.dg_step(c2, h, dt, 2)
        Ud = B.dg_get_state(c2, h, K, Np)
        assert np.all(np.isfinite(Ud))
        if N >= 5 and not av:
            assert 113 in cands, cands
        for cfg in cands:
            B.dg_set_tc_config(c2, h, cfg)
            B.dg_set_state(c2, h, case["U"])
            B.dg_step(c2, h, dt, 2)
            assert np.array_equal(B.dg_get_state(c2, h, K, Np), Ud), cfg
        with pytest.raises(B.DgError):
            B.dg_set_tc_config(c2, h, 99)
    finally:
        B.dg_destroy(c2)

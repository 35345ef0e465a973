"""Parity of the tetrahedral CUDA path (through the C ABI) with the FP64
tetrahedral oracle.

Tolerances (the arithmetic behind them), as on triangles:
  * DG_FP64_DEBUG: the same discretisation in FP64 with a different
    summation order, operator construction and mass-matrix factorisation ->
    round-off: <= 1e-11 of the volume term's norm per variable.
  * DG_FP32 right-hand side on an FP32-representable state: FP32 round-off
    over sums of N_q (up to 343) terms against the volume term that L is a
    small difference of -> <= 1e-5 of that term's norm per variable.
  * Steps: relative L2 per variable <= 1e-11 (FP64), 1e-5 (FP32).
  * DG_TF32 (N = 2, 3: the two volume products on the tensor cores): the
    operands are rounded to TF32 (11-bit significand, relative 2^-11) but
    act on deviations from the element's mean state and its flux, which
    are small against the volume term -> <= 2e-3 of the volume term's norm
    (the bound of the triangle tensor-core path); steps <= 1e-4.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg3 import Oracle3
from paper_1208_4772_gb300.inputs import states
from cases import make_case3

pytestmark = pytest.mark.gpu


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


def setup(B, ctx, kind, N, prec, flux="llf", size="small"):
    r, s, t = B.dg_tet_reference_nodes(N)
    case = make_case3(kind, N, r, s, t, size=size)
    m = case["mesh"]
    U = case["U"].astype(np.float32).astype(np.float64)
    p = B.make_params(u_inf=case["u_inf"], prec=prec, flux=flux)
    h = B.dg_tet_mesh_upload(ctx, N, m.EToV, m.bc, case["xyz"], p)
    B.dg_set_state(ctx, h, U)
    o = Oracle3(N, m.EToV, m.bc, case["xyz"], u_inf=case["u_inf"], flux=flux)
    return case, U, h, o


TF32_TOL = 2e-3        # DG_TF32: the products round their operands to TF32
TF32_STEP_TOL = 1e-4
CASES = [("box", 2), ("box", 3), ("box", 4), ("wbox", 3), ("bump", 2), ("bump", 3), ("bump", 4)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("tf32", TF32_TOL)])
@pytest.mark.parametrize("flux", ["llf", "hllc"])
@pytest.mark.parametrize("kind,N", CASES)
def test_tet_rhs_matches_oracle(B, ctx, kind, N, flux, prec, tol):
    if prec == "tf32" and N > 3:
        pytest.skip("the tensor-core tetrahedral kernel covers N = 2, 3")
    case, U, h, o = setup(B, ctx, kind, N, prec, flux)
    info = B.dg_mesh_info(ctx, h)
    assert (info["dim"], info["nvar"], info["N"]) == (3, 5, N)
    if kind != "box":
        assert info["curved"] > 0
    L = B.dg_eval_rhs(ctx, h)
    B.dg_mesh_free(ctx, h)
    Lo, vol, _ = o.rhs(U, parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry().Minv, vol)
    scale = np.linalg.norm(V.transpose(1, 0, 2).reshape(5, -1), axis=1)
    err = np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(5, -1), axis=1) / scale
    assert np.all(np.isfinite(L))
    assert np.all(err <= tol), (kind, N, flux, prec, err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("tf32", TF32_TOL)])
@pytest.mark.parametrize("flux", ["llf", "hllc"])
@pytest.mark.parametrize("kind,N", [("single", 2), ("single", 4), ("pair", 3), ("pair", 4)])
def test_tet_minimal_meshes_match_oracle(B, ctx, kind, N, flux, prec, tol):
    if prec == "tf32" and N > 3:
        pytest.skip("the tensor-core tetrahedral kernel covers N = 2, 3")
    """One element with only boundary faces, and two elements whose shared
    face has different orientation codes on its two sides (a tile far from
    full)."""
    case, U, h, o = setup(B, ctx, kind, N, prec, flux)
    L = B.dg_eval_rhs(ctx, h)
    B.dg_mesh_free(ctx, h)
    Lo, vol, _ = o.rhs(U, parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry().Minv, vol)
    scale = np.linalg.norm(V.transpose(1, 0, 2).reshape(5, -1), axis=1)
    err = np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(5, -1), axis=1) / scale
    assert L.shape == Lo.shape
    assert np.all(err <= tol), (kind, N, flux, prec, err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("tf32", TF32_STEP_TOL)])
@pytest.mark.parametrize("kind,N", [("box", 2), ("bump", 3)])
def test_tet_steps_match_oracle(B, ctx, kind, N, prec, tol):
    case, U, h, o = setup(B, ctx, kind, N, prec)
    m = case["mesh"]
    dt = states.time_step3(m.verts, U, N)
    B.dg_step(ctx, h, dt, 4)
    B.dg_step_lserk(ctx, h, dt, 2)
    Ug = B.dg_get_state(ctx, h)
    B.dg_mesh_free(ctx, h)
    Uo = U.copy()
    for _ in range(4):
        Uo = o.ssp_rk3_step(Uo, dt)
    for _ in range(2):
        Uo = o.lserk54_step(Uo, dt)
    # per variable, relative to the norm of that variable -- for the three
    # momentum components the norm of the whole momentum (w is ~0 on the
    # extruded vortex)
    nrm = np.linalg.norm(Uo.transpose(1, 0, 2).reshape(5, -1), axis=1)
    nrm[1:4] = np.linalg.norm(nrm[1:4])
    err = np.linalg.norm((Ug - Uo).transpose(1, 0, 2).reshape(5, -1), axis=1) / nrm
    assert np.all(err <= tol), err


def test_tet_residual_matches_oracle(B, ctx):
    case, U, h, o = setup(B, ctx, "bump", 3, "fp64")
    linf, l2 = B.dg_residual(ctx, h)
    B.dg_mesh_free(ctx, h)
    lo, l2o = o.residual(U)
    assert linf.shape == (5,)
    assert np.allclose(linf, lo, rtol=1e-10)
    assert np.allclose(l2, l2o, rtol=1e-10)


def test_tet_free_stream_on_curved_walls(B, ctx):
    """A uniform flow on the warped periodic box stays uniform (curved
    geometry, FP64)."""
    r, s, t = B.dg_tet_reference_nodes(3)
    case = make_case3("wbox", 3, r, s, t)
    m = case["mesh"]
    p = B.make_params(u_inf=case["u_inf"], prec="fp64")
    h = B.dg_tet_mesh_upload(ctx, 3, m.EToV, m.bc, case["xyz"], p)
    B.dg_set_state(ctx, h, states.uniform_state3(m.K, len(r), case["u_inf"]))
    L = B.dg_eval_rhs(ctx, h)
    B.dg_mesh_free(ctx, h)
    assert np.abs(L).max() < 1e-11


def test_tet_device_state_io(B, ctx):
    torch = pytest.importorskip("torch")
    case, U, h, o = setup(B, ctx, "bump", 2, "fp32")
    dev = torch.zeros(U.shape, dtype=torch.float32, device="cuda")
    B.dg_get_state_device(ctx, h, dev.data_ptr())
    B.dg_sync(ctx)
    assert np.array_equal(dev.cpu().numpy(), U.astype(np.float32))
    dev2 = dev * 2
    torch.cuda.synchronize()
    B.dg_set_state_device(ctx, h, dev2.data_ptr())
    assert np.array_equal(B.dg_get_state(ctx, h), 2 * U.astype(np.float32).astype(np.float64))
    B.dg_mesh_free(ctx, h)


def test_tet_argument_errors(B, ctx):
    r, s, t = B.dg_tet_reference_nodes(2)
    case = make_case3("bump", 2, r, s, t, size="tiny")
    m = case["mesh"]
    for kw in ({"prec": "bf16x3"}, {"prec": "tf32", "av_on": True}):
        p = B.make_params(u_inf=case["u_inf"], **kw)
        with pytest.raises(B.DgError) as e:
            B.dg_tet_mesh_upload(ctx, 2, m.EToV, m.bc, case["xyz"], p)
        assert e.value.status == B.DG_EINVAL
    r4, s4, t4 = B.dg_tet_reference_nodes(4)
    c4 = make_case3("box", 4, r4, s4, t4, size="tiny")
    with pytest.raises(B.DgError) as e:   # the tensor-core tetrahedral kernel covers N = 2, 3
        B.dg_tet_mesh_upload(ctx, 4, c4["mesh"].EToV, c4["mesh"].bc, c4["xyz"],
                             B.make_params(u_inf=c4["u_inf"], prec="tf32"))
    assert e.value.status == B.DG_EINVAL
    p = B.make_params(u_inf=case["u_inf"], prec="fp32")
    bad = m.bc.copy()
    bad[np.argwhere(m.bc == 0)[0][0], np.argwhere(m.bc == 0)[0][1]] = 1
    with pytest.raises(B.DgError):
        B.dg_tet_mesh_upload(ctx, 2, m.EToV, bad, case["xyz"], p)
    with pytest.raises(B.DgError):
        B.dg_tet_mesh_upload(ctx, 5, m.EToV, m.bc, case["xyz"], p)
    h = B.dg_tet_mesh_upload(ctx, 2, m.EToV, m.bc, case["xyz"], p)
    for call in (lambda: B.dg_prolong(ctx, h, h),
                 lambda: B.dg_batch_step(ctx, [h], [1e-3], 1)):
        with pytest.raises(B.DgError) as e:
            call()
        assert e.value.status == B.DG_EINVAL
    B.dg_mesh_free(ctx, h)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tet_autotune_keeps_state_and_results(B, ctx, prec):
    """The tile autotuner on a tetrahedral mesh: candidates timed, state
    unchanged, and the tuned tiles step bitwise like the default ones (each
    element's arithmetic is independent of its tile)."""
    case, U, h, o = setup(B, ctx, "bump", 3, prec, size="medium")
    dt = 0.5 * states.time_step3(case["mesh"].verts, U, 3)
    U0 = B.dg_get_state(ctx, h)
    best, table, _ = B.dg_autotune(ctx, h, 2)
    assert len(table) >= 2 and best in table and all(t > 0 for t in table.values()), table
    assert np.array_equal(B.dg_get_state(ctx, h), U0)
    B.dg_step(ctx, h, dt, 2)
    Ut = B.dg_get_state(ctx, h)
    B.dg_mesh_free(ctx, h)
    c2 = B.dg_create(0)
    try:
        m = case["mesh"]
        h2 = B.dg_tet_mesh_upload(c2, 3, m.EToV, m.bc, case["xyz"], B.make_params(u_inf=case["u_inf"], prec=prec))
        B.dg_set_state(c2, h2, U)
        B.dg_step(c2, h2, dt, 2)
        Ud = B.dg_get_state(c2, h2)
    finally:
        B.dg_destroy(c2)
    assert np.array_equal(Ut, Ud)


def test_tet_tf32_autotune_reports_fixed_tiles(B, ctx):
    """The tensor-core tetrahedral kernel has fixed tiles (the rows of its
    products): the autotuner times nothing and reports them."""
    for N, E in ((2, 16), (3, 8)):
        case, U, h, o = setup(B, ctx, "box", N, "tf32")
        best, table, _ = B.dg_autotune(ctx, h, 2)
        B.dg_mesh_free(ctx, h)
        assert best == E and table == {}

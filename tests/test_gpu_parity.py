"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the arithmetic behind them):
  * DG_FP64_DEBUG: the same discretisation in FP64 with a different summation
    order and mass-matrix factorisation -> agreement to round-off; relative
    max-norm <= 1e-11 of max |L| (free stream: <= 1e-12 of the term scale).
  * DG_FP32 right-hand side on the same FP32-representable state: FP32
    round-off (2^-24) over sums of N_q + 3 N_g terms, measured against the
    volume term that L is a small difference of -> <= 1e-5 of that term's
    norm per variable (1e-4 with artificial viscosity, which differentiates
    the state twice).
  * DG_FP32 after 100 SSP-RK3 steps of the vortex (K = 512, N = 2):
    relative L2 per conserved variable <= 1e-5 (the workload's bound).
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg import Oracle
from paper_1208_4772_gb300.inputs import meshes, states
from cases import make_case, rel_l2_per_var

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


def upload(B, ctx, case, prec, U=None):
    m = case["mesh"]
    p = B.make_params(u_inf=case["u_inf"], av_on=case["av"], prec=prec)
    h = B.dg_mesh_upload(ctx, case["N"], m.EToE, m.EToF, m.bc, case["xy"], p)
    B.dg_set_state(ctx, h, case["U"] if U is None else U)
    return h


def oracle_of(case):
    m = case["mesh"]
    return Oracle(case["N"], m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=case["av"])


CASES = [("vortex", N, False) for N in (2, 3, 4, 5, 6)] + \
        [("naca", 4, False), ("naca", 4, True), ("cyl", 6, False), ("cyl", 3, True), ("vortex", 3, True)]


@pytest.mark.parametrize("kind,N,av", CASES)
def test_rhs_fp64_matches_oracle(B, ctx, kind, N, av):
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    h = upload(B, ctx, case, "fp64")
    L = B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
    B.dg_mesh_free(ctx, h)
    Lo = oracle_of(case).rhs(case["U"])
    assert np.abs(L - Lo).max() <= 1e-11 * np.abs(Lo).max()


def term_scale(o, U):
    """Per-variable L2 norm of the volume term M^-1 (S_x F + S_y G): the size
    of the quantities whose difference is L."""
    _, vol, _ = o.rhs(U, parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry(None).Minv, vol)
    return np.linalg.norm(V.transpose(1, 0, 2).reshape(4, -1), axis=1)


@pytest.mark.parametrize("kind,N,av", CASES)
def test_rhs_fp32_matches_oracle(B, ctx, kind, N, av):
    """FP32 right-hand side against the oracle on the same (FP32-representable)
    state.  L is a difference of volume and surface terms that are 30-250x
    larger than L for these smooth states, so the FP32 round-off is bounded
    relative to the volume term: <= 1e-5 of its norm (N_q + 3 N_g FP32 terms
    at 2^-24); with artificial viscosity the state is differentiated twice
    (q, then div q), so <= 1e-4."""
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    case["U"] = case["U"].astype(np.float32).astype(np.float64)
    h = upload(B, ctx, case, "fp32")
    L = B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
    B.dg_mesh_free(ctx, h)
    o = oracle_of(case)
    Lo = o.rhs(case["U"])
    err = np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(4, -1), axis=1) / term_scale(o, case["U"])
    assert np.all(err <= (1e-4 if av else 1e-5)), err


@pytest.mark.parametrize("kind,N", [("naca", 4), ("cyl", 6), ("naca", 2)])
def test_free_stream_curved_gpu(B, ctx, kind, N):
    """L(U_inf) = 0 on the curved mesh with farfield boundaries."""
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s)
    m = case["mesh"]
    m.bc = np.where(m.bc != 0, 2, 0).astype(np.int8)
    U = states.uniform_state(m.K, len(r), case["u_inf"])
    _, vol, _ = oracle_of(case).rhs(U, parts=True)
    Minv = oracle_of(case).geometry(None).Minv
    scale = np.abs(np.einsum('kij,kvj->kvi', Minv, vol)).max()
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        h = upload(B, ctx, case, prec, U)
        L = B.dg_eval_rhs(ctx, h, m.K, len(r))
        B.dg_mesh_free(ctx, h)
        assert np.abs(L).max() <= tol * scale, prec


def test_vortex_100_steps(B, ctx):
    """Isentropic vortex, periodic [0,10]^2, 2x16x16 jittered triangles,
    N = 2, LLF, SSP-RK3 at CFL 0.3, 100 steps: FP32 within 1e-5 relative L2
    per variable of the FP64 oracle, FP64 within 1e-12."""
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
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-12)):
        h = upload(B, ctx, case, prec)
        B.dg_step(ctx, h, dt, 100)
        Ug = B.dg_get_state(ctx, h, m.K, len(r))
        B.dg_mesh_free(ctx, h)
        err = rel_l2_per_var(Ug, Uo)
        assert np.all(err <= tol), (prec, err)


@pytest.mark.parametrize("kind,N,av", [("naca", 4, True), ("cyl", 5, False)])
def test_steps_curved(B, ctx, kind, N, av):
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    m = case["mesh"]
    dt = 0.5 * states.time_step(m.verts, case["U"], N, eps0=0.3 if av else None)
    o = oracle_of(case)
    Uo = case["U"].copy()
    for _ in range(5):
        Uo = o.ssp_rk3_step(Uo, dt)
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-11)):
        h = upload(B, ctx, case, prec)
        B.dg_step(ctx, h, dt, 5)
        Ug = B.dg_get_state(ctx, h, m.K, len(r))
        B.dg_mesh_free(ctx, h)
        if prec == "fp64":   # the increment itself is resolved only in FP64
            assert np.all(rel_l2_per_var(Ug - case["U"], Uo - case["U"]) <= 1e-9), prec
        assert np.all(rel_l2_per_var(Ug, Uo) <= tol), prec


def test_residual_matches_oracle(B, ctx):
    N = 3
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, av=True)
    Lo = oracle_of(case).rhs(case["U"])
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-5)):
        h = upload(B, ctx, case, prec)
        linf, l2 = B.dg_residual(ctx, h)
        B.dg_mesh_free(ctx, h)
        assert np.allclose(linf, np.abs(Lo).max(axis=(0, 2)), rtol=tol * 10)
        assert np.allclose(l2, np.sqrt((Lo ** 2).sum(axis=(0, 2))), rtol=tol * 10)


def test_batch_equals_single(B, ctx):
    """Meshes stepped together by the persistent batched kernel give the same
    state as each stepped alone (same kernels, same order inside a tile)."""
    cases = []
    for i, (kind, N) in enumerate((("naca", 2), ("cyl", 3), ("vortex", 4), ("naca", 5), ("vortex", 2))):
        r, s = B.dg_reference_nodes(N)
        cases.append(make_case(kind, N, r, s, seed=i))
    dts = [0.3 * states.time_step(c["mesh"].verts, c["U"], c["N"]) for c in cases]
    single = []
    for c, dt in zip(cases, dts):
        h = upload(B, ctx, c, "fp32")
        B.dg_step(ctx, h, dt, 3)
        single.append(B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2]))
        B.dg_mesh_free(ctx, h)
    hs = [upload(B, ctx, c, "fp32") for c in cases]
    B.dg_batch_step(ctx, hs, dts, 3)
    for h, c, Us in zip(hs, cases, single):
        Ub = B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2])
        assert np.array_equal(Ub, Us)
    for h in hs:
        B.dg_mesh_free(ctx, h)


def test_ragged_and_single_element(B, ctx):
    """K = 1 (three farfield faces), and K not a multiple of any tile size."""
    N = 4
    r, s = B.dg_reference_nodes(N)
    verts = np.array([[[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]])
    m = meshes.TriMesh("one", verts, np.array([[0, 1, 2]]))
    meshes.connect(m)
    xy = meshes.straight_nodes(verts, r, s)
    ui = states.freestream(0.3, 10.0)
    rng = np.random.default_rng(1)
    U = states.uniform_state(1, len(r), ui) * (1 + 0.05 * rng.standard_normal((1, 4, len(r))))
    case = dict(mesh=m, xy=xy, u_inf=ui, U=U, av=False, N=N)
    Lo = oracle_of(case).rhs(U)
    h = upload(B, ctx, case, "fp64")
    L = B.dg_eval_rhs(ctx, h, 1, len(r))
    B.dg_mesh_free(ctx, h)
    assert np.abs(L - Lo).max() <= 1e-11 * np.abs(Lo).max()
    for n in (5, 7):   # 50 and 98 elements
        case = make_case("vortex", N, r, s, size=n, av=True)
        Lo = oracle_of(case).rhs(case["U"])
        h = upload(B, ctx, case, "fp64")
        L = B.dg_eval_rhs(ctx, h, case["mesh"].K, len(r))
        B.dg_mesh_free(ctx, h)
        assert np.abs(L - Lo).max() <= 1e-11 * np.abs(Lo).max()


def test_device_state_roundtrip(B, ctx):
    torch = pytest.importorskip("torch")
    N = 3
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s)
    h = upload(B, ctx, case, "fp32")
    Ud = torch.tensor(case["U"], dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    B.dg_set_state_device(ctx, h, Ud.data_ptr())
    out = torch.zeros_like(Ud)
    B.dg_get_state_device(ctx, h, out.data_ptr())
    B.dg_sync(ctx, 10.0)
    assert torch.equal(out, Ud)
    host = B.dg_get_state(ctx, h, case["mesh"].K, len(r))
    assert np.array_equal(host, Ud.cpu().numpy().astype(np.float64))
    B.dg_mesh_free(ctx, h)


def test_rejects_bad_meshes(B, ctx):
    N = 2
    r, s = B.dg_reference_nodes(N)
    case = make_case("vortex", N, r, s, size="tiny")
    m = case["mesh"]
    p = B.make_params(prec="fp32")
    bad = m.EToE.copy()
    bad[0, 0] = (bad[0, 0] + 1) % m.K
    with pytest.raises(B.DgError) as e:
        B.dg_mesh_upload(ctx, N, bad, m.EToF, m.bc, case["xy"], p)
    assert e.value.status == B.DG_EINVAL
    mirrored = case["xy"].copy()          # mirror image: clockwise elements, J < 0
    mirrored[..., 0] *= -1.0
    with pytest.raises(B.DgError) as e:
        B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, mirrored, p)
    assert e.value.status == B.DG_EINVAL
    with pytest.raises(B.DgError):
        B.dg_mesh_upload(ctx, 7, m.EToE, m.EToF, m.bc, case["xy"], p)
    with pytest.raises(B.DgError) as e:
        B.dg_step(ctx, 12345, 0.1, 1)
    assert e.value.status == B.DG_ENOTFOUND


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotune_keeps_state_and_results(B, ctx, prec):
    """dg_autotune times the candidate tile sizes of the CUDA-core path,
    leaves the state as it was, and the tuned tiles step bitwise like the
    default ones (each element's arithmetic is the same; only its CTA
    changes).  A later mesh of the same kind in the context inherits the
    choice."""
    N = 4
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, av=True)
    dt = 0.1 * states.time_step(case["mesh"].verts, case["U"], N, eps0=0.3)
    K, Np = case["mesh"].K, len(r)
    h = upload(B, ctx, case, prec)
    U0 = B.dg_get_state(ctx, h, K, Np)
    best, table, _ = B.dg_autotune(ctx, h, 3)
    assert len(table) >= 2 and best in table and all(t > 0 for t in table.values()), table
    assert np.array_equal(B.dg_get_state(ctx, h, K, Np), U0)
    B.dg_step(ctx, h, dt, 3)
    Ut = B.dg_get_state(ctx, h, K, Np)
    B.dg_mesh_free(ctx, h)
    c2 = B.dg_create(0)          # a fresh context: default tile sizes
    try:
        h2 = upload(B, c2, case, prec)
        B.dg_step(c2, h2, dt, 3)
        Ud = B.dg_get_state(c2, h2, K, Np)
    finally:
        B.dg_destroy(c2)
    assert np.array_equal(Ut, Ud)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("tf32", 1e-4), ("bf16x3", 1e-5)])
def test_lserk_steps_match_oracle(B, ctx, prec, tol):
    """The paper's integrator, LSERK(5,4), fused into the stage kernels:
    50 vortex steps against the oracle's LSERK(5,4) (per-variable relative
    L2, the step tolerances of SSP-RK3)."""
    N = 3
    r, s = B.dg_reference_nodes(N)
    m = meshes.periodic_square(8, length=10.0, jitter=0.1, seed=1000)
    xy = meshes.straight_nodes(m.verts, r, s)
    U0 = states.vortex_state(xy, period=(10.0, 10.0))
    dt = states.time_step(m.verts, U0, N, cfl=0.3)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy)
    Uo = U0.copy()
    for _ in range(50):
        Uo = o.lserk54_step(Uo, dt)
    case = dict(mesh=m, xy=xy, u_inf=states.freestream(0.5), U=U0, av=False, N=N)
    h = upload(B, ctx, case, prec)
    B.dg_step_lserk(ctx, h, dt, 50)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    assert np.all(rel_l2_per_var(Ug, Uo) <= tol), rel_l2_per_var(Ug, Uo)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_lserk_with_viscosity_and_curved(B, ctx, prec):
    """LSERK(5,4) on a curved NACA mesh with artificial viscosity (sensor
    kernel every stage): 5 steps against the oracle; then an SSP-RK3 step on
    the same mesh still matches (eps of the new state is recomputed)."""
    N = 3
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, av=True)
    m = case["mesh"]
    dt = 0.2 * states.time_step(m.verts, case["U"], N, eps0=0.3)
    o = oracle_of(case)
    U = case["U"].astype(np.float32).astype(np.float64)
    h = upload(B, ctx, case, prec, U=U)
    B.dg_step_lserk(ctx, h, dt, 5)
    B.dg_step(ctx, h, dt, 1)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    Uo = U.copy()
    for _ in range(5):
        Uo = o.lserk54_step(Uo, dt)
    Uo = o.ssp_rk3_step(Uo, dt)
    tol = 1e-5 if prec == "fp32" else 1e-4
    assert np.all(rel_l2_per_var(Ug, Uo) <= tol), rel_l2_per_var(Ug, Uo)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5), ("tf32", 2e-3), ("bf16x3", 1e-5)])
@pytest.mark.parametrize("kind,N,av", [("vortex", 3, False), ("naca", 4, True), ("cyl", 5, False)])
def test_hllc_rhs_matches_oracle(B, ctx, prec, tol, kind, N, av):
    """The HLLC flux (dg_params.flux = 1) in the CUDA-core and tensor-core
    face phases against the oracle's HLLC, relative to the volume term."""
    r, s = B.dg_reference_nodes(N)
    case = make_case(kind, N, r, s, av=av)
    m = case["mesh"]
    U = case["U"].astype(np.float32).astype(np.float64)
    p = B.make_params(u_inf=case["u_inf"], av_on=av, prec=prec, flux="hllc")
    h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, case["xy"], p)
    B.dg_set_state(ctx, h, U)
    L = B.dg_eval_rhs(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    o = Oracle(N, m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=av, flux="hllc")
    Lo, vol, _ = o.rhs(U, parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry(None).Minv, vol)
    scale = np.linalg.norm(V.transpose(1, 0, 2).reshape(4, -1), axis=1)
    err = np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(4, -1), axis=1) / scale
    assert np.all(err <= tol), (kind, N, prec, err)
    # the selection is live: on the noisy curved cases (face jumps) the
    # result is ten times closer to the oracle's HLLC than to its LLF.  (On
    # the smooth vortex both fluxes reduce to the central flux; the TF32
    # error, ~1e-3 of the volume term, is of the size of the difference.)
    if kind != "vortex" and prec != "tf32":
        Ll = Oracle(N, m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"], av=av).rhs(U)
        assert np.linalg.norm(L - Lo) < 0.1 * np.linalg.norm(L - Ll)

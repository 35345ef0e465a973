"""dg_prolong (paper Sec. 5, p-refinement) against the oracle's
prolongation: the state of one upload of a mesh embedded into an upload of
the same mesh at a higher degree, on triangles and on tetrahedra.
FP64-debug to 1e-12, FP32 to 1e-6 (FP32 operator and sums); bad pairs are
refused."""
import numpy as np
import pytest

import __graft_entry__
from oracle.prefine import prolong_state
from paper_1208_4772_gb300.inputs import curving, meshes, states

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


def upload(B, ctx, mesh, N, prec, ui):
    r, s = B.dg_reference_nodes(N)
    xy, _ = curving.curve_mesh(mesh, N, r, s)
    p = B.make_params(u_inf=ui, prec=prec)
    return B.dg_mesh_upload(ctx, N, mesh.EToE, mesh.EToF, mesh.bc, xy, p), xy


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6), ("tf32", 1e-6)])
@pytest.mark.parametrize("N,M", [(2, 3), (3, 4), (2, 4), (4, 6)])
def test_prolong_matches_oracle(B, ctx, prec, tol, N, M):
    mesh = meshes.cylinder_channel(n_t=24, n_r=4, seed=1002)
    ui = states.freestream(0.38, 0.0)
    hN, xy = upload(B, ctx, mesh, N, prec, ui)
    hM, _ = upload(B, ctx, mesh, M, prec, ui)
    rng = np.random.default_rng(N + M)
    U = states.uniform_state(mesh.K, xy.shape[1], ui) * (1 + 0.05 * rng.standard_normal((mesh.K, 4, xy.shape[1])))
    B.dg_set_state(ctx, hN, U)
    Uin = B.dg_get_state(ctx, hN, mesh.K, xy.shape[1])      # as stored (FP32 rounding included)
    B.dg_prolong(ctx, hN, hM)
    Np_M = (M + 1) * (M + 2) // 2
    got = B.dg_get_state(ctx, hM, mesh.K, Np_M)
    ref = prolong_state(Uin, N, M)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    with pytest.raises(B.DgError):
        B.dg_prolong(ctx, hM, hN)          # to a lower degree
    B.dg_mesh_free(ctx, hN)
    B.dg_mesh_free(ctx, hM)


def test_prolong_refuses_other_mesh(B, ctx):
    ui = states.freestream(0.38, 0.0)
    m1 = meshes.cylinder_channel(n_t=24, n_r=4, seed=1002)
    m2 = meshes.cylinder_channel(n_t=24, n_r=5, seed=1002)
    h1, _ = upload(B, ctx, m1, 2, "fp32", ui)
    h2, _ = upload(B, ctx, m2, 3, "fp32", ui)
    with pytest.raises(B.DgError) as e:
        B.dg_prolong(ctx, h1, h2)
    assert e.value.status == B.DG_EINVAL
    B.dg_mesh_free(ctx, h1)
    B.dg_mesh_free(ctx, h2)


@pytest.mark.parametrize("kind", ["box", "wbox", "bump"])
@pytest.mark.parametrize("prec,tol,N,M", [("fp64", 1e-12, 2, 3), ("fp64", 1e-12, 2, 4), ("fp64", 1e-12, 3, 4),
                                          ("fp32", 1e-6, 2, 4), ("tf32", 1e-6, 2, 3)])
def test_prolong_tetrahedra_matches_oracle(B, ctx, kind, prec, tol, N, M):
    """The paper's own use (Sec. 5): 3D runs refined from p = 2 to 3 and 4.
    Two uploads of one tetrahedral mesh (affine, every element curved, or the
    bump channel, whose elements at the edge of the bump are curved at some
    degrees only, so that the two uploads order their elements differently);
    the prolonged state against the oracle's, then one SSP-RK3 step at the
    higher degree against the oracle's step of the prolonged state."""
    from cases import make_case3
    from oracle.dg3 import Oracle3
    from oracle.prefine import prolong_state3
    rN, sN, tN = B.dg_tet_reference_nodes(N)
    rM, sM, tM = B.dg_tet_reference_nodes(M)
    cN = make_case3(kind, N, rN, sN, tN)
    cM = make_case3(kind, M, rM, sM, tM)
    m = cN["mesh"]
    hN = B.dg_tet_mesh_upload(ctx, N, m.EToV, m.bc, cN["xyz"], B.make_params(u_inf=cN["u_inf"], prec=prec))
    mprec = "fp32" if (prec == "tf32" and M > 3) else prec
    hM = B.dg_tet_mesh_upload(ctx, M, m.EToV, m.bc, cM["xyz"], B.make_params(u_inf=cM["u_inf"], prec=mprec))
    B.dg_set_state(ctx, hN, cN["U"])
    Uin = B.dg_get_state(ctx, hN)
    B.dg_prolong(ctx, hN, hM)
    got = B.dg_get_state(ctx, hM)
    ref = prolong_state3(Uin, N, M)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    with pytest.raises(B.DgError):
        B.dg_prolong(ctx, hM, hN)          # to a lower degree
    dt = 0.25 * states.time_step3(m.verts, ref, M)
    B.dg_step(ctx, hM, dt, 1)
    U1 = B.dg_get_state(ctx, hM)
    B.dg_mesh_free(ctx, hN)
    B.dg_mesh_free(ctx, hM)
    ref1 = Oracle3(M, m.EToV, m.bc, cM["xyz"], u_inf=cM["u_inf"]).ssp_rk3_step(got, dt)
    step_tol = {"fp64": 1e-11, "fp32": 1e-5, "tf32": 1e-4}[prec]
    assert np.linalg.norm(U1 - ref1) / np.linalg.norm(ref1) < step_tol


def test_prolong_refuses_triangle_to_tetrahedron(B, ctx):
    from cases import make_case3
    ui = states.freestream(0.38, 0.0)
    m1 = meshes.cylinder_channel(n_t=24, n_r=4, seed=1002)
    h1, _ = upload(B, ctx, m1, 2, "fp32", ui)
    r, s, t = B.dg_tet_reference_nodes(3)
    c = make_case3("box", 3, r, s, t)
    h2 = B.dg_tet_mesh_upload(ctx, 3, c["mesh"].EToV, c["mesh"].bc, c["xyz"], B.make_params(u_inf=c["u_inf"]))
    with pytest.raises(B.DgError) as e:
        B.dg_prolong(ctx, h1, h2)
    assert e.value.status == B.DG_EINVAL
    B.dg_mesh_free(ctx, h1)
    B.dg_mesh_free(ctx, h2)


def test_prefine_driver_on_tetrahedra(B, ctx):
    """The level driver on a tetrahedral mesh (the paper's 3D setting, Sec. 5:
    p = 2, then 3): its final state equals the same sequence done by hand --
    freestream at N = 2, the level's steps, dg_prolong to N = 3, its steps --
    bitwise."""
    from paper_1208_4772_gb300 import prefine
    from paper_1208_4772_gb300.inputs import meshes3d
    m = meshes3d.bump_channel(6, 3, 4, seed=2000)
    ui = states.freestream3(0.5, 0.0)
    h, rep = prefine.run_levels(ctx, m, [2, 3], ui, prec="fp32", drop=1e-3, check_every=25, max_steps=50)
    assert [r["N"] for r in rep] == [2, 3] and all(r["steps"] == 50 for r in rep)
    assert all(np.isfinite(r["r_last"]) for r in rep)
    U = B.dg_get_state(ctx, h)
    B.dg_mesh_free(ctx, h)
    hs = []
    for N in (2, 3):
        r, s, t = B.dg_tet_reference_nodes(N)
        X = meshes3d.node_coords(m, r, s, t)
        hs.append(B.dg_tet_mesh_upload(ctx, N, m.EToV, m.bc, X, B.make_params(u_inf=ui, prec="fp32")))
    B.dg_set_state(ctx, hs[0], states.uniform_state3(m.K, 10, ui))
    B.dg_step(ctx, hs[0], rep[0]["dt"], 50)
    B.dg_prolong(ctx, hs[0], hs[1])
    B.dg_step(ctx, hs[1], rep[1]["dt"], 50)
    Uh = B.dg_get_state(ctx, hs[1])
    for x in hs:
        B.dg_mesh_free(ctx, x)
    assert U.shape == (m.K, 5, 20)
    assert np.array_equal(U, Uh)


def test_prefine_driver_on_triangles(B, ctx):
    """The level driver on a curved triangle mesh (the workloads' setting):
    its final state equals the same sequence done by hand -- freestream at
    N = 2, the level's steps, dg_prolong to N = 3, its steps -- bitwise."""
    from paper_1208_4772_gb300 import prefine
    from paper_1208_4772_gb300.inputs import curving, meshes
    m = meshes.cylinder_channel(n_t=24, n_r=6, seed=1002)
    ui = states.freestream(0.38, 0.0)
    h, rep = prefine.run_levels(ctx, m, [2, 3], ui, prec="fp32", drop=1e-3, check_every=25, max_steps=50)
    assert [r["N"] for r in rep] == [2, 3] and all(r["steps"] == 50 for r in rep)
    assert all(np.isfinite(r["r_last"]) for r in rep)
    U = B.dg_get_state(ctx, h, m.K, 10)
    B.dg_mesh_free(ctx, h)
    hs = []
    for N in (2, 3):
        r, s = B.dg_reference_nodes(N)
        xy, _ = curving.curve_mesh(m, N, r, s)
        hs.append(B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, xy, B.make_params(u_inf=ui, prec="fp32")))
    B.dg_set_state(ctx, hs[0], states.uniform_state(m.K, 6, ui))
    B.dg_step(ctx, hs[0], rep[0]["dt"], 50)
    B.dg_prolong(ctx, hs[0], hs[1])
    B.dg_step(ctx, hs[1], rep[1]["dt"], 50)
    Uh = B.dg_get_state(ctx, hs[1], m.K, 10)
    for x in hs:
        B.dg_mesh_free(ctx, x)
    assert U.shape == (m.K, 4, 10)
    assert np.array_equal(U, Uh)

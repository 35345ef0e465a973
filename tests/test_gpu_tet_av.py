"""Artificial viscosity on tetrahedra (paper Sec. 2 with d = 3; the
paper's transonic 3D cases use it): the element sensor, the BR1 gradient
pass and the viscous terms of the CUDA-core stage kernel against the FP64
tetrahedral oracle.

The state is the curved bump channel's perturbed flow with a jump of all
variables by half across a plane, so that the elements the plane cuts sit
on the sensor's ramp (eps up to about 0.1) and the rest have eps = 0.  Tolerances: FP64 1e-11 of the volume term (round-off);
FP32 1e-4: the sensor's two sums run in FP32 (its ratio, logarithm and
ramp in FP64), which moves eps by ~1e-5 relative on elements on the ramp,
and the viscous terms inherit it (the bound of the triangle path).
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg3 import Oracle3
from paper_1208_4772_gb300.inputs import states
from cases import make_case3

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-4}


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


def av_case(B, N, size="small", kind="bump"):
    """The bump channel (432 elements), or the periodic box (162 elements, a
    ragged last tile), with the jump (box: across x = 4.1)."""
    r, s, t = B.dg_tet_reference_nodes(N)
    case = make_case3(kind, N, r, s, t, size=size)
    X = case["xyz"]
    U = case["U"].copy()
    U *= np.where(X[..., 0] > (1.37 if kind == "bump" else 4.1), 1.5, 1.0)[:, None, :]
    case["U"] = U.astype(np.float32).astype(np.float64)
    return case


def upload(B, ctx, case, N, prec, flux="llf"):
    m = case["mesh"]
    p = B.make_params(u_inf=case["u_inf"], prec=prec, flux=flux, av_on=True)
    h = B.dg_tet_mesh_upload(ctx, N, m.EToV, m.bc, case["xyz"], p)
    B.dg_set_state(ctx, h, case["U"])
    return h


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("flux", ["llf", "hllc"])
@pytest.mark.parametrize("kind,N", [("bump", 2), ("bump", 3), ("bump", 4), ("box", 2), ("box", 3)])
def test_tet_av_rhs_matches_oracle(B, ctx, kind, N, flux, prec):
    case = av_case(B, N, kind=kind)
    m = case["mesh"]
    h = upload(B, ctx, case, N, prec, flux)
    L = B.dg_eval_rhs(ctx, h)
    B.dg_mesh_free(ctx, h)
    o = Oracle3(N, m.EToV, m.bc, case["xyz"], u_inf=case["u_inf"], flux=flux, av=True)
    eps = o.sensor(case["U"])
    assert np.sum(eps > 0) > 0 and np.sum(eps == 0) > 0
    Lo, vol, _ = o.rhs(case["U"], parts=True)
    V = np.einsum('kij,kvj->kvi', o.geometry().Minv, vol)
    scale = np.linalg.norm(V.transpose(1, 0, 2).reshape(5, -1), axis=1)
    err = np.linalg.norm((L - Lo).transpose(1, 0, 2).reshape(5, -1), axis=1) / scale
    assert np.all(np.isfinite(L))
    assert np.all(err <= TOL[prec]), (N, flux, prec, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tet_av_count_matches_oracle_sensor(B, ctx, prec):
    N = 3
    case = av_case(B, N)
    m = case["mesh"]
    h = upload(B, ctx, case, N, prec)
    n = B.dg_av_count(ctx, h)
    B.dg_mesh_free(ctx, h)
    eps = Oracle3(N, m.EToV, m.bc, case["xyz"], u_inf=case["u_inf"], av=True).sensor(case["U"])
    if prec == "fp64":
        assert n == int(np.sum(eps > 0))
    else:   # FP32 sums: elements at the lower end of the ramp may flip
        assert abs(n - int(np.sum(eps > 0))) <= max(2, int(0.01 * m.K))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tet_av_steps_match_oracle(B, ctx, prec):
    N = 2
    case = av_case(B, N)
    m = case["mesh"]
    h = upload(B, ctx, case, N, prec)
    U = case["U"]
    dt = 0.25 * states.time_step3(m.verts, U, N)
    B.dg_step(ctx, h, dt, 2)
    B.dg_step_lserk(ctx, h, dt, 1)
    Ug = B.dg_get_state(ctx, h)
    B.dg_mesh_free(ctx, h)
    o = Oracle3(N, m.EToV, m.bc, case["xyz"], u_inf=case["u_inf"], av=True)
    Uo = U.copy()
    for _ in range(2):
        Uo = o.ssp_rk3_step(Uo, dt)
    Uo = o.lserk54_step(Uo, dt)
    nrm = np.linalg.norm(Uo.transpose(1, 0, 2).reshape(5, -1), axis=1)
    nrm[1:4] = np.linalg.norm(nrm[1:4])
    err = np.linalg.norm((Ug - Uo).transpose(1, 0, 2).reshape(5, -1), axis=1) / nrm
    assert np.all(err <= {"fp64": 1e-11, "fp32": 1e-5}[prec]), err


def test_tet_av_free_stream(B, ctx):
    """A uniform flow has eps = 0 and q = 0: L = 0 on the periodic box whose
    every element is curved."""
    N = 3
    r, s, t = B.dg_tet_reference_nodes(N)
    case = make_case3("wbox", N, r, s, t)
    m = case["mesh"]
    case["U"] = states.uniform_state3(m.K, len(r), case["u_inf"])
    h = upload(B, ctx, case, N, "fp64")
    assert B.dg_av_count(ctx, h) == 0
    L = B.dg_eval_rhs(ctx, h)
    B.dg_mesh_free(ctx, h)
    assert np.abs(L).max() < 1e-10

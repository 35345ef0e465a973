"""Artificial viscosity on the batched path (paper Sec. 2, the
Persson-Peraire sensor and viscosity; the batch of many meshes in one step
graph).

A batch mixes meshes with and without artificial viscosity: the ones with
viscosity run their own sensor / gradient / stage chains on branches of the
batched step graph, the others the shared persistent launches.  Checked:
every mesh ends in exactly the state dg_step gives it (bitwise), a state set
between batched steps is picked up (its sensor recomputed), and the meshes
with viscosity match the FP64 oracle's SSP-RK3 steps element by element
(relative to each element's state: FP32 and BF16 x3 1e-5, TF32 1e-4, as the
single-mesh step tests), on states with troubled cells.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg import Oracle
from paper_1208_4772_gb300.inputs import states
from cases import make_case

pytestmark = pytest.mark.gpu

STATE_TOL = {"fp32": 1e-5, "tf32": 1e-4, "bf16x3": 1e-5}


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


def batch_cases(B):
    cases = []
    for i, (kind, N, av) in enumerate((("naca", 4, True), ("vortex", 2, False), ("cyl", 3, True),
                                       ("naca", 5, False), ("vortex", 3, True))):
        r, s = B.dg_reference_nodes(N)
        c = make_case(kind, N, r, s, seed=20 + i, av=av)
        if av:   # troubled cells: every variable x1.5 beyond a line through the mesh
            x = c["xy"][..., 0]
            c["U"] = c["U"] * np.where(x > (5.0 if kind == "vortex" else 1.0), 1.5, 1.0)[:, None, :]
        c["U"] = c["U"].astype(np.float32).astype(np.float64)
        c["dt"] = 0.3 * states.time_step(c["mesh"].verts, c["U"], N, eps0=0.3 if av else None)
        cases.append(c)
    return cases


def upload(B, ctx, c, prec):
    m = c["mesh"]
    h = B.dg_mesh_upload(ctx, c["N"], m.EToE, m.EToF, m.bc, c["xy"],
                         B.make_params(u_inf=c["u_inf"], av_on=c["av"], prec=prec))
    B.dg_set_state(ctx, h, c["U"])
    return h


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_batch_with_viscosity_equals_single_mesh_steps(B, ctx, prec):
    cases = batch_cases(B)
    single = []
    for c in cases:
        h = upload(B, ctx, c, prec)
        B.dg_step(ctx, h, c["dt"], 2)
        B.dg_step(ctx, h, c["dt"], 1)
        single.append(B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2]))
        B.dg_mesh_free(ctx, h)
    hs = [upload(B, ctx, c, prec) for c in cases]
    assert all(B.dg_av_count(ctx, h) > 0 for h, c in zip(hs, cases) if c["av"])
    B.dg_batch_step(ctx, hs, [c["dt"] for c in cases], 2)
    B.dg_batch_step(ctx, hs, [c["dt"] for c in cases], 1)
    for h, c, Us in zip(hs, cases, single):
        Ub = B.dg_get_state(ctx, h, c["mesh"].K, c["U"].shape[2])
        assert np.array_equal(Ub, Us), (c["name"], c["N"], c["av"], np.abs(Ub - Us).max())
    # a state set between batched steps: its sensor is recomputed before the next step
    c0 = cases[0]
    U1 = c0["U"] * (1.0 + 1e-3 * np.cos(c0["xy"][..., 0]))[:, None, :]
    B.dg_set_state(ctx, hs[0], U1)
    B.dg_batch_step(ctx, hs, [c["dt"] for c in cases], 1)
    Ua = B.dg_get_state(ctx, hs[0], c0["mesh"].K, c0["U"].shape[2])
    for h in hs:
        B.dg_mesh_free(ctx, h)
    h = upload(B, ctx, dict(c0, U=U1), prec)
    B.dg_step(ctx, h, c0["dt"], 1)
    Ub = B.dg_get_state(ctx, h, c0["mesh"].K, c0["U"].shape[2])
    B.dg_mesh_free(ctx, h)
    assert np.array_equal(Ua, Ub)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_batch_with_viscosity_matches_oracle(B, ctx, prec):
    cases = batch_cases(B)
    hs = [upload(B, ctx, c, prec) for c in cases]
    B.dg_batch_step(ctx, hs, [c["dt"] for c in cases], 2)
    worst = []
    for h, c in zip(hs, cases):
        m = c["mesh"]
        U = B.dg_get_state(ctx, h, m.K, c["U"].shape[2])
        B.dg_mesh_free(ctx, h)
        o = Oracle(c["N"], m.EToE, m.EToF, m.bc, c["xy"], u_inf=c["u_inf"], av=c["av"])
        Uo = c["U"].copy()
        for _ in range(2):
            Uo = o.ssp_rk3_step(Uo, c["dt"])
        per_elt = np.linalg.norm(U - Uo, axis=(1, 2)) / np.linalg.norm(Uo, axis=(1, 2))
        worst.append((c["name"], c["N"], c["av"], "%.2e" % per_elt.max()))
        assert np.all(np.isfinite(U))
        assert per_elt.max() <= STATE_TOL[prec], worst[-1]
    print("\nbatch with viscosity %s: %s" % (prec, worst))

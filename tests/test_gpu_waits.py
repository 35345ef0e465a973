"""Failure detection without a GPU fault: every device-side wait of the
library is bounded, and the host-side wait of dg_sync has a timeout.

* A bounded mbarrier wait on which nothing arrives runs out after its poll
  limit and reports it (the kernel returns; no hang, no trap), while the
  same wait with its arrival completes; the context stays usable and the
  next step matches the oracle.
* dg_sync with a timeout shorter than the enqueued work returns DG_ETIMEOUT
  without cancelling it; an unbounded dg_sync then completes and the state
  is that of the full run.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle.dg import Oracle
from cases import make_case

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


def test_bounded_wait_runs_out_and_context_survives(B, ctx):
    assert B.dg_selftest_bounded_wait(ctx, 1000, 0) == 1
    assert B.dg_selftest_bounded_wait(ctx, 1000, 1) == 0
    with pytest.raises(B.DgError) as e:
        B.dg_selftest_bounded_wait(ctx, 0, 0)
    assert e.value.status == B.DG_EINVAL
    # the context still computes correctly after the wait that ran out
    N = 3
    r, s = B.dg_reference_nodes(N)
    case = make_case("vortex", N, r, s, size="tiny")
    m = case["mesh"]
    U = case["U"].astype(np.float32).astype(np.float64)
    h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, case["xy"], B.make_params(u_inf=case["u_inf"], prec="tf32"))
    B.dg_set_state(ctx, h, U)
    dt = 1e-3
    B.dg_step(ctx, h, dt, 1)
    B.dg_sync(ctx)
    Ug = B.dg_get_state(ctx, h, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    ref = Oracle(N, m.EToE, m.EToF, m.bc, case["xy"], u_inf=case["u_inf"]).ssp_rk3_step(U, dt)
    assert np.linalg.norm(Ug - ref) / np.linalg.norm(ref) < 1e-4


def test_sync_timeout_leaves_work_running(B, ctx):
    N = 4
    r, s = B.dg_reference_nodes(N)
    case = make_case("naca", N, r, s, size="config", av=True)
    m = case["mesh"]
    U = case["U"].astype(np.float32).astype(np.float64)
    h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, case["xy"],
                         B.make_params(u_inf=case["u_inf"], av_on=True, prec="tf32"))
    B.dg_set_state(ctx, h, U)
    dt = 1e-10                          # below the mesh's stable step (about 2e-10: thin wall cells)
    B.dg_step(ctx, h, dt, 1)            # graph built and run once
    B.dg_sync(ctx)
    B.dg_step(ctx, h, dt, 400)          # tens of milliseconds of device work
    with pytest.raises(B.DgError) as e:
        B.dg_sync(ctx, 1e-4)
    assert e.value.status == B.DG_ETIMEOUT
    B.dg_sync(ctx)                      # unbounded: completes
    U1 = B.dg_get_state(ctx, h, m.K, len(r))
    assert np.all(np.isfinite(U1))
    # the run was not cancelled: a fresh upload stepped 401 times agrees
    h2 = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, case["xy"],
                          B.make_params(u_inf=case["u_inf"], av_on=True, prec="tf32"))
    B.dg_set_state(ctx, h2, U)
    B.dg_step(ctx, h2, dt, 401)
    U2 = B.dg_get_state(ctx, h2, m.K, len(r))
    B.dg_mesh_free(ctx, h)
    B.dg_mesh_free(ctx, h2)
    assert np.array_equal(U1, U2)

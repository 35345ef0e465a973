"""Serving loop on the GPU: requests of different sizes and degrees arrive
while others run, are admitted under an HBM budget, share the persistent
batched launches, and each result equals the same request run alone for
the same number of steps (same tile code, so bit-for-bit)."""
import numpy as np
import pytest

import __graft_entry__

pytestmark = pytest.mark.gpu


def test_serve_mix_equals_alone():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B
    from paper_1208_4772_gb300 import serve
    B.load()
    reqs = serve.poisson_requests(8, rate=400.0, seed=11, K_range=(300, 4000), N_range=(2, 5))
    for r in reqs:
        rr, ss = B.dg_reference_nodes(r.N)
        serve.prepare(r, rr, ss)
    budget = 2.5 * max(serve.estimate_bytes(r.K, r.N, curved=int(np.any(r.mesh.bc == 1, axis=1).sum()))
                       for r in reqs)
    ctx = B.dg_create(0)
    try:
        loop = serve.ServeLoop(ctx, budget_bytes=budget, check_every=20, max_steps=60, drop=1e-12)
        done = loop.run(reqs)
        assert len(done) == len(reqs)
        assert loop.peak_used <= budget
        assert loop.peak_active >= 2
        for r in done:
            assert r.reason in ("max_steps", "converged") and r.finished > r.arrival
        stats = serve.latency_stats(done)
        assert 0 < stats["p50_s"] <= stats["p99_s"]
        for r in done:
            p = B.make_params(u_inf=r.u_inf, prec="fp32")
            m = r.mesh
            h = B.dg_mesh_upload(ctx, r.N, m.EToE, m.EToF, m.bc, r.xy, p)
            assert B.dg_mesh_bytes(ctx, h) == r.bytes
            B.dg_set_state(ctx, h, r.U0)
            B.dg_step(ctx, h, r.dt, r.steps)
            alone = B.dg_get_state(ctx, h, m.K, r.Np)
            B.dg_mesh_free(ctx, h)
            assert np.array_equal(alone, r.extra["state"]), r.rid
    finally:
        B.dg_destroy(ctx)


def test_estimate_matches_library():
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B
    from paper_1208_4772_gb300 import serve
    ctx = B.dg_create(0)
    try:
        for kind, N in (("naca", 3), ("cyl", 5)):
            r = serve.Request(rid=0, arrival=0.0, kind=kind, n_t=40, n_r=6, N=N, mach=0.5, aoa=1.0)
            rr, ss = B.dg_reference_nodes(N)
            serve.prepare(r, rr, ss)
            h = B.dg_mesh_upload(ctx, N, r.mesh.EToE, r.mesh.EToF, r.mesh.bc, r.xy, B.make_params(u_inf=r.u_inf))
            curved = int(np.any(r.mesh.bc == 1, axis=1).sum())
            assert B.dg_mesh_bytes(ctx, h) == serve.estimate_bytes(r.K, N, curved=curved)
            B.dg_mesh_free(ctx, h)
    finally:
        B.dg_destroy(ctx)

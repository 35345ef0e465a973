"""Host logic of the continuous-batching loop against a fake library: HBM
budget admission, retirement on convergence / step cap / non-finite
residual, and latency accounting.  The failure (a NaN residual) is injected
on the host; nothing runs on a GPU."""
import math

import numpy as np
import pytest

from paper_1208_4772_gb300 import serve


class FakeLib:
    """Stands in for the binding: each mesh's residual decays by a factor
    per step; mesh 'bad' returns NaN."""

    def __init__(self, decay=0.5, bad=()):
        self.decay = decay
        self.bad = set(bad)
        self.meshes = {}
        self.next = 1
        self.batches = []

    def make_params(self, **kw):
        return kw

    def dg_mesh_upload(self, ctx, N, EToE, EToF, bc, xy, p):
        h = self.next
        self.next += 1
        self.meshes[h] = dict(K=EToE.shape[0], N=N, steps=0, rid=p.get("rid"))
        return h

    def dg_mesh_prepare(self, N, EToE, EToF, bc, xy, p):
        return ("prepared", N, EToE, p)

    def dg_mesh_upload_prepared(self, ctx, prep):
        _, N, EToE, p = prep
        return self.dg_mesh_upload(ctx, N, EToE, None, None, None, p)

    def dg_prepared_free(self, prep):
        pass

    def dg_batch_residual(self, ctx, hs, allow_nonfinite=False):
        res = [self.dg_residual(ctx, h) for h in hs]
        return np.array([a for a, _ in res]), np.array([b for _, b in res])

    def dg_set_state(self, ctx, h, U):
        self.meshes[h]["U"] = U

    def dg_mesh_bytes(self, ctx, h):
        m = self.meshes[h]
        return serve.estimate_bytes(m["K"], m["N"])

    def dg_batch_step(self, ctx, hs, dts, n):
        self.batches.append([self.meshes[h]["K"] for h in hs])
        for h in hs:
            self.meshes[h]["steps"] += n

    def dg_residual(self, ctx, h, allow_nonfinite=False):
        m = self.meshes[h]
        if m["K"] in self.bad:
            return np.full(4, np.nan), np.full(4, np.nan)
        r = self.decay ** m["steps"]
        return np.full(4, r), np.full(4, r)

    def dg_get_state(self, ctx, h, K, Np):
        return self.meshes[h]["U"]

    def dg_mesh_free(self, ctx, h):
        del self.meshes[h]


def fake_request(rid, arrival, K, N=2):
    n_r = 2
    n_t = K // (2 * n_r)
    r = serve.Request(rid=rid, arrival=arrival, kind="naca", n_t=n_t, n_r=n_r, N=N, mach=0.5, aoa=0.0)

    class M:
        pass
    r.mesh = M()
    r.mesh.K = r.K
    r.mesh.EToE = np.zeros((r.K, 3), np.int32)
    r.mesh.EToF = np.zeros((r.K, 3), np.int8)
    r.mesh.bc = np.zeros((r.K, 3), np.int8)
    r.xy = None
    r.U0 = np.zeros((r.K, 4, r.Np))
    r.u_inf = np.array([1.0, 0.5, 0.0, 2.0])
    r.dt = 1e-3
    return r


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def test_budget_admission_and_retirement(monkeypatch):
    fake = FakeLib(decay=0.5, bad={400})
    monkeypatch.setattr(serve, "B", fake)
    reqs = [fake_request(0, 0.0, 800), fake_request(1, 0.0, 800), fake_request(2, 0.0, 400),
            fake_request(3, 0.0, 800)]
    one = serve.estimate_bytes(800, 2)
    loop = serve.ServeLoop(ctx=None, budget_bytes=2.5 * one, check_every=10, max_steps=200, drop=1e-6,
                           clock=Clock())
    done = loop.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    assert loop.peak_used <= 2.5 * one
    # never more than two 800-element meshes resident at once
    for b in fake.batches:
        assert sum(K == 800 for K in b) <= 2
    assert max(len(b) for b in fake.batches) >= 2          # requests overlapped on the device
    reasons = {r.rid: r.reason for r in done}
    assert reasons[2] == "nonfinite"
    assert reasons[0] == reasons[1] == reasons[3] == "converged"
    # 0.5^steps <= 1e-6 * 0.5^10 needs 30 steps after the first check
    assert all(r.steps == 30 for r in done if r.reason == "converged")
    # the last 800-element request waited for memory
    r3 = [r for r in done if r.rid == 3][0]
    assert r3.admitted > r3.arrival
    assert all(r.finished > r.arrival for r in done)
    stats = serve.latency_stats(done)
    assert stats["p50_s"] <= stats["p99_s"]


def test_step_cap_and_oversized_request(monkeypatch):
    fake = FakeLib(decay=1.0)
    monkeypatch.setattr(serve, "B", fake)
    reqs = [fake_request(0, 0.0, 400)]
    loop = serve.ServeLoop(ctx=None, budget_bytes=1e12, check_every=7, max_steps=50, clock=Clock())
    done = loop.run(reqs)
    assert done[0].reason == "max_steps" and done[0].steps == 50
    loop = serve.ServeLoop(ctx=None, budget_bytes=10.0, clock=Clock())
    with pytest.raises(ValueError):
        loop.run([fake_request(1, 0.0, 400)])


def test_poisson_requests_shapes():
    reqs = serve.poisson_requests(200, rate=5.0, seed=3, K_range=(1000, 500000))
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert abs(1.0 / np.mean(np.diff(arr)) - 5.0) < 1.5
    Ks = np.array([r.K for r in reqs])
    assert Ks.min() >= 800 and Ks.max() <= 520000
    assert set(r.N for r in reqs) <= {2, 3, 4, 5, 6}
    assert math.isclose(np.mean(np.log(Ks)), 0.5 * (math.log(1000) + math.log(500000)), rel_tol=0.1)


class FakeLibNeedsViscosity(FakeLib):
    """A mesh without artificial viscosity returns a NaN residual (its flow
    develops a shock); with viscosity of at least `need` it converges."""

    def __init__(self, need):
        super().__init__(decay=0.5)
        self.need = need

    def dg_mesh_upload(self, ctx, N, EToE, EToF, bc, xy, p):
        h = super().dg_mesh_upload(ctx, N, EToE, EToF, bc, xy, p)
        self.meshes[h]["eps0"] = p.get("eps0", 0.0) if p.get("av_on") else 0.0
        return h

    def dg_residual(self, ctx, h, allow_nonfinite=False):
        if self.meshes[h]["eps0"] < self.need:
            return np.full(4, np.nan), np.full(4, np.nan)
        return super().dg_residual(ctx, h)


def with_geometry(r):
    """Vertices and a finite freestream state for the viscosity strength."""
    K = r.K
    r.mesh.verts = np.tile(np.array([[0.0, 0.0], [0.001, 0.0], [0.0, 0.001]]), (K, 1, 1))
    r.U0 = np.zeros((K, 4, r.Np))
    r.U0[:, 0], r.U0[:, 1], r.U0[:, 3] = 1.0, 0.5, 2.0
    return r


def test_nonfinite_requests_restart_with_more_viscosity(monkeypatch):
    """A request that turns non-finite is restarted from its initial state
    with artificial viscosity, then with ten times more, until it is finite
    (here on the second restart) or the retries run out."""
    r = with_geometry(fake_request(0, 0.0, 400))
    eps_first = serve.av_eps0(r.mesh, r.U0, r.N)
    fake = FakeLibNeedsViscosity(need=5 * eps_first)
    monkeypatch.setattr(serve, "B", fake)
    loop = serve.ServeLoop(ctx=None, budget_bytes=1e12, check_every=10, max_steps=500, clock=Clock(), workers=0)
    done = loop.run([r])
    assert done[0].reason == "converged" and done[0].retries == 2 and done[0].av
    assert math.isclose(done[0].eps0, 10 * eps_first)
    r2 = with_geometry(fake_request(1, 0.0, 400))
    fake = FakeLibNeedsViscosity(need=1.0)          # more than the cap 0.3: never finite
    monkeypatch.setattr(serve, "B", fake)
    loop = serve.ServeLoop(ctx=None, budget_bytes=1e12, check_every=10, max_steps=500, clock=Clock(), workers=0,
                           max_retries=5)
    done = loop.run([r2])
    assert done[0].reason == "nonfinite" and done[0].eps0 == 0.3


class SlowFakeLib(FakeLib):
    """Host half of an upload and each chunk of steps take real time (the
    residual read is where the loop waits for the device)."""

    def dg_mesh_prepare(self, N, EToE, EToF, bc, xy, p):
        import time
        time.sleep(0.05)
        return super().dg_mesh_prepare(N, EToE, EToF, bc, xy, p)

    def dg_batch_residual(self, ctx, hs, allow_nonfinite=False):
        import time
        time.sleep(0.01)
        return super().dg_batch_residual(ctx, hs, allow_nonfinite)


def test_host_preparation_overlaps_device_steps(monkeypatch):
    """A request that arrives while another is being stepped gets the host
    half of its upload on a worker thread at its arrival, and that work
    runs while the loop keeps stepping the active request (the event trace
    shows preparation inside stepping intervals); it is admitted once its
    host half is done."""
    import time
    fake = SlowFakeLib(decay=0.97)
    monkeypatch.setattr(serve, "B", fake)
    reqs = [fake_request(0, 0.0, 400), fake_request(1, 0.15, 400)]
    loop = serve.ServeLoop(ctx=None, budget_bytes=1e12, check_every=10, max_steps=1000, clock=time.perf_counter,
                           workers=2)
    done = loop.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1]
    ov = loop.overlap()
    assert ov["prepare_s"] > 0.08 and ov["prepare_during_steps_s"] > 0.02, ov
    starts = {rid: t for t, ev, rid in loop.trace if ev == "prepare_start"}
    assert starts[1] >= 0.15                      # not before the request arrived
    r1 = [r for r in done if r.rid == 1][0]
    assert r1.admitted >= starts[1] + 0.05        # after its host half
    assert max(len(b) for b in fake.batches) == 2

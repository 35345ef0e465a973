"""Continuous-batching request loop for steady-state flow solves.

Requests (a mesh, a degree, a flow condition) arrive over time.  The loop
admits a request as soon as it has arrived and its device bytes fit in the
HBM budget, keeps its state resident on the device, advances every admitted
request together with one persistent batched launch per Runge-Kutta stage
(``dg_batch_step``, replayed from a CUDA graph that is re-captured when the
active set changes), checks each request's FP64 residual every
``check_every`` steps and retires it when the residual has dropped by
``drop`` relative to its first check or it reaches ``max_steps``.  Latency
is measured from arrival to retirement.

Host set-up of a request (mesh generation, wall curving) happens before its
arrival time; admission covers the upload to the device.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from .inputs import curving, meshes, states


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    kind: str                      # "naca" or "cyl"
    n_t: int
    n_r: int
    N: int
    mach: float
    aoa: float
    seed: int = 0
    # filled by the loop
    mesh: object = None
    xy: np.ndarray = None
    U0: np.ndarray = None
    u_inf: np.ndarray = None
    dt: float = 0.0
    handle: int = -1
    bytes: int = 0
    steps: int = 0
    r0: float = math.nan
    r_last: float = math.nan
    admitted: float = math.nan
    finished: float = math.nan
    reason: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return 2 * self.n_t * self.n_r

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2


def prepare(req, r, s):
    """Host FP64 set-up: seeded mesh, curved nodes, freestream state, dt."""
    if req.kind == "naca":
        m = meshes.naca_omesh(n_t=req.n_t, n_r=req.n_r, seed=req.seed)
    else:
        m = meshes.cylinder_channel(n_t=req.n_t, n_r=req.n_r, seed=req.seed)
    xy, _ = curving.curve_mesh(m, req.N, r, s)
    req.mesh, req.xy = m, xy
    req.u_inf = states.freestream(req.mach, req.aoa)
    req.U0 = states.uniform_state(m.K, len(r), req.u_inf)
    req.dt = states.time_step(m.verts, req.U0, req.N, cfl=0.3)
    return req


def estimate_bytes(K, N, curved=0, prec_bytes=4, av=False, tensor=False):
    """Device bytes dg_mesh_upload allocates for a mesh (without the shared
    operator tables): three state buffers and the right-hand-side scratch,
    connectivity, geometry, permutation maps, reduction scratch; with AV eps
    (three copies on the tensor-core path) and q."""
    Np = (N + 1) * (N + 2) // 2
    q = (3 * N + 2) // 2
    Nq, Nf = q * q, 3 * q
    b = 4 * K * 4 * Np * prec_bytes              # U^n, two stage buffers, L
    b += K * 16                                  # connectivity
    b += (K - curved) * 4 * prec_bytes           # affine geometry
    b += curved * (5 * Nq + 3 * Nf + Np * Np) * prec_bytes
    b += 2 * K * 8                               # permutation maps
    b += (304 * 10 + 10) * 8 + 64                # reduction scratch, error words, counters
    if av:
        b += (3 if tensor else 1) * ((K + 31) // 32 * 32) * prec_bytes    # eps padded to whole tiles
        b += K * 8 * Np * prec_bytes
    return b


def poisson_requests(n, rate, seed=0, K_range=(1000, 500000), N_range=(2, 6), mach=(0.3, 0.85),
                     aoa=(-2.0, 4.0)):
    """n requests with exponential inter-arrival times (rate per second),
    K log-uniform in K_range, N uniform in N_range, alternating airfoil and
    cylinder geometries."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        K = math.exp(rng.uniform(math.log(K_range[0]), math.log(K_range[1])))
        n_r = max(2, int(round(math.sqrt(K / 6.0))))
        n_t = max(8, int(round(K / (2 * n_r))))
        reqs.append(Request(rid=i, arrival=float(t[i]), kind="naca" if i % 2 == 0 else "cyl", n_t=n_t, n_r=n_r,
                            N=int(rng.integers(N_range[0], N_range[1] + 1)),
                            mach=float(rng.uniform(*mach)), aoa=float(rng.uniform(*aoa)), seed=3000 + i))
    return reqs


class ServeLoop:
    def __init__(self, ctx, budget_bytes=150e9, check_every=100, max_steps=20000, drop=1e-6, prec="fp32",
                 clock=time.perf_counter):
        self.ctx = ctx
        self.budget = float(budget_bytes)
        self.check_every = int(check_every)
        self.max_steps = int(max_steps)
        self.drop = float(drop)
        self.prec = prec
        self.clock = clock
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0

    def _admit(self, req, now):
        p = B.make_params(u_inf=req.u_inf, prec=self.prec)
        m = req.mesh
        req.handle = B.dg_mesh_upload(self.ctx, req.N, m.EToE, m.EToF, m.bc, req.xy, p)
        B.dg_set_state(self.ctx, req.handle, req.U0)
        req.bytes = B.dg_mesh_bytes(self.ctx, req.handle)
        self.used += req.bytes
        self.peak_used = max(self.peak_used, self.used)
        req.admitted = now

    def _retire(self, req, now, reason):
        req.finished = now
        req.reason = reason
        req.extra["state"] = B.dg_get_state(self.ctx, req.handle, req.mesh.K, req.U0.shape[2])
        B.dg_mesh_free(self.ctx, req.handle)
        self.used -= req.bytes
        req.handle = -1

    def run(self, requests, keep_states=True):
        """Serve requests (prepared, sorted by arrival); returns them with
        timing fields filled."""
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []
        done = []
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                nxt = pending[0]
                curved = int(np.any(nxt.mesh.bc == 1, axis=1).sum()) if nxt.mesh is not None else 0
                est = estimate_bytes(nxt.K, nxt.N, curved=curved)
                if est > self.budget:
                    raise ValueError("request %d exceeds the whole HBM budget" % pending[0].rid)
                if self.used + est > self.budget:
                    break                            # wait for memory to free up
                req = pending.pop(0)
                self._admit(req, now)
                active.append(req)
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            self.peak_active = max(self.peak_active, len(active))
            n = min(self.check_every, min(self.max_steps - r.steps for r in active))
            B.dg_batch_step(self.ctx, [r.handle for r in active], [r.dt for r in active], n)
            for r in active:
                r.steps += n
            still = []
            for r in active:
                linf, l2 = B.dg_residual(self.ctx, r.handle, allow_nonfinite=True)
                res = float(np.max(l2))
                if math.isnan(r.r0):
                    r.r0 = res
                r.r_last = res
                now = self.clock() - t0
                if not np.isfinite(res):
                    self._retire(r, now, "nonfinite")
                elif r.r0 > 0 and res <= self.drop * r.r0:
                    self._retire(r, now, "converged")
                elif r.steps >= self.max_steps:
                    self._retire(r, now, "max_steps")
                else:
                    still.append(r)
                    continue
                if not keep_states:
                    r.extra.pop("state", None)
                done.append(r)
            active = still
        return done


def latency_stats(done):
    lat = np.array([r.finished - r.arrival for r in done])
    return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()),
            "dof_updates": float(sum(3.0 * r.steps * r.K * r.Np * 4 for r in done))}

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
arrival time (the client brings its mesh).  The library's host half of the
upload (dg_mesh_prepare: classification, device order, FP64 geometric
factors) starts on a worker thread when the request arrives and runs while
the device steps the active requests; the request is admitted once it is
done and memory allows: admission is the device half
(dg_mesh_upload_prepared) and the state upload.  The residuals of all active requests are read with one
synchronisation per check (dg_batch_residual).

Transonic requests (Mach >= av_mach) run with the Persson-Peraire
artificial viscosity of paper Sec. 2.  Its strength eps0 is a per-request
parameter: the default makes the explicit viscous time-step limit
0.5 CFL h^2 / ((N+1)^4 eps0) a hundred times the convective one's equal,
eps0 = 100 * 0.5 h lambda / (N+1)^2 (h the smallest inradius, lambda the
largest wave speed), capped at the paper's 0.3; a request that still turns
non-finite is restarted from its initial state with ten times the
viscosity (up to 0.3), at most max_retries times; a request without
viscosity that turns non-finite is restarted with it.
"""
import concurrent.futures as cf
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
    av: bool = False
    eps0: float = 0.0
    retries: int = 0
    prepared: object = None        # future of the host half of the upload
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return 2 * self.n_t * self.n_r

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2


def av_eps0(mesh, U0, N, factor=100.0, cap=0.3):
    """The viscosity strength whose explicit time-step limit is `factor`
    times smaller than the convective one (capped at the paper's eps0)."""
    h = float(np.min(states.inradius(mesh.verts)))
    return min(cap, factor * 0.5 * h * states.max_wave_speed(U0) / (N + 1) ** 2)


def prepare(req, r, s, av_mach=None):
    """Host FP64 set-up: seeded mesh, curved nodes, freestream state, dt;
    with av_mach, artificial viscosity for requests at or above that Mach
    number."""
    if req.kind == "naca":
        m = meshes.naca_omesh(n_t=req.n_t, n_r=req.n_r, seed=req.seed)
    else:
        m = meshes.cylinder_channel(n_t=req.n_t, n_r=req.n_r, seed=req.seed)
    xy, _ = curving.curve_mesh(m, req.N, r, s)
    req.mesh, req.xy = m, xy
    req.u_inf = states.freestream(req.mach, req.aoa)
    req.U0 = states.uniform_state(m.K, len(r), req.u_inf)
    req.av = av_mach is not None and req.mach >= av_mach
    req.eps0 = av_eps0(m, req.U0, req.N) if req.av else 0.0
    req.dt = states.time_step(m.verts, req.U0, req.N, cfl=0.3, eps0=req.eps0 if req.av else None)
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
                 clock=time.perf_counter, max_retries=3, workers=2):
        self.ctx = ctx
        self.budget = float(budget_bytes)
        self.check_every = int(check_every)
        self.max_steps = int(max_steps)
        self.drop = float(drop)
        self.prec = prec
        self.clock = clock
        self.max_retries = int(max_retries)
        self.workers = int(workers)
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0
        self.trace = []            # (seconds, event, request id)
        self._t0 = 0.0

    def _event(self, name, rid):
        self.trace.append((self.clock() - self._t0, name, rid))

    def _params(self, req):
        if req.av:
            return B.make_params(u_inf=req.u_inf, prec=self.prec, av_on=True, eps0=req.eps0)
        return B.make_params(u_inf=req.u_inf, prec=self.prec)

    def _prepare_host(self, req):
        """Worker thread: the host half of the upload (no context calls)."""
        self._event("prepare_start", req.rid)
        m = req.mesh
        h = B.dg_mesh_prepare(req.N, m.EToE, m.EToF, m.bc, req.xy, self._params(req))
        self._event("prepare_end", req.rid)
        return h

    def _admit(self, req, now):
        self._event("admit_start", req.rid)
        prep = req.prepared.result() if req.prepared is not None else None
        req.prepared = None
        if prep is None:
            m = req.mesh
            req.handle = B.dg_mesh_upload(self.ctx, req.N, m.EToE, m.EToF, m.bc, req.xy, self._params(req))
        else:
            req.handle = B.dg_mesh_upload_prepared(self.ctx, prep)
        B.dg_set_state(self.ctx, req.handle, req.U0)
        req.bytes = B.dg_mesh_bytes(self.ctx, req.handle)
        self.used += req.bytes
        self.peak_used = max(self.peak_used, self.used)
        if math.isnan(req.admitted):
            req.admitted = now
        self._event("admit_end", req.rid)

    def _release(self, req):
        B.dg_mesh_free(self.ctx, req.handle)
        self.used -= req.bytes
        req.handle = -1

    def _retire(self, req, now, reason, keep_state=True):
        req.finished = now
        req.reason = reason
        if keep_state:
            req.extra["state"] = B.dg_get_state(self.ctx, req.handle, req.mesh.K, req.U0.shape[2])
        self._release(req)

    def _restart_with_more_viscosity(self, req, now):
        """A transonic request that turned non-finite: again from its initial
        state with ten times the viscosity (and the matching dt)."""
        self._release(req)
        req.retries += 1
        req.eps0 = min(0.3, 10.0 * req.eps0) if req.av else av_eps0(req.mesh, req.U0, req.N)
        req.av = True
        req.dt = states.time_step(req.mesh.verts, req.U0, req.N, cfl=0.3, eps0=req.eps0)
        req.steps = 0
        req.r0 = math.nan
        req.prepared = None
        self._admit(req, now)

    def run(self, requests, keep_states=True):
        """Serve requests (prepared, sorted by arrival); returns them with
        timing fields filled."""
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []
        done = []
        self._t0 = t0 = self.clock()
        pool = cf.ThreadPoolExecutor(max_workers=self.workers) if self.workers > 0 else None
        try:
            while pending or active:
                now = self.clock() - t0
                if pool is not None:
                    # the host half of each arrived request's upload starts on
                    # a worker thread while the device steps the active ones
                    for r in pending:
                        if r.arrival > now:
                            break
                        if r.prepared is None:
                            r.prepared = pool.submit(self._prepare_host, r)
                while pending and pending[0].arrival <= now:
                    nxt = pending[0]
                    if nxt.prepared is not None and not nxt.prepared.done():
                        break                            # its host half is still running
                    curved = int(np.any(nxt.mesh.bc == 1, axis=1).sum()) if nxt.mesh is not None else 0
                    est = estimate_bytes(nxt.K, nxt.N, curved=curved, av=nxt.av,
                                         tensor=self.prec in ("tf32", "bf16x3"))
                    if est > self.budget:
                        raise ValueError("request %d exceeds the whole HBM budget" % pending[0].rid)
                    if self.used + est > self.budget:
                        break                            # wait for memory to free up
                    req = pending.pop(0)
                    self._admit(req, now)
                    active.append(req)
                if not active:
                    if pending:
                        time.sleep(max(0.001, min(0.01, pending[0].arrival - now)))
                    continue
                self.peak_active = max(self.peak_active, len(active))
                n = min(self.check_every, min(self.max_steps - r.steps for r in active))
                self._event("steps_start", len(active))
                B.dg_batch_step(self.ctx, [r.handle for r in active], [r.dt for r in active], n)
                for r in active:
                    r.steps += n
                linf, l2 = B.dg_batch_residual(self.ctx, [r.handle for r in active], allow_nonfinite=True)
                self._event("steps_end", len(active))
                still = []
                for i, r in enumerate(active):
                    res = float(np.max(l2[i]))
                    if math.isnan(r.r0):
                        r.r0 = res
                    r.r_last = res
                    now = self.clock() - t0
                    if not np.isfinite(res):
                        if r.retries < self.max_retries and (not r.av or r.eps0 < 0.3) and r.mesh is not None \
                                and hasattr(r.mesh, "verts"):
                            self._restart_with_more_viscosity(r, now)
                            still.append(r)
                            continue
                        self._retire(r, now, "nonfinite", keep_states)
                    elif r.r0 > 0 and res <= self.drop * r.r0:
                        self._retire(r, now, "converged", keep_states)
                    elif r.steps >= self.max_steps:
                        self._retire(r, now, "max_steps", keep_states)
                    else:
                        still.append(r)
                        continue
                    done.append(r)
                active = still
        finally:
            if pool is not None:
                for r in pending:
                    if r.prepared is not None and r.prepared.done() and r.prepared.exception() is None:
                        B.dg_prepared_free(r.prepared.result())
                pool.shutdown(wait=True)
        return done

    def overlap(self):
        """Seconds of host preparation that ran while the device was
        stepping (from the event trace), and the total of each."""
        prep, steps = [], []
        open_p, open_s = {}, None
        for t, ev, rid in self.trace:
            if ev == "prepare_start":
                open_p[rid] = t
            elif ev == "prepare_end" and rid in open_p:
                prep.append((open_p.pop(rid), t))
            elif ev == "steps_start":
                open_s = t
            elif ev == "steps_end" and open_s is not None:
                steps.append((open_s, t))
                open_s = None
        both = sum(max(0.0, min(b, d) - max(a, c)) for a, b in prep for c, d in steps)
        adm, open_a = [], {}
        for t, ev, rid in self.trace:
            if ev == "admit_start":
                open_a[rid] = t
            elif ev == "admit_end" and rid in open_a:
                adm.append(t - open_a.pop(rid))
        return {"prepare_s": sum(b - a for a, b in prep), "stepping_s": sum(d - c for c, d in steps),
                "prepare_during_steps_s": both, "admit_s": sum(adm), "admit_max_s": max(adm) if adm else 0.0}


def latency_stats(done):
    lat = np.array([r.finished - r.arrival for r in done])
    return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()),
            "dof_updates": float(sum(3.0 * r.steps * r.K * r.Np * 4 for r in done)),
            "service_s": float(np.mean([r.finished - r.admitted for r in done]))}

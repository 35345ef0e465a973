#!/usr/bin/env python3
"""Benchmark of the curved-element RKDG hot path on GB300.

Metric: RK-stage DOF-updates/s = K * N_p * 4 * (RK stages) / device time,
for the mixed-precision products and the FP32 path on the same GPU.
Default workload: the precision sweep on a curved cylinder-in-channel mesh
(Mach 0.38, 250,000 triangles, wall elements curved to degree N = 6 by the
linear-elasticity set-up, FP32 state, SSP-RK3): TF32 products timed, FP32
and split-BF16 products timed beside them, each precision's error against
the FP64 oracle (and, on the isentropic-vortex twin of the same N and K,
against the FP64 path and the exact solution) in `error_vs_oracle`.  The
NACA 0012 workload (Mach 0.8, 60,000 triangles, N = 4, artificial viscosity
on) starts from a state with troubled cells (a jump across the wake) and
reports its viscous and inviscid stage launches.

One "step" = one SSP-RK3 step = 3 right-hand-side evaluations with the stage
update fused in (sensor, gradient and stage kernels per stage), replayed from
the library's captured CUDA graph.  Each timed step is bracketed by CUDA
events on the library's stream; L2 is flushed (512 MiB memset) before every
timed step, outside the events.  Per-kernel device times come from event
nodes inside the step graph, read after every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank runs an
independent replica of the workload (the method is not sharded here);
value = all ranks' DOF-updates / max-over-ranks time.
"""
import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK-stage DOF-updates/s"
UNIT = "DOF-updates/s"
# arithmetic of the path per --prec: FP32 state and fluxes throughout; the
# element-local operator products in TF32 or split BF16 on the tensor cores
DTYPE = {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3", "fp64": "f64"}

# DRAM bytes (read + write) of one stage-kernel launch from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (workload,
# products, flux, launch kind), SSP-RK3 stages only.  Each entry carries the
# hash of the kernel sources it was taken on; a line whose sources differ
# reports traffic null.
TRAFFIC = {
    # cylinder N = 6, 250k elements, inviscid launch (stage 1 of a timed step, after the L2 flush)
    ("cylinder_m0.38_n6", "tf32", "llf", "stage"): (129.754112e6 + 72.465920e6, "2342ba159b1e"),
    # NACA 0012 N = 4, 60k elements: a viscous launch (troubled cells) and an inviscid one
    ("naca0012_m0.8_n4_av", "tf32", "llf", "stage_viscous"): (46.189824e6 + 0.414720e6, "2342ba159b1e"),
    ("naca0012_m0.8_n4_av", "tf32", "llf", "stage"): (17.494272e6 + 0.000256e6, "2342ba159b1e"),
}

# the sources of each stage kernel, hashed into the traffic key above
KERNEL_SOURCES = {"tri": ("tc_kernels.cuh", "tc_ptx.cuh", "kernels.cuh", "dg_device.h"),
                  "tet": ("kernels3_tc.cu", "kernels3.cuh", "kernels3.cu", "dg3_device.h")}


def kernel_source_hash(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1208_4772_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def traffic_of(workload, prec, flux, kind, launch="stage"):
    """ncu DRAM bytes of one launch, if taken on the current sources."""
    t = TRAFFIC.get((workload, prec, flux, launch))
    if t is None or t[1] != kernel_source_hash(kind):
        return None
    return t[0]

WORKLOADS = {
    "naca0012_m0.8_n4_av": dict(kind="naca", N=4, n_t=300, n_r=100, mach=0.8, aoa=1.25, av=True,
                                describe="NACA 0012, Mach 0.8, AoA 1.25 deg, 60k curved-wall triangles, "
                                         "N=4, artificial viscosity on"),
    "cylinder_m0.38_n6": dict(kind="cyl", N=6, n_t=500, n_r=250, mach=0.38, aoa=0.0, av=False,
                              describe="cylinder in a channel, Mach 0.38, 250k triangles, N=6"),
    # many meshes at once (dg_batch_step): not a single-mesh workload
    "batch64": dict(kind="batch", describe="64 meshes, K log-uniform in [2k, 200k], N uniform in {2,3,4,5}, "
                                           "airfoil and cylinder alternating, Mach U[0.3,0.85], AoA U[-2,4] deg, "
                                           "artificial viscosity from Mach 0.5; one persistent launch per RK stage "
                                           "for the meshes without viscosity, the others on branches of the step "
                                           "graph"),
    "prefine": dict(kind="prefine", describe="p-refinement (paper Sec. 5): cylinder channel, 15,360 elements, "
                                             "Mach 0.38, no AV; degrees 2 -> 3 -> 4 against N = 4 from the "
                                             "freestream, to the same residual"),
    # the tetrahedral method (the paper's 3D setting): a single mesh
    "bump3d_m0.5_n3": dict(kind="tet", N=3, cells=(50, 25, 40), Zd=0.4, mach=0.5,
                           describe="tetrahedra: channel 3 x 1.5 x 0.8 over a smooth floor bump of height 0.1, "
                                    "50 x 25 x 40 Kuhn-split cells = 300k tetrahedra (curved below z = 0.4 over "
                                    "the bump), "
                                    "N=3, Mach 0.5, slip walls, farfield in/outflow, LLF"),
    "serve": dict(kind="serve", describe="continuous batching: Poisson arrivals, K log-uniform in [1k, 500k], "
                                         "N uniform in {2..6}, Mach U[0.3,0.85] (artificial viscosity from Mach "
                                         "0.5), admission by an HBM budget, retirement at a 1e-6 residual drop or "
                                         "20,000 steps"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cylinder_m0.38_n6", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="tf32", help="products: tf32 (default), bf16x3, fp32, fp64")
    ap.add_argument("--compare-prec", default="fp32,bf16x3",
                    help="also time these precisions, comma-separated (none or '' to skip)")
    ap.add_argument("--no-errors", action="store_true", help="skip the error_vs_oracle measurements")
    ap.add_argument("--av-start", default="jump", choices=["jump", "freestream"],
                    help="AV workloads: start from a state with troubled cells (jump) or the freestream")
    ap.add_argument("--integrator", default="ssp3", choices=["ssp3", "lserk"],
                    help="SSP-RK3 (3 stages) or the paper's low-storage RK(5,4) (5 stages)")
    ap.add_argument("--flux", default="llf", choices=["llf", "hllc"], help="numerical flux at the faces")
    ap.add_argument("--tet-av", action="store_true",
                    help="tetrahedra: artificial viscosity on (sensor, gradient pass, viscous stage; FP32/FP64)")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-meshes", type=int, default=64, help="batch64: number of meshes")
    ap.add_argument("--batch-av-mach", type=float, default=0.5,
                    help="batch64: artificial viscosity for meshes at or above this Mach number")
    ap.add_argument("--prefine-drop", type=float, default=0.1, help="prefine: residual drop of the lower levels")
    ap.add_argument("--prefine-max-steps", type=int, default=20000, help="prefine: steps of the N = 4 runs")
    ap.add_argument("--prefine-max-steps-low", type=int, default=5000, help="prefine: steps of the lower levels")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-max-steps", type=int, default=20000)
    ap.add_argument("--serve-rates", default="0.5,1,2", help="serve: arrival rates as multiples of the service rate")
    ap.add_argument("--serve-av-mach", type=float, default=0.5,
                    help="serve: artificial viscosity for requests at or above this Mach number")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--cpu-sample", default="", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-start", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------------ workload
def make_workload(name, r, s, av_start="jump"):
    """Seeded mesh, curved nodes, initial state and time step (inputs only).
    With artificial viscosity and av_start == "jump" every variable is
    multiplied by 1.5 downstream of x = 2 (a jump of density and energy at
    unchanged velocity and sound speed), so that the elements the line cuts
    are troubled cells (eps > 0) from the first step."""
    import numpy as np
    from paper_1208_4772_gb300.inputs import curving, meshes, states
    w = WORKLOADS[name]
    if w["kind"] == "naca":
        mesh = meshes.naca_omesh(n_t=w["n_t"], n_r=w["n_r"], seed=1001)
    else:
        mesh = meshes.cylinder_channel(n_t=w["n_t"], n_r=w["n_r"], seed=1002)
    xy, curved = curving.curve_mesh(mesh, w["N"], r, s)
    ui = states.freestream(w["mach"], w["aoa"])
    U0 = states.uniform_state(mesh.K, len(r), ui)
    if w["av"] and av_start == "jump":
        U0 = U0 * np.where(xy[..., 0] > 2.0, 1.5, 1.0)[:, None, :]
    dt = states.time_step(mesh.verts, U0, w["N"], cfl=0.3, eps0=0.3 if w["av"] else None)
    return dict(mesh=mesh, xy=xy, curved=curved, u_inf=ui, U0=U0, dt=dt, av_start=av_start if w["av"] else None, **w)


def make_vortex_twin(N, n, r, s):
    """The isentropic-vortex twin of a workload: the periodic square [0,10]^2
    of n x n cells cut along one diagonal (K = 2 n^2), jittered vertices,
    the vortex state; its exact solution is the translated vortex."""
    from paper_1208_4772_gb300.inputs import meshes, states
    mesh = meshes.periodic_square(n, length=10.0, seed=1000)
    xy = meshes.straight_nodes(mesh.verts, r, s)
    U0 = states.vortex_state(xy, period=(10.0, 10.0))
    dt = states.time_step(mesh.verts, U0, N, cfl=0.3)
    return dict(mesh=mesh, xy=xy, U0=U0, dt=dt, u_inf=states.freestream(0.5, 45.0))


def make_tet_workload(name, r, s, t):
    """Seeded tetrahedral mesh, nodes, initial state and time step (inputs only)."""
    from paper_1208_4772_gb300.inputs import meshes3d, states
    w = WORKLOADS[name]
    mesh = meshes3d.bump_channel(*w["cells"], Zd=w["Zd"], seed=2000)
    X = meshes3d.node_coords(mesh, r, s, t)
    ui = states.freestream3(w["mach"], 0.0)
    U0 = states.uniform_state3(mesh.K, len(r), ui)
    dt = states.time_step3(mesh.verts, U0, w["N"], cfl=0.3)
    curved = meshes3d.mapped_elements(mesh, r, s, t)
    return dict(mesh=mesh, xyz=X, curved=curved, u_inf=ui, U0=U0, dt=dt, **w)


def tet_sizes(N):
    q = (3 * N + 2) // 2
    return (N + 1) * (N + 2) * (N + 3) // 6, q ** 3, q * q, (N + 1) * (N + 2) // 2


def tet_stage_flops(N):
    """Algorithmic FP32 operations of one element in one tetrahedral stage:
    interpolation to the cubature points (2 N_q N_p per variable), the three
    weighted derivative products (6 N_p N_q per variable), face-node ->
    face-point interpolation on both sides and its transpose for the lift
    (3 x 2 N_g N_fp per face and variable), the inverse mass (2 N_p^2 per
    variable), the Euler flux with its contravariant form (~40 per cubature
    point) and the numerical flux (~70 per face point)."""
    Np, Nq, Ng, Nfp = tet_sizes(N)
    return 5 * (2 * Nq * Np + 6 * Np * Nq + 4 * 3 * 2 * Ng * Nfp + 2 * Np * Np) + 40 * Nq + 70 * 4 * Ng


def tet_stage_bytes(K, Kc, N):
    """Algorithmic HBM bytes of one tetrahedral stage launch (SSP-RK3
    average): read U_s, read U^n in stages 2 and 3, write U_out (5 N_p FP32
    each), affine geometry 36 B, neighbours 16 B and face codes 8 B per
    element, the curved elements' record (cofactors at the cubature points,
    face normals and area factors, M_k^-1); neighbour face nodes are L2
    hits and count 0."""
    Np, Nq, Ng, Nfp = tet_sizes(N)
    state = 5 * Np * 4
    return K * (state * (1 + 2.0 / 3.0 + 1) + 24) + (K - Kc) * 36 + Kc * (9 * Nq + 16 * Ng + Np * Np) * 4


def stage_kernel_bytes(K, Kc, N, av, viscous=True):
    """Algorithmic HBM bytes of one stage-kernel launch, averaged over the
    three SSP-RK3 stages: read U_s, read U^n (stages 2 and 3), write U_out
    (4 N_p FP32 each), affine geometry 16 B + connectivity 16 B per element,
    curved elements' factor record; with artificial viscosity the next
    stage's eps (4 B written) and, in a launch whose input has viscous
    elements, q (8 N_p FP32) and eps (4 B) read.  Neighbour traces are L2
    hits and count 0."""
    q = (3 * N + 2) // 2
    Np, Nq, Nf = (N + 1) * (N + 2) // 2, q * q, 3 * q
    state = 4 * Np * 4
    b = K * (state * (1 + 2.0 / 3.0 + 1) + 16) + (K - Kc) * 16 + Kc * (5 * Nq + 3 * Nf + Np * Np) * 4
    if av:
        b += K * 4
        if viscous:
            b += K * (8 * Np * 4 + 4)
    return b


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region: the
    sampler runs every 20 ms from before the region (start() returns once
    the first sample has arrived, so that the region is covered from its
    beginning) and stop() keeps the samples read between mark() and stop()
    (all of them if none fell inside a very short region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None
        self.t_mark = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.t_mark = time.perf_counter()

    def mark(self):
        """The timed region begins now."""
        self.t_mark = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        t_end = time.perf_counter()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if self.t_mark is not None and self.t_mark <= t <= t_end + 0.03]
        for ln in (inside or [ln for _, ln in self.lines]):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
# The FP64 oracle as it stands, timed on the host cores on a bounded sample
# of the workload: right-hand sides of one contiguous block of elements
# (with the artificial viscosity, each call also computes the sensor and the
# gradient on the rings of neighbours the block needs, as the oracle does
# for any subset).  The oracle builds the geometry of a subset in every
# call; here it is built once per subset before the timer, as the geometry
# of the whole mesh is built once at set-up.  The single-core leg, the
# all-cores leg (one process per core on disjoint blocks, like the paper's
# OpenMP loop over elements) and the reference arm share this sampler.
def oracle_inputs_path(wl, flux, kind):
    """Write the oracle's inputs once (inputs only, no arithmetic of the
    method) for the CPU legs' worker processes; returns the file's path."""
    import tempfile
    import numpy as np
    fd, path = tempfile.mkstemp(suffix=".npz", prefix="dg_oracle_inputs_")
    os.close(fd)
    m = wl["mesh"]
    if kind == "tet":
        np.savez(path, kind="tet", N=wl["N"], EToV=m.EToV, bc=m.bc, X=wl["xyz"], U0=wl["U0"],
                 u_inf=wl["u_inf"], av=False, flux=flux)
    else:
        np.savez(path, kind="tri", N=wl["N"], EToE=m.EToE, EToF=m.EToF, bc=m.bc, X=wl["xy"], U0=wl["U0"],
                 u_inf=wl["u_inf"], av=bool(wl["av"]), flux=flux)
    return path


class OracleSampler:
    """Right-hand sides of the oracle on one contiguous block of elements."""

    def __init__(self, path):
        import numpy as np
        d = np.load(path)
        self.kind = str(d["kind"])
        self.N = int(d["N"])
        self.U0 = d["U0"]
        flux, av = str(d["flux"]), bool(d["av"])
        if self.kind == "tet":
            from oracle.dg3 import Oracle3
            base, args = Oracle3, (self.N, d["EToV"], d["bc"], d["X"])
            self.nv = 5
        else:
            from oracle.dg import Oracle
            base, args = Oracle, (self.N, d["EToE"], d["EToF"], d["bc"], d["X"])
            self.nv = 4
        cache = {}

        class Cached(base):
            def geometry(self, idx=None):
                if idx is None:
                    return super().geometry(None)
                key = np.asarray(idx).tobytes()
                if key not in cache:
                    cache[key] = super().geometry(idx)
                return cache[key]
        kw = dict(u_inf=d["u_inf"], flux=flux)
        if av:
            kw["av"] = True
        self.o = Cached(*args, **kw)
        self.K = self.o.K
        self.Np = self.U0.shape[2]

    def block(self, start, size):
        import numpy as np
        size = max(1, min(int(size), self.K))
        start = int(start) % max(1, self.K - size + 1)
        return np.arange(start, start + size)

    def calibrate(self, start, seconds_per_call):
        """Block size whose right-hand side takes about seconds_per_call
        (after its geometry has been built)."""
        import time as _t
        S = 64
        while True:
            idx = self.block(start, S)
            self.o.rhs(self.U0, idx)                        # builds and caches the geometry
            t0 = _t.perf_counter()
            self.o.rhs(self.U0, idx)
            el = _t.perf_counter() - t0
            if el > 0.5 * seconds_per_call or S >= self.K:
                return max(16, min(self.K, int(S * seconds_per_call / max(el, 1e-6))))
            S *= 4

    def rate(self, idx, budget_s):
        """DOF-updates/s of right-hand sides on idx, repeated for budget_s."""
        import time as _t
        self.o.rhs(self.U0, idx)                            # geometry of idx and its rings, untimed
        t0 = _t.perf_counter()
        n = 0
        while True:
            self.o.rhs(self.U0, idx)
            n += 1
            el = _t.perf_counter() - t0
            if el > budget_s:
                break
        return len(idx) * self.Np * self.nv * n / el, n


def cpu_worker(path, start, budget_s):
    """One process of a CPU leg: the oracle on the block at `start`."""
    sm = OracleSampler(path)
    S = sm.calibrate(start, 1.0)
    idx = sm.block(start, S)
    value, n = sm.rate(idx, budget_s)
    return {"value": value, "evals": n, "block": [int(idx[0]), int(len(idx))], "K": int(sm.K)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_cpu_baseline(path, budget_s):
    """The single-core leg and the all-cores leg (one single-threaded
    worker process per core, each on its own block; the sum of their
    rates).  Fresh processes: no CUDA context, one BLAS thread each."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")

    def launch(P):
        procs = []
        for i in range(P):
            start = (i * 7919 * 64) if P > 1 else 0
            procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-sample", path,
                                           "--cpu-budget-s", str(budget_s), "--cpu-start", str(start)],
                                          stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env))
        res = []
        for pr in procs:
            out, err = pr.communicate(timeout=900)
            if pr.returncode != 0:
                return None, err[-500:]
            res.append(json.loads(out.strip().splitlines()[-1]))
        return res, None

    one, err = launch(1)
    if one is None:
        return {"error": err}
    ncores = os.cpu_count() or 1
    allc, err = launch(ncores)
    r1 = one[0]
    line = {"value": r1["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "right-hand sides of a block of %d contiguous elements of the %d-element mesh, repeated "
                      "for %.0f s (%d calls); the block's geometry built before the timer"
                      % (r1["block"][1], r1["K"], budget_s, r1["evals"]),
            "nproc": ncores, "cpu_model": cpu_model()}
    if allc is not None:
        line["all_cores"] = {"value": sum(r["value"] for r in allc), "unit": UNIT, "cores": ncores,
                             "sample": "%d single-threaded processes, one block each (%s elements), the "
                                       "sum of their rates" % (ncores, ",".join(str(r["block"][1]) for r in allc))}
    else:
        line["all_cores"] = {"error": err}
    return line


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle arm: each step is one SSP-RK3 step (three right-hand
    sides with the stage combinations) on a contiguous block of elements
    of about one second of oracle work per right-hand side (less when the
    warm-up and timed steps would take more than 100 s)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if WORKLOADS[args.workload]["kind"] in ("batch", "serve", "prefine"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm is timed on the single-mesh "
                                                              "workloads only"}), flush=True)
        return 0
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"          # before numpy loads: the oracle runs on one core
    kind = "tet" if WORKLOADS[args.workload]["kind"] == "tet" else "tri"
    if kind == "tet":
        from oracle.tet import ReferenceTet
        ref = ReferenceTet(WORKLOADS[args.workload]["N"])
        wl = make_tet_workload(args.workload, ref.r, ref.s, ref.t)
        cfg = {"workload": args.workload, "describe": wl["describe"], "K": int(wl["mesh"].K), "N": wl["N"],
               "flux": args.flux.upper()}
    else:
        from oracle.operators import ReferenceElement
        ref = ReferenceElement(WORKLOADS[args.workload]["N"])
        wl = make_workload(args.workload, ref.r, ref.s, args.av_start)
        cfg = config_of(args, wl)
    path = oracle_inputs_path(wl, args.flux, kind)
    try:
        sm = OracleSampler(path)
        per_step = 100.0 / max(1, args.steps + args.warmup)
        S = int(sm.calibrate(0, 0.5) * min(1.0, per_step / 3.0) / 0.5)
        idx = sm.block(sm.K // 2, S)
        o, dt = sm.o, wl["dt"]
        U = sm.U0.copy()

        def step():
            Us = U
            for a, b in ((0.0, 1.0), (0.75, 0.25), (1 / 3, 2 / 3)):
                L = o.rhs(Us, idx)
                Us = Us.copy()
                Us[idx] = a * U[idx] + b * (Us[idx] + dt * L)
            return Us

        o.rhs(U, idx)             # geometry of the block and its rings, before the warm-up
        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    finally:
        os.unlink(path)
    value = len(idx) * sm.Np * sm.nv * 3 * args.steps / el
    sample = ("a block of %d contiguous elements of %d per SSP-RK3 step (3 right-hand sides on the block; its "
              "geometry built before the timer)" % (len(idx), sm.K))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(args, wl):
    m = wl["mesh"]
    Np = (wl["N"] + 1) * (wl["N"] + 2) // 2
    return {"workload": args.workload, "describe": wl["describe"], "K": int(m.K), "N": wl["N"], "Np": Np,
            "curved_elements": int(wl["curved"].sum()), "artificial_viscosity": bool(wl["av"]),
            "state_precision": "fp32" if args.prec != "fp64" else "fp64", "products": args.prec,
            "time_integrator": "LSERK(5,4)" if getattr(args, "integrator", "ssp3") == "lserk" else "SSP-RK3",
            "flux": getattr(args, "flux", "llf").upper(),
            "dt": wl["dt"], "dof_per_stage": int(m.K * Np * 4),
            "start_state": ("troubled cells: every variable x1.5 downstream of x = 2" if wl.get("av_start") == "jump"
                            else "freestream"),
            "l2": "flushed before every timed step (%d MiB memset, outside the step events)" % args.flush_mb,
            "parallelism": "replicas (one independent solve per GPU)"}


# ------------------------------------------------------------------ ranks
# One independent replica per GPU (the path does not shard): every rank
# times its own steps, the job's time is the slowest rank's, and the job's
# rate counts the work of all ranks.
def max_over_ranks(ms, dist, device):
    """The largest of the ranks' times (ms); the value itself without
    torch.distributed."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, job_ms):
    """Units per second of the whole job: all ranks' units over the job's time."""
    return world * units_per_rank / (job_ms / 1e3)


# ------------------------------------------------------------------ our arm
def timed_steps(B, ctx, h, dt, steps, stream, flush, torch, profiled=False, step=None):
    """Time `steps` single-step graph replays; returns (step_ms list, summed
    per-kind kernel ms, kernel launches) -- the last two only when the mesh
    records per-kernel events (profiled)."""
    import numpy as np
    kt = np.zeros(3)
    launches = 0
    times = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        (step or B.dg_step)(ctx, h, dt, 1)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        if profiled:
            t = B.dg_kernel_times(ctx, h)
            kt += t[:3]
            launches += int(t[3])
    return times, kt, launches


def oracle_step_sample(o, U, dt, idx, depth):
    """One SSP-RK3 step of the oracle on the elements idx only: each stage
    on the rings of neighbours the next stage needs (depth rings per stage:
    1 for the Euler right-hand side, 2 with the artificial viscosity)."""
    import numpy as np
    rings = [np.asarray(idx)]
    for _ in range(2 * depth):
        rings.append(o.neighbours(rings[-1]))
    S1, S2, S3 = rings[2 * depth], rings[depth], rings[0]
    U1 = U.copy()
    U1[S1] = U[S1] + dt * o.rhs(U, S1)
    U2 = U.copy()
    U2[S2] = 0.75 * U[S2] + 0.25 * (U1[S2] + dt * o.rhs(U1, S2))
    return U[S3] / 3.0 + 2.0 / 3.0 * (U2[S3] + dt * o.rhs(U2, S3))


def rel_l2_max(a, b):
    """max over the conserved variables of ||a - b|| / ||b|| (arrays [n, nv, Np])."""
    import numpy as np
    nv = a.shape[1]
    d = np.linalg.norm((a - b).transpose(1, 0, 2).reshape(nv, -1), axis=1)
    return float(np.max(d / np.linalg.norm(b.transpose(1, 0, 2).reshape(nv, -1), axis=1)))


def precision_errors(B, ctx, args, wl, precs, r, s):
    """error_vs_oracle of the bench line, per precision of the products.

    rhs_sampled: the right-hand side of the workload mesh for a perturbed
    state (the AV workload: its start state, whose troubled cells are in the
    sample) against the FP64 oracle on 160 random and 64 wall elements (and
    64 troubled ones), relative L2, the largest over the variables.
    vortex_twin (N = 6 workload): the isentropic vortex on the periodic
    square of the same N and about the same K (n = 354, K = 250,632), 100
    SSP-RK3 steps in each precision: the increment U_100 - U_0 against that
    of the FP64 path (itself within 1e-12 of the oracle on the parity
    meshes), the state against the exact (translated) vortex, and the
    sampled right-hand side against the oracle."""
    import numpy as np
    from oracle.dg import Oracle
    N = wl["N"]
    m = wl["mesh"]
    Np = len(r)
    rng = np.random.default_rng(17)
    out = {}
    x, y = wl["xy"][..., 0], wl["xy"][..., 1]
    U = wl["U0"].copy()
    if not wl["av"]:
        U[:, 0] *= 1.0 + 0.02 * np.sin(1.3 * x) * np.cos(0.7 * y)
        U[:, 3] *= 1.0 + 0.02 * np.cos(0.9 * x + 0.4 * y)
        U[:, 1] += 0.02 * np.sin(y)
        U[:, 2] += 0.02 * np.cos(x)
    U = U.astype(np.float32).astype(np.float64)
    wall = np.nonzero(np.any(m.bc == 1, axis=1))[0]
    parts = [rng.choice(m.K, 160, replace=False), rng.choice(wall, min(64, len(wall)), replace=False)]
    if wl["av"]:
        cut = np.nonzero((x.min(axis=1) < 2.0) & (x.max(axis=1) > 2.0))[0]
        parts.append(rng.choice(cut, min(64, len(cut)), replace=False))
    idx = np.unique(np.concatenate(parts))
    o = Oracle(N, m.EToE, m.EToF, m.bc, wl["xy"], u_inf=wl["u_inf"], av=wl["av"], flux=args.flux)
    Lo = o.rhs(U, idx)
    rs = {}
    for prec in precs:
        h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, wl["xy"],
                             B.make_params(u_inf=wl["u_inf"], av_on=wl["av"], prec=prec, flux=args.flux))
        B.dg_set_state(ctx, h, U)
        L = B.dg_eval_rhs(ctx, h, m.K, Np)
        B.dg_mesh_free(ctx, h)
        rs[prec] = rel_l2_max(L[idx], Lo)
    out["rhs_sampled"] = {"elements": int(len(idx)), "rel_l2": rs,
                          "state": "start state (troubled cells)" if wl["av"] else "smoothly perturbed freestream"}
    if N == 6:
        from paper_1208_4772_gb300.inputs import states
        tw = make_vortex_twin(N, 354, r, s)
        mt = tw["mesh"]
        U0 = tw["U0"].astype(np.float32).astype(np.float64)
        nsteps = 100
        res = {}
        for prec in list(precs) + (["fp64"] if "fp64" not in precs else []):
            h = B.dg_mesh_upload(ctx, N, mt.EToE, mt.EToF, mt.bc, tw["xy"],
                                 B.make_params(u_inf=tw["u_inf"], prec=prec, flux=args.flux))
            B.dg_set_state(ctx, h, U0)
            Lt = B.dg_eval_rhs(ctx, h, mt.K, Np)
            B.dg_step(ctx, h, tw["dt"], nsteps)
            res[prec] = (B.dg_get_state(ctx, h, mt.K, Np), Lt)
            B.dg_mesh_free(ctx, h)
        ref_inc = res["fp64"][0] - U0
        exact = states.vortex_state(tw["xy"], t=nsteps * tw["dt"], period=(10.0, 10.0))
        it = np.unique(rng.choice(mt.K, 192, replace=False))
        ot = Oracle(N, mt.EToE, mt.EToF, mt.bc, tw["xy"], flux=args.flux)
        Lot = ot.rhs(U0, it)
        out["vortex_twin"] = {
            "K": int(mt.K), "N": N, "steps": nsteps, "dt": tw["dt"],
            "increment_vs_fp64_path": {p: rel_l2_max(v[0] - U0, ref_inc) for p, v in res.items() if p != "fp64"},
            "state_vs_exact": {p: rel_l2_max(v[0], exact) for p, v in res.items()},
            "rhs_sampled_vs_oracle": {p: rel_l2_max(v[1][it], Lot) for p, v in res.items()}}
    return out


def run_ours(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_1208_4772_gb300 import binding as B
    B.load()
    N = WORKLOADS[args.workload]["N"]
    r, s = B.dg_reference_nodes(N)
    wl = make_workload(args.workload, r, s, args.av_start)
    m = wl["mesh"]
    Np = len(r)
    dof_stage = m.K * Np * 4
    # a dedicated stream: the library, the L2 flush and the timing events all
    # run on it (the legacy default stream has handle 0, which the C ABI
    # reads as "no stream given")
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = B.dg_create(local, stream.cuda_stream)
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device="cuda")

    def upload(prec, U0=None):
        p = B.make_params(u_inf=wl["u_inf"], av_on=wl["av"], prec=prec, flux=args.flux)
        h = B.dg_mesh_upload(ctx, N, m.EToE, m.EToF, m.bc, wl["xy"], p)
        B.dg_set_state(ctx, h, wl["U0"] if U0 is None else U0)
        return h

    step = B.dg_step_lserk if args.integrator == "lserk" else B.dg_step
    nstage = 5 if args.integrator == "lserk" else 3

    def warm(h):
        for _ in range(args.warmup):
            flush.zero_()
            step(ctx, h, wl["dt"], 1)
        torch.cuda.synchronize()

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"

    def stage_roofline(h, nsteps, viscous):
        """Per-kernel times from a pass with CUDA events around every kernel
        inside the step graph; the stage kernel's average launch against its
        algorithmic bytes."""
        B.dg_set_profiling(ctx, h, 1)
        warm(h)
        pt, kt, launches = timed_steps(B, ctx, h, wl["dt"], nsteps, stream, flush, torch, profiled=True)
        B.dg_set_profiling(ctx, h, 0)
        ms = kt[2] / (3 * nsteps)
        nbytes = stage_kernel_bytes(m.K, int(wl["curved"].sum()), N, wl["av"], viscous)
        ach = nbytes / (ms * 1e-3) / 1e9
        return {"kernel": "stage_kernel_tc (N=%d, %s launch)" % (N, "viscous" if viscous else "inviscid")
                if args.prec in ("tf32", "bf16x3") else "stage_kernel (N=%d)" % N,
                "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": peak_src,
                "traffic": traffic_of(args.workload, args.prec, args.flux, "tri",
                                      "stage_viscous" if viscous else "stage"),
                "bytes_per_launch": nbytes, "avg_launch_ms": ms}, kt / nsteps, pt, launches / nsteps

    h = upload(args.prec)
    visc = {"start": B.dg_av_count(ctx, h)} if wl["av"] else None
    # timed choice of the work distribution: CUDA-core tile size, or the
    # tensor-core stage kernel's tile-pipeline configuration
    tuned = {args.prec: B.dg_autotune(ctx, h, 5)}
    B.dg_set_state(ctx, h, wl["U0"])
    warm(h)

    # headline: the step graph as a user runs it (no timing events inside it,
    # so consecutive kernels may overlap their prologues and tails)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    times, _, _ = timed_steps(B, ctx, h, wl["dt"], args.steps, stream, flush, torch, step=step)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dist, "cuda")
    value = whole_job_rate(world, dof_stage * nstage * args.steps, total_ms)
    linf, l2 = B.dg_residual(ctx, h, allow_nonfinite=True)
    if visc is not None:
        visc["end"] = B.dg_av_count(ctx, h)

    # the roofline of the dominant kernel (the fused stage kernel) from a
    # second pass with events around every kernel; with the artificial
    # viscosity the timed launches are viscous ones (troubled cells) and an
    # inviscid pass (freestream start) is reported beside them
    kinds = ["sensor", "gradient", "stage"]
    n_prof = min(args.steps, 300)
    extra = {}
    if args.integrator == "ssp3":
        viscous = visc is None or visc["start"] > 0 or visc["end"] > 0
        B.dg_set_state(ctx, h, wl["U0"])
        roofline, kt_step, ptimes, launches_step = stage_roofline(h, n_prof, viscous if wl["av"] else False)
        if wl["av"]:
            B.dg_set_state(ctx, h, np.broadcast_to(np.asarray(wl["u_inf"])[None, :, None], wl["U0"].shape).copy())
            inv, _, _, _ = stage_roofline(h, n_prof, False)
            extra["roofline_inviscid"] = inv
        launches = int(launches_step * args.steps)
        kt = kt_step * args.steps
    else:   # no timing nodes in the low-storage graph: kernels counted, not timed one by one
        ptimes, kt = times[:1], np.zeros(3)
        launches = args.steps * 5 * (3 if wl["av"] else 1)
        ms = total_ms / args.steps / 5
        nbytes = stage_kernel_bytes(m.K, int(wl["curved"].sum()), N, wl["av"], True)
        roofline = {"kernel": "whole low-storage step / 5 stages", "bound": "hbm",
                    "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": nbytes / (ms * 1e-3) / 1e9 / peak, "peak_source": peak_src, "traffic": None,
                    "bytes_per_launch": nbytes, "avg_launch_ms": ms}
    roofline["dominant_kind_by_time"] = kinds[int(np.argmax(kt))]

    compares = [c for c in args.compare_prec.split(",") if c and c not in ("none", args.prec)]
    cmp_lines = []
    for cp in compares:
        h2 = upload(cp)
        tuned[cp] = B.dg_autotune(ctx, h2, 5)
        B.dg_set_state(ctx, h2, wl["U0"])
        warm(h2)
        n2 = min(args.steps, 500)
        t2, _, _ = timed_steps(B, ctx, h2, wl["dt"], n2, stream, flush, torch, step=step)
        c = {"products": cp, "value": world * dof_stage * nstage * n2 / (sum(t2) / 1e3), "ms_per_step": sum(t2) / n2}
        c["tile_e"] = tuned[cp][0]
        c["autotune_ms_per_step"] = {str(k): v for k, v in tuned[cp][1].items()}
        c["tuned_choice"] = tuned[cp][2]
        cmp_lines.append(c)
        B.dg_mesh_free(ctx, h2)
    if cmp_lines:
        extra["compare"] = cmp_lines

    e2e = None
    if not args.no_e2e:
        step(ctx, h, wl["dt"], 1)     # capture the plain graph outside the timing
        torch.cuda.synchronize()
        U_host = np.ascontiguousarray(wl["U0"])
        auto = B.dg_host_io(ctx)

        def e2e_run():
            t0 = time.perf_counter()
            B.dg_set_state(ctx, h, U_host)
            step(ctx, h, wl["dt"], args.steps)
            U_out = B.dg_get_state(ctx, h, m.K, Np)
            return time.perf_counter() - t0, U_out.nbytes

        # every host I/O mode the device offers, the context's own (auto) last
        by_mode = {}
        for mode in [x for x in ("staged", "device") if x != auto] + [auto]:
            try:
                B.dg_set_host_io(ctx, mode)
            except B.DgError:
                continue
            el, out_bytes = e2e_run()
            by_mode[mode] = dof_stage * nstage * args.steps / el
        nbytes = U_host.nbytes
        e2e = {"value": by_mode[auto], "unit": UNIT,
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": out_bytes / args.steps,
               "host_io": auto, "by_host_io": by_mode,
               "how": "dg_set_state(host FP64) + %s(%d) + dg_get_state(host FP64), wall clock"
                      % ("dg_step_lserk" if args.integrator == "lserk" else "dg_step", args.steps)}
    B.dg_mesh_free(ctx, h)

    errors = None
    if rank == 0 and not args.no_errors and args.integrator == "ssp3":
        errors = precision_errors(B, ctx, args, wl, [args.prec] + compares, r, s)
    B.dg_destroy(ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        path = oracle_inputs_path(wl, args.flux, "tri")
        try:
            cpu = run_cpu_baseline(path, args.cpu_budget_s)
        finally:
            os.unlink(path)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec],
                "data": "synthetic", "config": config_of(args, wl), "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches * world),
                "clocks": clk,
                "kernel_ms_per_step": {k: float(kt[i] / args.steps) for i, k in enumerate(kinds)},
                "profiled_ms_per_step": float(sum(ptimes) / max(1, len(ptimes))),
                "tile_e": tuned[args.prec][0],
                "autotune": {"candidates_ms_per_step": {str(k): v for k, v in tuned[args.prec][1].items()},
                             "choice": tuned[args.prec][2],
                             "what": "tile-pipeline configuration 10 C + P of the tensor-core stage kernel (C CTAs "
                                     "per SM of P tile pipelines)" if args.prec in ("tf32", "bf16x3")
                                     else "elements per CUDA-core tile"},
                "residual_linf": [float(x) for x in linf],
                "viscous_elements": visc, "error_vs_oracle": errors, **extra}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ tetrahedra
def run_tet(args):
    """The tetrahedral stage kernel on one mesh: SSP-RK3 steps through
    dg_step, L2 flushed before every timed step; a second pass with events
    around every kernel gives the stage kernel's launch time.  FP32 runs on
    the CUDA cores, TF32 (the default) puts the two volume products on the
    tensor cores; the roofline is the FP32 ALU peak on the method's
    algorithmic flops either way."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B
    B.load()
    torch.cuda.set_device(0)
    w = WORKLOADS[args.workload]
    N = w["N"]
    prec = args.prec if args.prec in ("fp32", "fp64", "tf32") else "fp32"
    if args.tet_av and prec == "tf32":
        prec = "fp32"    # the viscous path runs on the CUDA cores
    r, s_, t = B.dg_tet_reference_nodes(N)
    wl = make_tet_workload(args.workload, r, s_, t)
    m = wl["mesh"]
    Np = len(r)
    dof_stage = m.K * Np * 5
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = B.dg_create(0, stream.cuda_stream)
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device="cuda")
    p = B.make_params(u_inf=wl["u_inf"], prec=prec, flux=args.flux, av_on=args.tet_av)
    h = B.dg_tet_mesh_upload(ctx, N, m.EToV, m.bc, wl["xyz"], p)
    info = B.dg_mesh_info(ctx, h)
    nvisc = None
    if args.tet_av:
        # troubled cells for the viscous path: every variable times 1.5
        # downstream of the plane x = 1.5 (velocity and sound speed unchanged)
        wl["U0"] = wl["U0"] * np.where(wl["xyz"][..., 0] > 1.5, 1.5, 1.0)[:, None, :]
        from paper_1208_4772_gb300.inputs import states as st3
        wl["dt"] = st3.time_step3(m.verts, wl["U0"], N, cfl=0.3, eps0=0.3)   # the viscous limit as well
    B.dg_set_state(ctx, h, wl["U0"])
    if args.tet_av:
        nvisc = B.dg_av_count(ctx, h)
    tuned = B.dg_autotune(ctx, h, 5)       # elements per tile for this mesh (fixed on the tensor cores)
    step = B.dg_step_lserk if args.integrator == "lserk" else B.dg_step
    nstage = 5 if args.integrator == "lserk" else 3

    def warm():
        for _ in range(args.warmup):
            flush.zero_()
            step(ctx, h, wl["dt"], 1)
        torch.cuda.synchronize()

    warm()
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    clocks.mark()
    times, _, _ = timed_steps(B, ctx, h, wl["dt"], args.steps, stream, flush, torch, step=step)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(sum(times))
    value = dof_stage * nstage * args.steps / (total_ms / 1e3)
    linf, l2 = B.dg_residual(ctx, h, allow_nonfinite=True)
    n_prof = min(args.steps, 200)
    if args.integrator == "ssp3":
        B.dg_set_profiling(ctx, h, 1)
        warm()
        _, kt, launches = timed_steps(B, ctx, h, wl["dt"], n_prof, stream, flush, torch, profiled=True)
        B.dg_set_profiling(ctx, h, 0)
        launch_ms = kt[2] / (3 * n_prof)
        launches = launches * args.steps // n_prof
        if args.tet_av:   # each stage: the sensor, three gradient passes and the stage kernel (events wrap the last)
            launches = args.steps * 3 * 5
    else:
        launch_ms = total_ms / args.steps / 5
        launches = args.steps * 5 * (5 if args.tet_av else 1)
    flops = tet_stage_flops(N) * m.K
    bytes_launch = tet_stage_bytes(m.K, info["curved"], N)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak_tflops = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (launch_ms * 1e-3) / 1e12
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = float(json.load(open(peaks_path))["hbm_gbs"]) if os.path.exists(peaks_path) else 6800.0
    kname = "stage3_tc_kernel" if prec == "tf32" else \
        ("sensor3_kernel + 3 gradient passes + viscous stage3_kernel" if args.tet_av else "stage3_kernel")
    hbm_gbs = bytes_launch / (launch_ms * 1e-3) / 1e9
    if prec == "tf32":
        # the volume products run on the tensor pipe: the bound the kernel is
        # measured against is HBM (its bytes), the FP32-peak figure is kept
        roofline = {"kernel": "%s (tetrahedra, N=%d, %s)" % (kname, N, prec), "bound": "hbm",
                    "achieved": hbm_gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_gbs / hbm,
                    "peak_source": "measured" if os.path.exists(peaks_path) else "fallback",
                    "traffic": traffic_of(args.workload, prec, args.flux, "tet") if args.integrator == "ssp3" else None,
                    "bytes_per_launch": bytes_launch, "avg_launch_ms": launch_ms, "flops_per_launch": flops,
                    "fp32_equivalent_tflops": achieved, "fp32_alu_peak_tflops": peak_tflops}
    else:
        roofline = {"kernel": "%s (tetrahedra, N=%d, %s)" % (kname, N, prec), "bound": "alu",
                    "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock %.0f MHz" % sm_max,
                    "traffic": traffic_of(args.workload, prec, args.flux, "tet") if args.integrator == "ssp3" else None,
                    "flops_per_launch": flops,
                    "bytes_per_launch": bytes_launch, "avg_launch_ms": launch_ms,
                    "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm}
    if args.tet_av:
        roofline["note"] = ("with artificial viscosity the timed unit is the whole viscous stage (five launches); "
                            "flops and bytes are those of the inviscid stage, so the fractions understate the work")
    e2e = None
    if not args.no_e2e:
        step(ctx, h, wl["dt"], 1)
        torch.cuda.synchronize()
        U_host = np.ascontiguousarray(wl["U0"])
        n_e2e = min(args.steps, 500)
        t0 = time.perf_counter()
        B.dg_set_state(ctx, h, U_host)
        step(ctx, h, wl["dt"], n_e2e)
        U_out = B.dg_get_state(ctx, h)
        el = time.perf_counter() - t0
        e2e = {"value": dof_stage * nstage * n_e2e / el, "unit": UNIT, "h2d_bytes_per_step": U_host.nbytes / n_e2e,
               "d2h_bytes_per_step": U_out.nbytes / n_e2e, "host_io": B.dg_host_io(ctx),
               "how": "dg_set_state(host FP64) + %s(%d) + dg_get_state(host FP64), wall clock"
                      % ("dg_step_lserk" if args.integrator == "lserk" else "dg_step", n_e2e)}
    B.dg_destroy(ctx)
    cpu = None
    if not args.no_cpu_baseline:
        path = oracle_inputs_path(wl, args.flux, "tet")
        try:
            cpu = run_cpu_baseline(path, args.cpu_budget_s)
        finally:
            os.unlink(path)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": args.workload, "describe": w["describe"], "K": int(m.K), "N": N, "Np": Np,
                       "variables": 5, "curved_elements": int(info["curved"]), "state_precision": prec,
                       "time_integrator": "LSERK(5,4)" if args.integrator == "lserk" else "SSP-RK3",
                       "flux": args.flux.upper(), "dt": wl["dt"], "dof_per_stage": int(dof_stage),
                       "artificial_viscosity": bool(args.tet_av),
                       "viscous_elements_at_start": nvisc,
                       "l2": "flushed before every timed step (%d MiB memset, outside the step events)"
                             % args.flush_mb,
                       "parallelism": "replicas (one independent solve per GPU)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "tile_e": tuned[0], "autotune_ms_per_step": {str(k): v for k, v in tuned[1].items()},
            "residual_linf": [float(x) for x in linf]}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batch and serving
def make_batch(n, seed0=2000):
    """Seeded batch of n mesh requests (inputs only): K log-uniform in
    [2k, 200k], N uniform in {2..5}, airfoil / cylinder alternating, Mach
    U[0.3, 0.85], AoA U[-2, 4] deg; item i draws from seed seed0 + i."""
    import math
    import numpy as np
    from paper_1208_4772_gb300 import serve
    reqs = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        K = math.exp(rng.uniform(math.log(2000), math.log(200000)))
        n_r = max(2, int(round(math.sqrt(K / 6.0))))
        n_t = max(8, int(round(K / (2 * n_r))))
        reqs.append(serve.Request(rid=i, arrival=0.0, kind="naca" if i % 2 == 0 else "cyl", n_t=n_t, n_r=n_r,
                                  N=int(rng.integers(2, 6)), mach=float(rng.uniform(0.3, 0.85)),
                                  aoa=float(rng.uniform(-2.0, 4.0)), seed=seed0 + i))
    return reqs


def batch_launches_per_step(reqs, prec):
    """Kernels of one batched SSP-RK3 step: per stage one persistent launch
    for the meshes without viscosity (a second one when a degree-6 mesh is
    among them), and on each viscous mesh's branch its gradient and stage
    launches (the sensor is fused into the tensor-core stage kernel; the
    CUDA-core path launches it separately)."""
    plain = [r for r in reqs if not r.av]
    n = 0
    if plain:
        n += 3 * (2 if any(r.N == 6 for r in plain) else 1)
    per_stage = 2 if prec in ("tf32", "bf16x3") else 3
    n += 3 * per_stage * sum(1 for r in reqs if r.av)
    return n


def run_batch(args):
    """All meshes of the batch advanced together by dg_batch_step; one
    timed step = one SSP-RK3 step of every mesh.  The batch's device
    footprint is far above L2, so no flush is needed between steps."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B, serve
    B.load()
    torch.cuda.set_device(0)
    reqs = make_batch(args.batch_meshes)
    nodes = {N: B.dg_reference_nodes(N) for N in range(2, 7)}
    for r in reqs:
        serve.prepare(r, *nodes[r.N], av_mach=args.batch_av_mach)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = B.dg_create(0, stream.cuda_stream)
    hs, dts = [], []
    for r in reqs:
        p = B.make_params(u_inf=r.u_inf, prec=args.prec, av_on=r.av, eps0=r.eps0 if r.av else 0.3)
        hs.append(B.dg_mesh_upload(ctx, r.N, r.mesh.EToE, r.mesh.EToF, r.mesh.bc, r.xy, p))
        B.dg_set_state(ctx, hs[-1], r.U0)
        dts.append(r.dt)
    dev_bytes = sum(B.dg_mesh_bytes(ctx, h) for h in hs)
    tuned = {}
    if args.prec in ("fp32", "fp64"):     # CUDA-core tiles: tuned on the largest mesh of each degree
        for N in sorted(set(r.N for r in reqs)):
            i = max((i for i, r in enumerate(reqs) if r.N == N), key=lambda i: reqs[i].mesh.K)
            tuned[str(N)] = B.dg_autotune(ctx, hs[i], 3)[0]
    for _ in range(args.warmup):
        B.dg_batch_step(ctx, hs, dts, 1)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    times = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.dg_batch_step(ctx, hs, dts, 1)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    clk = clocks.stop()
    total_ms = float(sum(times))
    dof_step = sum(3 * r.mesh.K * (r.N + 1) * (r.N + 2) // 2 * 4 for r in reqs)
    value = dof_step * args.steps / (total_ms / 1e3)
    curved = [int(np.any(r.mesh.bc == 1, axis=1).sum()) for r in reqs]
    bytes_step = sum(3 * stage_kernel_bytes(r.mesh.K, c, r.N, r.av, r.av) for r, c in zip(reqs, curved))
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    achieved = bytes_step / (total_ms / args.steps * 1e-3) / 1e9
    # end to end: host FP64 states in, steps, host FP64 states out
    e2e = None
    if not args.no_e2e:
        t0 = time.perf_counter()
        for r, h in zip(reqs, hs):
            B.dg_set_state(ctx, h, r.U0)
        B.dg_batch_step(ctx, hs, dts, args.steps)
        out_bytes = 0
        for r, h in zip(reqs, hs):
            out_bytes += B.dg_get_state(ctx, h, r.mesh.K, r.U0.shape[2]).nbytes
        el = time.perf_counter() - t0
        e2e = {"value": dof_step * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": sum(r.U0.nbytes for r in reqs) / args.steps,
               "d2h_bytes_per_step": out_bytes / args.steps, "host_io": B.dg_host_io(ctx),
               "how": "dg_set_state x%d (host FP64) + dg_batch_step(%d) + dg_get_state x%d, wall clock"
                      % (len(reqs), args.steps, len(reqs))}
    B.dg_destroy(ctx)
    Ks = [int(r.mesh.K) for r in reqs]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": "batch64", "describe": WORKLOADS["batch64"]["describe"],
                       "meshes": len(reqs), "total_K": int(sum(Ks)), "K_min": min(Ks), "K_max": max(Ks),
                       "viscous_meshes": sum(1 for r in reqs if r.av),
                       "N_counts": {str(N): sum(1 for r in reqs if r.N == N) for N in range(2, 6)},
                       "dof_per_step": int(dof_step), "device_bytes": int(dev_bytes),
                       "tile_e_by_degree": tuned or "32 (tensor-core tiles)",
                       "state_precision": "fp32", "products": args.prec, "time_integrator": "SSP-RK3",
                       "l2": "not flushed: the batch's device footprint is far above L2",
                       "parallelism": "one GPU, all meshes in one persistent launch per stage"},
            "roofline": {"kernel": "batched stage kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
                         "bytes_per_step": bytes_step},
            "cpu_baseline": None, "e2e": e2e, "gpu_launches": args.steps * batch_launches_per_step(reqs, args.prec),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Continuous batching over Poisson arrivals (serve.ServeLoop): latency
    from arrival to result and the throughput over the run.  First all
    requests at once (arrival rate unbounded) to measure the service rate
    mu = requests / makespan, then Poisson arrivals at the multiples of mu
    given by --serve-rates; the line's value and latencies are those of the
    1x run."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B, serve
    B.load()
    torch.cuda.set_device(0)
    nodes = {N: B.dg_reference_nodes(N) for N in range(2, 7)}
    base = serve.poisson_requests(args.serve_requests, 1.0, seed=3000)
    gaps = np.diff([0.0] + [r.arrival for r in base])     # unit-rate inter-arrival times

    def requests_at(rate):
        reqs = serve.poisson_requests(args.serve_requests, 1.0, seed=3000)
        t = np.cumsum(gaps / rate) if np.isfinite(rate) else np.zeros(len(reqs))
        for r, ti in zip(reqs, t):
            r.arrival = float(ti)
            serve.prepare(r, *nodes[r.N], av_mach=args.serve_av_mach)
        return reqs

    def one_run(rate):
        reqs = requests_at(rate)
        ctx = B.dg_create(0)
        loop = serve.ServeLoop(ctx, budget_bytes=args.serve_budget_gb * 1e9, check_every=100,
                               max_steps=args.serve_max_steps, prec=args.prec)
        t0 = time.perf_counter()
        done = loop.run(reqs, keep_states=False)
        wall = time.perf_counter() - t0
        B.dg_destroy(ctx)
        st = serve.latency_stats(done)
        return {"arrival_rate_per_s": rate if np.isfinite(rate) else None, "wall_s": wall,
                "throughput_dof_per_s": st["dof_updates"] / wall, "requests_per_s": len(done) / wall,
                "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"], "mean_service_s": st["service_s"],
                "peak_active": loop.peak_active, "peak_bytes": loop.peak_used,
                "retired": {k: sum(1 for r in done if r.reason == k) for k in sorted(set(r.reason for r in done))},
                "viscous_requests": sum(1 for r in done if r.av),
                "restarts_with_more_viscosity": sum(r.retries for r in done),
                "nonfinite": [[r.rid, r.kind, r.N, int(r.K), round(r.mach, 3)] for r in done if r.reason == "nonfinite"],
                "overlap": loop.overlap()}

    clocks = ClockSampler(0)
    clocks.start()
    calib = one_run(float("inf"))
    mu = args.serve_requests / calib["wall_s"]
    sweep = {}
    for mult in [float(x) for x in args.serve_rates.split(",") if x]:
        sweep["%gx" % mult] = one_run(mult * mu)
    clk = clocks.stop()
    head = sweep.get("1x") or calib
    line = {"metric": METRIC, "value": head["throughput_dof_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": "serve", "describe": WORKLOADS["serve"]["describe"],
                       "requests": args.serve_requests, "service_rate_per_s": mu,
                       "step_cap": args.serve_max_steps, "check_every": 100, "drop": 1e-6,
                       "budget_GB": args.serve_budget_gb, "products": args.prec,
                       "artificial_viscosity_from_mach": args.serve_av_mach},
            "latency": {"p50_s": head["p50_s"], "p99_s": head["p99_s"], "mean_s": head["mean_s"]},
            "all_at_once": calib, "rates": sweep,
            "cpu_baseline": None, "e2e": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_prefine(args):
    """Time to a steady residual: N = 4 from the freestream for
    --prefine-max-steps steps, against degrees 2 and 3 first (each to a
    residual drop of --prefine-drop or --prefine-max-steps-low steps), then
    N = 4 until it reaches the residual the direct run ended with."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1208_4772_gb300 import binding as B, prefine
    from paper_1208_4772_gb300.inputs import meshes, states
    B.load()
    torch.cuda.set_device(0)
    mesh = meshes.cylinder_channel(n_t=160, n_r=48, seed=1002)
    ui = states.freestream(0.38, 0.0)
    ctx = B.dg_create(0)
    clocks = ClockSampler(0)
    clocks.start()
    h, direct = prefine.run_levels(ctx, mesh, [4], ui, prec=args.prec, drop=args.prefine_drop,
                                   max_steps=args.prefine_max_steps)
    B.dg_mesh_free(ctx, h)
    target = direct[-1]["r_last"]
    h, levels = prefine.run_levels(ctx, mesh, [2, 3, 4], ui, prec=args.prec, drop=args.prefine_drop, target=target,
                                   max_steps=args.prefine_max_steps, max_steps_low=args.prefine_max_steps_low)
    B.dg_mesh_free(ctx, h)
    clk = clocks.stop()
    B.dg_destroy(ctx)
    t_direct = sum(l["seconds"] for l in direct)
    t_pref = sum(l["seconds"] for l in levels)
    dof = sum(l["dof_updates"] for l in direct + levels)
    strip = lambda ls: [{k: v for k, v in l.items() if k != "history"} for l in ls]
    line = {"metric": METRIC, "value": dof / (t_direct + t_pref), "unit": UNIT, "n_gpus": 1, "steps": None,
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": "prefine", "describe": WORKLOADS["prefine"]["describe"], "K": int(mesh.K),
                       "drop_lower_levels": args.prefine_drop, "max_steps_N4": args.prefine_max_steps,
                       "max_steps_lower_levels": args.prefine_max_steps_low,
                       "products": args.prec},
            "prefine": {"direct_N4_s": t_direct, "levels_2_3_4_s": t_pref, "speedup": t_direct / t_pref,
                        "target_residual": target, "direct": strip(direct), "levels": strip(levels)},
            "cpu_baseline": None, "e2e": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    faulthandler.enable()
    args = parse_args()
    if args.cpu_sample:
        print(json.dumps(cpu_worker(args.cpu_sample, args.cpu_start, args.cpu_budget_s)))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload]["kind"] in ("batch", "serve", "prefine", "tet") and int(os.environ.get("RANK", "0")) != 0:
        return 0    # these workloads run on one GPU: under a multi-rank launch rank 0 alone runs and prints
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "prefine":
        return run_prefine(args)
    if WORKLOADS[args.workload]["kind"] == "tet":
        return run_tet(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

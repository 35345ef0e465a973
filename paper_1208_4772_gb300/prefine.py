"""p-refinement driver (paper Sec. 5, Table 2): converge a steady flow at a
low degree, embed the solution exactly at the next degree (dg_prolong), and
continue, so that the expensive high-degree steps start from a converged
low-degree field instead of the freestream.

run_levels(ctx, mesh, levels, ...) uploads the mesh at each degree in turn
(curved nodes for that degree; a triangle mesh through dg_mesh_upload, a
tetrahedral one -- four vertices per element -- through dg_tet_mesh_upload
with its map applied to the nodes), starts the first level from the freestream,
advances each level with dg_step in blocks of check_every steps and stops it
when the largest per-variable L2 residual norm has dropped by `drop` from the
level's first check, or reaches `target` (absolute), or max_steps.  The step
size is recomputed per level from the level's state (per-level dt).
"""
import math
import time

import numpy as np

from . import binding as B
from .inputs import curving, meshes3d, states


def _is_tet(mesh):
    """A tetrahedral mesh: four vertices per element (triangle meshes
    carry EToV too, with three)."""
    return mesh.EToV.shape[1] == 4


def _upload(ctx, mesh, N, u_inf, prec, av_on):
    """Upload the mesh at degree N; returns (handle, nodes, variables)."""
    p = B.make_params(u_inf=u_inf, prec=prec, av_on=av_on)
    if _is_tet(mesh):
        r, s, t = B.dg_tet_reference_nodes(N)
        X = meshes3d.node_coords(mesh, r, s, t)
        return B.dg_tet_mesh_upload(ctx, N, mesh.EToV, mesh.bc, X, p), len(r), 5
    r, s = B.dg_reference_nodes(N)
    xy, _ = curving.curve_mesh(mesh, N, r, s)
    return B.dg_mesh_upload(ctx, N, mesh.EToE, mesh.EToF, mesh.bc, xy, p), len(r), 4


def run_levels(ctx, mesh, levels, u_inf, prec="tf32", drop=1e-2, target=None, check_every=100, max_steps=20000,
               cfl=0.3, max_steps_low=None, clock=time.perf_counter, av_on=False):
    """Returns (handle of the last level's mesh, per-level report).  Levels
    below the last stop at `drop` or max_steps_low (default max_steps); the
    last at `target` when given, else at `drop`, or max_steps."""
    prev, prevN, report = None, None, []
    tet = _is_tet(mesh)
    for N in levels:
        h, Np, nvar = _upload(ctx, mesh, N, u_inf, prec, av_on)
        if prev is None:
            B.dg_set_state(ctx, h, (states.uniform_state3 if tet else states.uniform_state)(mesh.K, Np, u_inf))
        else:
            B.dg_prolong(ctx, prev, h)
            B.dg_mesh_free(ctx, prev)
        U = B.dg_get_state(ctx, h, mesh.K, Np)
        dt = (states.time_step3 if tet else states.time_step)(mesh.verts, U, N, cfl=cfl)
        t0 = clock()
        steps, r0, res, hist = 0, None, math.nan, []
        last = N == levels[-1]
        cap = max_steps if (last or max_steps_low is None) else max_steps_low
        while steps < cap:
            n = min(check_every, cap - steps)
            B.dg_step(ctx, h, dt, n)
            steps += n
            _, l2 = B.dg_residual(ctx, h, allow_nonfinite=True)
            res = float(np.max(l2))
            hist.append(res)
            if r0 is None:
                r0 = res
            if not math.isfinite(res):
                break
            if (last and target is not None and res <= target) or (not (last and target is not None)
                                                                    and res <= drop * r0):
                break
        B.dg_sync(ctx)
        report.append(dict(N=N, K=int(mesh.K), steps=steps, seconds=clock() - t0, dt=dt, r_first=r0, r_last=res,
                           dof_updates=3.0 * steps * mesh.K * Np * nvar, history=hist))
        prev, prevN = h, N
    return prev, report

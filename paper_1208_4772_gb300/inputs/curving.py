"""Isoparametric wall curving, FP64 host setup (paper Sec. 3 in 2D).

The curved element map lives in the same degree-N Lagrange basis as the
solution, so only the displacement of the collocation nodes is needed.  In
2D only the elements with a face on the wall move, and the nodes on their two
other faces stay where they are, so neighbours are untouched (Sec. 3).  The
displacement of a wall element is the degree-N finite-element solution of
linear elasticity (Sec. 3),

    div sigma = 0,  sigma = lambda tr(eps) I + 2 mu eps,
    lambda = nu E / ((1+nu)(1-2nu)),  mu = E / (2(1+nu)),

on that straight element, with u = g on the wall face (g = closest point on
the exact curve minus the straight node, Sec. 3 closest-point problem solved
by Gauss-Newton) and u = 0 on the other two faces.  Because the two other
faces are clamped, the band of wall elements decouples into one small solve
per element.  E drops out; nu defaults to 0.45.

Inputs only: the reference node set (r, s) is passed in by the caller, and
the Lagrange basis of the elasticity solve is built here from monomials.
"""
import numpy as np

from .meshes import BC_WALL, straight_nodes


def _monomials(N, r, s):
    P = [(a, d - a) for d in range(N + 1) for a in range(d + 1)]
    V = np.stack([r ** a * s ** b for (a, b) in P], axis=-1)
    Vr = np.stack([a * r ** max(a - 1, 0) * s ** b if a > 0 else 0 * r for (a, b) in P], axis=-1)
    Vs = np.stack([b * r ** a * s ** max(b - 1, 0) if b > 0 else 0 * r for (a, b) in P], axis=-1)
    return V, Vr, Vs


def _triangle_rule(n):
    """Duffy-collapsed Gauss-Legendre rule on T (exact to degree 2n-2)."""
    a, wa = np.polynomial.legendre.leggauss(n)
    R, S, W = [], [], []
    for j in range(n):
        for i in range(n):
            R.append(0.5 * (1 + a[i]) * (1 - a[j]) - 1)
            S.append(a[j])
            W.append(wa[i] * wa[j] * 0.5 * (1 - a[j]))
    return np.array(R), np.array(S), np.array(W)


def _on_face(r, s, f, tol=1e-10):
    if f == 0:
        return np.abs(s + 1) < tol
    if f == 1:
        return np.abs(r + s) < tol
    return np.abs(r + 1) < tol


def elastic_fill(verts, g, interior, Lr, Ls, qw, nu):
    """Degree-N linear-elasticity displacement [Np, 2] on the straight
    triangle verts [3, 2]: Dirichlet values g on the non-interior nodes, the
    interior nodes from K_II u_I = -K_IB u_B (plane strain, E = 1)."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    v0, v1, v2 = verts
    xr, xs = 0.5 * (v1 - v0), 0.5 * (v2 - v0)
    J = xr[0] * xs[1] - xs[0] * xr[1]
    rx, ry, sx, sy = xs[1] / J, -xs[0] / J, -xr[1] / J, xr[0] / J
    Lx = Lr * rx + Ls * sx
    Ly = Lr * ry + Ls * sy
    w = qw * J
    Np = g.shape[0]
    # vector unknowns ordered (u_0..u_{Np-1}, v_0..v_{Np-1})
    Kxx = (lam + 2 * mu) * (Lx.T * w) @ Lx + mu * (Ly.T * w) @ Ly
    Kyy = (lam + 2 * mu) * (Ly.T * w) @ Ly + mu * (Lx.T * w) @ Lx
    Kxy = lam * (Lx.T * w) @ Ly + mu * (Ly.T * w) @ Lx
    Kmat = np.block([[Kxx, Kxy], [Kxy.T, Kyy]])
    free = np.concatenate([interior, interior])
    u = np.concatenate([g[:, 0], g[:, 1]])
    if np.any(free):
        rhs = -Kmat[np.ix_(free, ~free)] @ u[~free]
        u[free] = np.linalg.solve(Kmat[np.ix_(free, free)], rhs)
    return np.stack([u[:Np], u[Np:]], axis=-1)


def basis_pieces(N, r, s):
    """Lagrange-basis derivatives on the nodes (r, s) at the elasticity
    quadrature points, and that rule's weights."""
    Vn, _, _ = _monomials(N, r, s)
    C = np.linalg.inv(Vn)
    qr, qs, qw = _triangle_rule(N + 1)
    _, Mr, Ms = _monomials(N, qr, qs)
    return Mr @ C, Ms @ C, qw


def curve_mesh(mesh, N, r, s, nu=0.45):
    """Collocation-node coordinates [K, Np, 2] for mesh at degree N on the
    reference nodes (r, s); wall elements curved onto mesh.curve.  Returns
    (node_xy, curved_mask)."""
    node_xy = straight_nodes(mesh.verts, r, s)
    K, Np = node_xy.shape[:2]
    curved = np.zeros(K, dtype=bool)
    if mesh.curve is None or N < 2:
        return node_xy, curved
    walls = np.nonzero(mesh.bc == BC_WALL)
    if len(walls[0]) == 0:
        return node_xy, curved

    Lr, Ls, qw = basis_pieces(N, r, s)
    boundary = _on_face(r, s, 0) | _on_face(r, s, 1) | _on_face(r, s, 2)
    interior = ~boundary
    is_vertex = ((np.abs(r + 1) < 1e-10) | (np.abs(r - 1) < 1e-10)) & ((np.abs(s + 1) < 1e-10) | (np.abs(s - 1) < 1e-10))
    param = mesh.meta.get("wall_param")
    n_t = mesh.meta.get("n_t")

    for k, f in zip(*walls):
        k, f = int(k), int(f)
        X = node_xy[k].copy()
        on = _on_face(r, s, f)
        # closest point on the curve for the wall-face nodes
        if param is not None:
            ia, ib = int(mesh.EToV[k, f]), int(mesh.EToV[k, (f + 1) % 3])
            if {ia, ib} == {n_t - 1, 0}:
                ia, ib = (n_t if ia == 0 else ia), (n_t if ib == 0 else ib)
            pa, pb = param[ia], param[ib]
            va, vb = mesh.verts[k, f], mesh.verts[k, (f + 1) % 3]
            seg = vb - va
            t = np.clip(((X[on] - va) @ seg) / (seg @ seg), 0.0, 1.0)
            target, _ = mesh.curve.project(X[on], pa + t * (pb - pa), min(pa, pb), max(pa, pb))
        else:
            target, _ = mesh.curve.project(X[on])
        g = np.zeros_like(X)
        g[on] = target - X[on]
        g[is_vertex] = 0.0          # vertices already lie on the curve; keep them shared exactly
        u = elastic_fill(mesh.verts[k], g, interior, Lr, Ls, qw, nu)
        node_xy[k] += u
        curved[k] = True
    return node_xy, curved

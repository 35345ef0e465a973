"""Reference tetrahedron: basis, nodes, cubature, face rule and operators for
the 3D form of the method (paper Sec. 2, which is written for tetrahedra).

Reference element T3 = {(r, s, t): r, s, t >= -1, r + s + t <= -1} with
vertices v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1), v3 = (-1,-1,1).
Faces, each listed with its vertices in the order that makes
(vb - va) x (vc - va) point outward:
    face 0: (v0, v2, v1)   t = -1
    face 1: (v0, v1, v3)   s = -1
    face 2: (v1, v2, v3)   r + s + t = -1
    face 3: (v0, v3, v2)   r = -1

Basis (paper Sec. 2: orthonormal, hierarchical modal set), in the collapsed
coordinates a = 2(1+r)/(-s-t) - 1, b = 2(1+s)/(1-t) - 1, c = t:
    psi_ijk = 2 sqrt(2) P~_i^(0,0)(a) P~_j^(2i+1,0)(b) (1-b)^i
                         P~_k^(2i+2j+2,0)(c) (1-c)^(i+j),   i + j + k <= N,
with normalised Jacobi polynomials P~; modes ordered by total degree, then
i, then j.  The factor 2 sqrt(2) makes int_T3 psi^2 = 1, since
dr ds dt = (1-b)(1-c)^2 / 8 da db dc.

Nodes: warp & blend after Warburton (2006) with blending parameter 0, the
3D counterpart of the triangle nodes in oracle/nodes.py (see
`warp_blend_nodes_3d`).  Canonical order: equidistant lattice index k (t)
outer, j (s) middle, i (r) inner.

Volume rule: collapsed product rule with q points per direction,
Gauss-Legendre in a, Gauss-Jacobi(1,0) in b, Gauss-Jacobi(2,0) in c (the
(1-b) and (1-c)^2 factors of the Jacobian carried by the weights), exact to
total degree 2q - 1; q = ceil((3N+1)/2) as in 2D.

Face rule: the triangle rule of oracle/quadrature.py (q^2 points) placed on
the face in a canonical frame: the face's three vertices ordered by their
global vertex numbers.  Both elements sharing a face then evaluate the face
integral at the same physical points with the same weights, whatever their
local numbering (the collapsed rule is not symmetric under vertex
permutations).

Test infrastructure only.
"""
from itertools import permutations
from math import sqrt

import numpy as np
from scipy.special import roots_jacobi

from . import basis as basis2
from . import nodes as nodes2
from . import quadrature as quad2

VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
FACE_VERTS = ((0, 2, 1), (0, 1, 3), (1, 2, 3), (0, 3, 2))
# the six orderings of a face's three vertices, indexed by orientation code
PERMS3 = tuple(permutations(range(3)))


def n_modes(N):
    """N_p = (N+1)(N+2)(N+3)/6 (paper Sec. 2 with d = 3)."""
    return (N + 1) * (N + 2) * (N + 3) // 6


def n_face_nodes(N):
    return (N + 1) * (N + 2) // 2


def mode_list(N):
    return [(i, j, d - i - j) for d in range(N + 1) for i in range(d + 1) for j in range(d - i + 1)]


def mode_degrees(N):
    return np.array([sum(m) for m in mode_list(N)], dtype=np.int64)


# ------------------------------------------------------------------ basis
def collapse(r, s, t):
    r, s, t = (np.asarray(x, dtype=np.float64) for x in (r, s, t))
    den_a = -s - t
    a = np.where(np.abs(den_a) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(den_a) > 1e-14, den_a, 1.0) - 1.0, -1.0)
    den_b = 1.0 - t
    b = np.where(np.abs(den_b) > 1e-14, 2.0 * (1.0 + s) / np.where(np.abs(den_b) > 1e-14, den_b, 1.0) - 1.0, -1.0)
    return a, b, t


def vandermonde(N, r, s, t):
    """V_ij = psi_j(x_i)."""
    a, b, c = collapse(r, s, t)
    cols = []
    for (i, j, k) in mode_list(N):
        cols.append(2.0 * sqrt(2.0) * basis2.jacobi(a, 0.0, 0.0, i)
                    * basis2.jacobi(b, 2.0 * i + 1.0, 0.0, j) * (1.0 - b) ** i
                    * basis2.jacobi(c, 2.0 * i + 2.0 * j + 2.0, 0.0, k) * (1.0 - c) ** (i + j))
    return np.stack(cols, axis=1)


def grad_vandermonde(N, r, s, t):
    """(V_r, V_s, V_t) by the chain rule through the collapsed coordinates:
        da/dr = 4/((1-b)(1-c)),  da/ds = da/dt = 2(1+a)/((1-b)(1-c)),
        db/ds = 2/(1-c),         db/dt = (1+b)/(1-c),        dc/dt = 1.
    Points must keep away from the collapsed edges b = 1 and c = 1 (cubature
    and face-rule points do)."""
    a, b, c = collapse(r, s, t)
    if np.any(b > 1.0 - 1e-12) or np.any(c > 1.0 - 1e-12):
        raise ValueError("gradient requested on a collapsed edge")
    K = 2.0 * sqrt(2.0)
    Vr, Vs, Vt = [], [], []
    for (i, j, k) in mode_list(N):
        al, ak = 2.0 * i + 1.0, 2.0 * i + 2.0 * j + 2.0
        fa, dfa = basis2.jacobi(a, 0.0, 0.0, i), basis2.djacobi(a, 0.0, 0.0, i)
        gb, dgb = basis2.jacobi(b, al, 0.0, j), basis2.djacobi(b, al, 0.0, j)
        hc, dhc = basis2.jacobi(c, ak, 0.0, k), basis2.djacobi(c, ak, 0.0, k)
        ob, oc = 1.0 - b, 1.0 - c
        # the three partial derivatives in collapsed coordinates
        psi_a = dfa * gb * ob ** i * hc * oc ** (i + j)
        dgb_full = dgb * ob ** i - (i * gb * ob ** (i - 1) if i > 0 else 0.0)
        psi_b = fa * dgb_full * hc * oc ** (i + j)
        dhc_full = dhc * oc ** (i + j) - ((i + j) * hc * oc ** (i + j - 1) if i + j > 0 else 0.0)
        psi_c = fa * gb * ob ** i * dhc_full
        dr = psi_a * 4.0 / (ob * oc)
        ds = psi_a * 2.0 * (1.0 + a) / (ob * oc) + psi_b * 2.0 / oc
        dt = psi_a * 2.0 * (1.0 + a) / (ob * oc) + psi_b * (1.0 + b) / oc + psi_c
        Vr.append(K * dr)
        Vs.append(K * ds)
        Vt.append(K * dt)
    return np.stack(Vr, axis=1), np.stack(Vs, axis=1), np.stack(Vt, axis=1)


# ------------------------------------------------------------------ nodes
_EQ = np.array([[-1.0, -1.0 / sqrt(3.0), -1.0 / sqrt(6.0)],
                [1.0, -1.0 / sqrt(3.0), -1.0 / sqrt(6.0)],
                [0.0, 2.0 / sqrt(3.0), -1.0 / sqrt(6.0)],
                [0.0, 0.0, 3.0 / sqrt(6.0)]])   # equilateral tetrahedron, edge 2


def lattice_3d(N):
    """Equidistant barycentric lattice [Np, 4] in the canonical order (k outer,
    j middle, i inner); columns weight v0..v3."""
    L = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - j - k):
                L.append((1.0 - (i + j + k) / N, i / N, j / N, k / N))
    return np.array(L)


def warp_blend_nodes_3d(N):
    """Warp & blend nodes (alpha = 0) on T3; returns (r, s, t).

    Construction (written from the published method):
      1. the equidistant lattice, placed on the equilateral tetrahedron;
      2. for each face (opposite barycentric L_a, face barycentrics
         L_b, L_c, L_d) the 2D face warp: for each edge (P, Q) of the face,
         4 L_P L_Q w(L_Q - L_P) / (1 - (L_Q - L_P)^2) along the unit edge
         direction, w being the degree-N equidistant -> GLL shift
         interpolant (oracle/nodes.py);
      3. blended into the interior by
         L_b L_c L_d / ((L_b + L_a/2)(L_c + L_a/2)(L_d + L_a/2)),
         which is 1 on the face and 0 on the other three;
      4. a node on an edge or vertex of a face (L_a = 0 and one of
         L_b, L_c, L_d = 0) takes that face's warp alone (the blend is 0/0
         there; the faces sharing an edge agree on it: the GLL shift);
      5. mapped back to T3 by barycentric coordinates.
    Each face then carries the triangle's warp & blend nodes and each edge
    the GLL points."""
    if N == 0:
        return np.array([-0.5]), np.array([-0.5]), np.array([-0.5])
    L = lattice_3d(N)
    X = L @ _EQ
    shift = np.zeros_like(X)
    tol = 1e-10
    done = np.zeros(len(L), dtype=bool)
    for fa in range(4):
        others = [v for v in range(4) if v != fa]
        La = L[:, fa]
        warp = np.zeros_like(X)
        for (p, q) in ((others[0], others[1]), (others[1], others[2]), (others[2], others[0])):
            d = _EQ[q] - _EQ[p]
            d = d / np.linalg.norm(d)
            tt = L[:, q] - L[:, p]
            warp += np.outer(4.0 * L[:, p] * L[:, q] * nodes2._warp_factor(N, tt), d)
        Lb, Lc, Ld = L[:, others[0]], L[:, others[1]], L[:, others[2]]
        den = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La)
        blend = np.where(den > tol, Lb * Lc * Ld / np.where(den > tol, den, 1.0), 0.0)
        on_face_edge = (La < tol) & (((Lb > tol).astype(int) + (Lc > tol) + (Ld > tol)) < 3)
        shift += blend[:, None] * warp
        take = on_face_edge & ~done
        shift[take] = warp[take]
        done |= take
    X = X + shift
    # barycentrics on the equilateral tetrahedron, then the same combination
    # of the reference vertices
    M = np.vstack([_EQ.T, np.ones(4)])
    lam = np.linalg.solve(M, np.vstack([X.T, np.ones(len(X))]))
    P = lam.T @ VERTS
    return P[:, 0], P[:, 1], P[:, 2]


# ------------------------------------------------------------------ rules
def tet_cubature(q):
    """Collapsed rule on T3: (r, s, t, w); c index outer, b middle, a inner."""
    a, wa = np.polynomial.legendre.leggauss(q)
    b, wb = roots_jacobi(q, 1.0, 0.0)
    c, wc = roots_jacobi(q, 2.0, 0.0)
    R, S, Tt, W = [], [], [], []
    for kc in range(q):
        for jb in range(q):
            for ia in range(q):
                R.append(0.25 * (1.0 + a[ia]) * (1.0 - b[jb]) * (1.0 - c[kc]) - 1.0)
                S.append(0.5 * (1.0 + b[jb]) * (1.0 - c[kc]) - 1.0)
                Tt.append(c[kc])
                W.append(wa[ia] * wb[jb] * wc[kc] / 8.0)
    return np.array(R), np.array(S), np.array(Tt), np.array(W)


def face_rule(q):
    """Triangle rule for the faces: barycentrics mu [Ng, 3] of the points in
    a face frame (mu_0 at the frame's first vertex) and weights w [Ng] for
    the reference triangle of area 2."""
    u, v, w = quad2.triangle_cubature(q)
    mu = np.stack([-(u + v) / 2.0, (1.0 + u) / 2.0, (1.0 + v) / 2.0], axis=1)
    return mu, w


def face_points(mu, f, order):
    """Reference coordinates [Ng, 3] on face f of the points with frame
    barycentrics mu, when the frame's vertex m is the face's local vertex
    order[m] (a permutation of 0, 1, 2 of FACE_VERTS[f])."""
    fv = FACE_VERTS[f]
    P = np.zeros((len(mu), 3))
    for m in range(3):
        P += mu[:, m:m + 1] * VERTS[fv[order[m]]][None, :]
    return P


class ReferenceTet:
    """Operators of degree N on T3 (test infrastructure):
      V, Vinv at the nodes; I_cub, D_r, D_s, D_t at the cubature points;
      for each face f and frame order o (PERMS3): I_g[f][o] and the
      derivative matrices at the face points (for curved face normals)."""

    def __init__(self, N, q=None):
        self.N = N
        self.Np = n_modes(N)
        self.q = quad2.default_q(N) if q is None else q
        self.r, self.s, self.t = warp_blend_nodes_3d(N)
        self.V = vandermonde(N, self.r, self.s, self.t)
        self.Vinv = np.linalg.inv(self.V)
        self.rq, self.sq, self.tq, self.wq = tet_cubature(self.q)
        self.Nq = len(self.wq)
        self.Icub = vandermonde(N, self.rq, self.sq, self.tq) @ self.Vinv
        Vr, Vs, Vt = grad_vandermonde(N, self.rq, self.sq, self.tq)
        self.Dr, self.Ds, self.Dt = Vr @ self.Vinv, Vs @ self.Vinv, Vt @ self.Vinv
        self.mu, self.wg = face_rule(self.q)
        self.Ng = len(self.wg)
        shape = (4, 6, self.Ng, self.Np)
        self.Ig = np.zeros(shape)
        self.Drg, self.Dsg, self.Dtg = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        self.face_xyz = np.zeros((4, 6, self.Ng, 3))
        for f in range(4):
            for o, order in enumerate(PERMS3):
                P = face_points(self.mu, f, order)
                self.face_xyz[f, o] = P
                self.Ig[f, o] = vandermonde(N, *P.T) @ self.Vinv
                gr, gs, gt = grad_vandermonde(N, *P.T)
                self.Drg[f, o] = gr @ self.Vinv
                self.Dsg[f, o] = gs @ self.Vinv
                self.Dtg[f, o] = gt @ self.Vinv
        # reference tangents of each face's own parametrisation (u, v):
        # d/du = (vb - va)/2, d/dv = (vc - va)/2 for FACE_VERTS[f] = (a, b, c)
        self.tan_u = np.array([(VERTS[fv[1]] - VERTS[fv[0]]) / 2.0 for fv in FACE_VERTS])
        self.tan_v = np.array([(VERTS[fv[2]] - VERTS[fv[0]]) / 2.0 for fv in FACE_VERTS])

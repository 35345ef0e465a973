"""Collocation nodes on the reference triangle.

Paper Sec. 2 takes the collocation points r_i "according to Warburton 2006"
(the explicit warp & blend construction).  The paper does not print the
blending parameter alpha; this oracle uses alpha = 0 (the closed-form
construction with Gauss-Lobatto-Legendre points on every edge).

Construction (written from the published method):
  1. equidistant barycentric points (lA, lB, lC) = ((N-i-j)/N, i/N, j/N),
     ordered with j (the s index) outer and i (the r index) inner;
  2. placed on the equilateral triangle A=(-1,-1/sqrt3), B=(1,-1/sqrt3),
     C=(0,2/sqrt3), whose edges all have length 2;
  3. for each edge (P, Q) with barycentrics (lP, lQ) the point moves along
     the unit edge direction by 4 lP lQ * w(lQ - lP) / (1 - (lQ - lP)^2),
     where w(t) is the degree-N interpolant on equidistant points of the
     shift from equidistant to GLL points;
  4. mapped back to T by barycentric coordinates.
On each edge the blend 4 lP lQ equals 1 - t^2, so edge nodes land exactly on
the GLL points.

Test infrastructure only.
"""
import numpy as np

SQRT3 = np.sqrt(3.0)


def gll_points(N):
    """Gauss-Lobatto-Legendre points on [-1,1]: +-1 and the roots of P_N'."""
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots()
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def _warp_factor(N, t):
    req = np.linspace(-1.0, 1.0, N + 1)
    shift = gll_points(N) - req
    w = np.zeros_like(t)
    for i in range(N + 1):
        ell = np.ones_like(t)
        for m in range(N + 1):
            if m != i:
                ell = ell * (t - req[m]) / (req[i] - req[m])
        w = w + shift[i] * ell
    interior = np.abs(t) < 1.0 - 1e-10
    return np.where(interior, w / np.where(interior, 1.0 - t * t, 1.0), 0.0)


def warp_blend_nodes(N):
    """Return (r, s), each of length N_p, in the canonical node order."""
    if N == 0:
        return np.array([-1.0 / 3.0]), np.array([-1.0 / 3.0])
    lA, lB, lC = [], [], []
    for j in range(N + 1):
        for i in range(N + 1 - j):
            lB.append(i / N)
            lC.append(j / N)
            lA.append(1.0 - i / N - j / N)
    lA, lB, lC = map(np.array, (lA, lB, lC))
    A = np.array([-1.0, -1.0 / SQRT3])
    B = np.array([1.0, -1.0 / SQRT3])
    C = np.array([0.0, 2.0 / SQRT3])
    P = np.outer(lA, A) + np.outer(lB, B) + np.outer(lC, C)
    disp = np.zeros_like(P)
    for (lp, lq, Pp, Pq) in ((lA, lB, A, B), (lB, lC, B, C), (lC, lA, C, A)):
        t = lq - lp
        direction = (Pq - Pp) / np.linalg.norm(Pq - Pp)
        disp += np.outer(4.0 * lp * lq * _warp_factor(N, t), direction)
    P = P + disp
    # back to barycentrics on the equilateral triangle, then to T
    M = np.array([[A[0], B[0], C[0]], [A[1], B[1], C[1]], [1.0, 1.0, 1.0]])
    lam = np.linalg.solve(M, np.vstack([P[:, 0], P[:, 1], np.ones(len(P))]))
    r = -lam[0] + lam[1] - lam[2]
    s = -lam[0] - lam[1] + lam[2]
    return r, s

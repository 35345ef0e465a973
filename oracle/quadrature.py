"""Volume cubature and edge quadrature on the reference triangle.

Paper Sec. 2 integrates volume terms with a cubature rule r_i^cub (weights
W_i^cub) and face terms with a Gauss rule r_i^g (weights W_i^g), and Sec. 4
asks for a "very high order" rule because the rational Jacobian of curved
elements enters the integrands.  The paper does not fix the 2D rules, so
this oracle reads them as:

  * volume: the collapsed-coordinate (Stroud conical) product rule with q
    points per direction, Gauss-Legendre in a and Gauss-Jacobi(1,0) in b,
    exact for all polynomials of total degree <= 2q - 1;
  * faces: q-point Gauss-Legendre on each edge, exact to degree 2q - 1;

with q = ceil((3N + 1) / 2), so both are exact to degree >= 3N.

Test infrastructure only.
"""
import numpy as np
from scipy.special import roots_jacobi


def default_q(N):
    return (3 * N + 2) // 2


def gauss_legendre(q):
    return np.polynomial.legendre.leggauss(q)


def gauss_jacobi_10(q):
    """Gauss rule for the weight (1 - x) on [-1, 1] (library routine)."""
    x, w = roots_jacobi(q, 1.0, 0.0)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def triangle_cubature(q):
    """Collapsed rule on T.  Returns (r, s, w); order: b index outer, a inner.

    r = (1+a)(1-b)/2 - 1, s = b, and dr ds = (1-b)/2 da db, the factor (1-b)
    being carried by the Gauss-Jacobi(1,0) weights.
    """
    a, wa = gauss_legendre(q)
    b, wb = gauss_jacobi_10(q)
    rr, ss, ww = [], [], []
    for j in range(q):
        for i in range(q):
            rr.append(0.5 * (1.0 + a[i]) * (1.0 - b[j]) - 1.0)
            ss.append(b[j])
            ww.append(0.5 * wa[i] * wb[j])
    return np.array(rr), np.array(ss), np.array(ww)


def face_points(t):
    """Map the edge parameter t in [-1, 1] to (r, s) on each face of T.

    Face f runs from vertex f to vertex (f+1) mod 3 of (-1,-1), (1,-1), (-1,1):
      face 0: (t, -1);  face 1: (-t, t);  face 2: (-1, -t).
    Returns arrays r[f, g], s[f, g] and the constant (dr/dt, ds/dt) per face.
    """
    t = np.asarray(t, dtype=np.float64)
    r = np.stack([t, -t, -np.ones_like(t)])
    s = np.stack([-np.ones_like(t), t, -t])
    drdt = np.array([1.0, -1.0, 0.0])
    dsdt = np.array([0.0, 1.0, -1.0])
    return r, s, drdt, dsdt

"""Orthonormal, hierarchical modal basis on the reference triangle.

Paper Sec. 2 ("orthonormal, hierarchical set of modal basis functions psi_i on
the reference element") in 2D: the reference triangle is
T = {(r, s): r, s >= -1, r + s <= 0} with vertices (-1,-1), (1,-1), (-1,1).
The basis is the Dubiner/Koornwinder product of Jacobi polynomials in the
collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s:

    psi_ij(r, s) = sqrt(2) * P~_i^(0,0)(a) * P~_j^(2i+1,0)(b) * (1-b)^i,

i + j <= N, where P~ are Jacobi polynomials normalised to unit weighted L2
norm.  Modes are ordered hierarchically: by total degree d = i + j, then by
i.  The sensor of Sec. 2 keeps the modes of degree <= N-1.

Test infrastructure only.
"""
from math import lgamma, exp, sqrt

import numpy as np


def jacobi_classical(x, alpha, beta, n):
    """Classical Jacobi polynomial P_n^(alpha,beta)(x) by its three-term
    recurrence (Abramowitz & Stegun 22.7.1)."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if n == 0:
        return p_prev
    p = 0.5 * ((alpha + beta + 2.0) * x + (alpha - beta))
    for m in range(2, n + 1):
        c = 2.0 * m + alpha + beta
        a1 = 2.0 * m * (m + alpha + beta) * (c - 2.0)
        a2 = (c - 1.0) * (alpha * alpha - beta * beta)
        a3 = (c - 2.0) * (c - 1.0) * c
        a4 = 2.0 * (m + alpha - 1.0) * (m + beta - 1.0) * c
        p_prev, p = p, ((a2 + a3 * x) * p - a4 * p_prev) / a1
    return p


def jacobi_norm2(alpha, beta, n):
    """h_n = int_{-1}^{1} (1-x)^alpha (1+x)^beta P_n^2 dx."""
    logh = ((alpha + beta + 1.0) * np.log(2.0) + lgamma(n + alpha + 1.0)
            + lgamma(n + beta + 1.0) - lgamma(n + alpha + beta + 1.0)
            - lgamma(n + 1.0))
    return exp(logh) / (2.0 * n + alpha + beta + 1.0)


def jacobi(x, alpha, beta, n):
    """Normalised Jacobi polynomial P~_n^(alpha,beta)."""
    return jacobi_classical(x, alpha, beta, n) / sqrt(jacobi_norm2(alpha, beta, n))


def djacobi(x, alpha, beta, n):
    """Derivative of the normalised Jacobi polynomial, from
    d/dx P_n^(a,b) = (n+a+b+1)/2 * P_{n-1}^(a+1,b+1)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    d = 0.5 * (n + alpha + beta + 1.0) * jacobi_classical(x, alpha + 1.0, beta + 1.0, n - 1)
    return d / sqrt(jacobi_norm2(alpha, beta, n))


def n_modes(N):
    """N_p = (N+1)(N+2)/2 (paper Sec. 2, N_p = (p+d)!/(d! p!) with d = 2)."""
    return (N + 1) * (N + 2) // 2


def mode_list(N):
    """Hierarchical mode order: list of (i, j), total degree first, then i."""
    return [(i, d - i) for d in range(N + 1) for i in range(d + 1)]


def mode_degrees(N):
    return np.array([i + j for (i, j) in mode_list(N)], dtype=np.int64)


def collapse(r, s):
    """Collapsed coordinates (a, b); a := -1 at the top vertex s = 1."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    a = np.where(np.abs(1.0 - s) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(1.0 - s) > 1e-14, 1.0 - s, 1.0) - 1.0, -1.0)
    return a, s


def vandermonde(N, r, s):
    """V_ij = psi_j(r_i) (paper Sec. 2)."""
    a, b = collapse(r, s)
    cols = []
    for (i, j) in mode_list(N):
        cols.append(sqrt(2.0) * jacobi(a, 0.0, 0.0, i) * jacobi(b, 2.0 * i + 1.0, 0.0, j) * (1.0 - b) ** i)
    return np.stack(cols, axis=1)


def grad_vandermonde(N, r, s):
    """(V_r)_ij = d psi_j / dr (r_i), (V_s)_ij = d psi_j / ds (r_i).

    Chain rule through the collapsed coordinates:
      d/dr = 2/(1-b) d/da,  d/ds = (1+a)/(1-b) d/da + d/db.
    Points must avoid the top vertex s = 1 (cubature and edge Gauss points do).
    """
    a, b = collapse(r, s)
    if np.any(b > 1.0 - 1e-12):
        raise ValueError("gradient requested at the collapsed vertex s = 1")
    Vr, Vs = [], []
    for (i, j) in mode_list(N):
        fa, dfa = jacobi(a, 0.0, 0.0, i), djacobi(a, 0.0, 0.0, i)
        gb, dgb = jacobi(b, 2.0 * i + 1.0, 0.0, j), djacobi(b, 2.0 * i + 1.0, 0.0, j)
        # d psi/da divided by (1-b):  dfa * gb * (1-b)^(i-1)  (zero for i = 0)
        da_over = dfa * gb * (1.0 - b) ** (i - 1) if i > 0 else np.zeros_like(a)
        dr = 2.0 * da_over
        db = fa * dgb * (1.0 - b) ** i
        if i > 0:
            db = db - i * fa * gb * (1.0 - b) ** (i - 1)
        ds = (1.0 + a) * da_over + db
        Vr.append(sqrt(2.0) * dr)
        Vs.append(sqrt(2.0) * ds)
    return np.stack(Vr, axis=1), np.stack(Vs, axis=1)

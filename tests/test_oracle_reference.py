"""Pins of the oracle's reference-element pieces against closed forms,
library routines and brute force (paper Sec. 2 basis, nodes, rules,
operators)."""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest
from scipy.special import eval_jacobi

from oracle import basis, nodes, quadrature
from oracle.operators import ReferenceElement

ORDERS = [1, 2, 3, 4, 5, 6]


def exact_monomial_integral(a, b):
    """int_T r^a s^b dr ds on T = (-1,-1),(1,-1),(-1,1), exactly:
    r = 2u - 1, s = 2v - 1, dr ds = 4 du dv, int u^m v^n = m! n! / (m+n+2)!."""
    total = Fraction(0)
    for m in range(a + 1):
        for n in range(b + 1):
            c = comb(a, m) * comb(b, n) * 2 ** (m + n) * (-1) ** (a - m + b - n)
            total += c * Fraction(factorial(m) * factorial(n), factorial(m + n + 2))
    return 4 * total


@pytest.mark.parametrize("alpha,beta", [(0, 0), (1, 0), (3, 0), (5, 0), (1, 1)])
def test_jacobi_matches_library(alpha, beta):
    x = np.linspace(-1, 1, 37)
    for n in range(9):
        np.testing.assert_allclose(basis.jacobi_classical(x, alpha, beta, n),
                                   eval_jacobi(n, alpha, beta, x), rtol=1e-12, atol=1e-12)


def test_jacobi_derivative_finite_difference():
    x = np.linspace(-0.9, 0.9, 11)
    h = 1e-6
    for n in range(7):
        fd = (basis.jacobi(x + h, 3.0, 0.0, n) - basis.jacobi(x - h, 3.0, 0.0, n)) / (2 * h)
        np.testing.assert_allclose(basis.djacobi(x, 3.0, 0.0, n), fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("q", [1, 2, 4, 5, 7, 8, 10])
def test_cubature_exact_to_degree_2q_minus_1(q):
    r, s, w = quadrature.triangle_cubature(q)
    assert np.all(w > 0)
    for d in range(2 * q):
        for a in range(d + 1):
            b = d - a
            exact = float(exact_monomial_integral(a, b))
            got = np.sum(w * r ** a * s ** b)
            assert abs(got - exact) < 1e-14 * max(1.0, abs(exact)) * 10, (q, a, b, got, exact)
    # and not beyond: some monomial of degree 2q fails (the rule is sharp)
    errs = [abs(np.sum(w * r ** a * s ** (2 * q - a)) - float(exact_monomial_integral(a, 2 * q - a)))
            for a in range(2 * q + 1)]
    assert max(errs) > 1e-10


@pytest.mark.parametrize("q", [2, 4, 7, 10])
def test_face_rule_exact(q):
    t, w = quadrature.gauss_legendre(q)
    for d in range(2 * q):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * t ** d) - exact) < 1e-14


def test_default_q_rule():
    for N in ORDERS:
        q = quadrature.default_q(N)
        assert 2 * q - 1 >= 3 * N and 2 * (q - 1) - 1 < 3 * N


@pytest.mark.parametrize("N", ORDERS)
def test_basis_orthonormal_and_hierarchical(N):
    ref = ReferenceElement(N)
    G = ref.Vq.T @ (ref.wq[:, None] * ref.Vq)
    assert np.abs(G - np.eye(ref.Np)).max() < 1e-13
    # psi_00 = 1 / sqrt(area) with area 2
    assert np.allclose(ref.Vq[:, 0], 1.0 / np.sqrt(2.0), atol=1e-14)
    deg = basis.mode_degrees(N)
    assert np.all(np.diff(deg) >= 0) and deg[-1] == N
    assert np.sum(deg <= N - 1) == N * (N + 1) // 2


@pytest.mark.parametrize("N", [2, 4, 6])
def test_basis_gradient_finite_difference(N):
    rng = np.random.default_rng(3)
    u = rng.uniform(0.05, 0.9, size=(20, 2))
    u = u[u.sum(axis=1) < 0.95]
    r, s = 2 * u[:, 0] - 1, 2 * u[:, 1] - 1
    Vr, Vs = basis.grad_vandermonde(N, r, s)
    h = 1e-6
    fr = (basis.vandermonde(N, r + h, s) - basis.vandermonde(N, r - h, s)) / (2 * h)
    fs = (basis.vandermonde(N, r, s + h) - basis.vandermonde(N, r, s - h)) / (2 * h)
    assert np.abs(Vr - fr).max() < 1e-6 * max(1, np.abs(fr).max())
    assert np.abs(Vs - fs).max() < 1e-6 * max(1, np.abs(fs).max())


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_edges_are_gll(N):
    r, s = nodes.warp_blend_nodes(N)
    assert len(r) == basis.n_modes(N)
    gll = nodes.gll_points(N)
    for on, coord in ((np.abs(s + 1) < 1e-12, r), (np.abs(r + 1) < 1e-12, s), (np.abs(r + s) < 1e-12, r)):
        assert on.sum() == N + 1
        np.testing.assert_allclose(np.sort(coord[on]), gll, atol=1e-14)
    # inside the triangle
    assert np.all(r >= -1 - 1e-14) and np.all(s >= -1 - 1e-14) and np.all(r + s <= 1e-14)
    # vertices present
    for vr, vs in ((-1, -1), (1, -1), (-1, 1)):
        assert np.min(np.hypot(r - vr, s - vs)) < 1e-14


def test_nodes_n2_equidistant():
    """For N <= 2 GLL and equidistant points coincide, so there is no warp."""
    r, s = nodes.warp_blend_nodes(2)
    er, es = [], []
    for j in range(3):
        for i in range(3 - j):
            er.append(-1 + i)
            es.append(-1 + j)
    np.testing.assert_allclose(r, er, atol=1e-15)
    np.testing.assert_allclose(s, es, atol=1e-15)


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_nodes_symmetric(N):
    """The node set is invariant under the vertex rotation of T (barycentric
    cyclic shift) and the reflection r <-> s."""
    r, s = nodes.warp_blend_nodes(N)
    l1, l2, l3 = -(r + s) / 2, (1 + r) / 2, (1 + s) / 2
    pts = np.stack([r, s], 1)

    def same(a, b):
        d = np.linalg.norm(a[:, None, :] - b[None, :, :], axis=-1)
        return np.all(d.min(axis=1) < 1e-13)
    rot = np.stack([-l2 + l3 - l1, -l2 - l3 + l1], 1)   # (l1,l2,l3) -> (l2,l3,l1)
    assert same(pts, rot)
    assert same(pts, np.stack([s, r], 1))


@pytest.mark.parametrize("N", ORDERS)
def test_operators_exact_on_polynomials(N):
    ref = ReferenceElement(N)
    rng = np.random.default_rng(N)
    terms = [(a, d - a, rng.normal()) for d in range(N + 1) for a in range(d + 1)]

    def f(r, s):
        return sum(c * r ** a * s ** b for a, b, c in terms)

    def fr(r, s):
        return sum(c * a * r ** max(a - 1, 0) * s ** b for a, b, c in terms if a > 0)

    def fs(r, s):
        return sum(c * b * r ** a * s ** max(b - 1, 0) for a, b, c in terms if b > 0)
    u = f(ref.r, ref.s)
    assert np.abs(ref.Icub @ u - f(ref.rq, ref.sq)).max() < 1e-12
    assert np.abs(ref.Dr @ u - fr(ref.rq, ref.sq)).max() < 1e-11
    assert np.abs(ref.Ds @ u - fs(ref.rq, ref.sq)).max() < 1e-11
    for face in range(3):
        fr_, fs_ = ref.face_r[face], ref.face_s[face]
        assert np.abs(ref.Ig[face] @ u - f(fr_, fs_)).max() < 1e-12
        assert np.abs(ref.Drg[face] @ u - fr(fr_, fs_)).max() < 1e-11
        assert np.abs(ref.Dsg[face] @ u - fs(fr_, fs_)).max() < 1e-11


@pytest.mark.parametrize("N", ORDERS)
def test_reference_mass_is_inverse_vvt(N):
    """On T itself (J = 1) eq. (mass) equals (V V^T)^-1 for an orthonormal
    basis."""
    ref = ReferenceElement(N)
    M = ref.Icub.T @ (ref.wq[:, None] * ref.Icub)
    assert np.abs(M - np.linalg.inv(ref.V @ ref.V.T)).max() < 1e-12 * np.abs(M).max() * 10

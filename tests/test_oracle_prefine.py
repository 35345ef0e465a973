"""Pins of the p-refinement prolongation (paper Sec. 5): exact on
polynomials of degree <= N (checked against the polynomial itself, not the
operator), hierarchical (the embedded field has no modes above degree N
and the same low modes), and the identity at equal degree."""
import numpy as np
import pytest

from oracle import basis, nodes, tet
from oracle.prefine import prolongation, prolong_state, prolongation3, prolong_state3


def poly(c, r, s, N):
    return sum(c[a, b] * r ** a * s ** b for a in range(N + 1) for b in range(N + 1 - a))


@pytest.mark.parametrize("N,M", [(2, 3), (2, 4), (3, 4), (4, 5), (5, 6), (2, 6)])
def test_exact_on_degree_n_polynomials(N, M):
    rng = np.random.default_rng(N * 10 + M)
    c = rng.standard_normal((N + 1, N + 1))
    rN, sN = nodes.warp_blend_nodes(N)
    rM, sM = nodes.warp_blend_nodes(M)
    assert np.abs(prolongation(N, M) @ poly(c, rN, sN, N) - poly(c, rM, sM, N)).max() < 1e-12


@pytest.mark.parametrize("N,M", [(2, 3), (3, 5), (4, 5), (4, 6)])
def test_hierarchical_modes(N, M):
    rng = np.random.default_rng(7)
    u = rng.standard_normal(basis.n_modes(N))
    rN, sN = nodes.warp_blend_nodes(N)
    rM, sM = nodes.warp_blend_nodes(M)
    uhat_N = np.linalg.solve(basis.vandermonde(N, rN, sN), u)
    uhat_M = np.linalg.solve(basis.vandermonde(M, rM, sM), prolongation(N, M) @ u)
    deg = basis.mode_degrees(M)
    assert np.abs(uhat_M[deg > N]).max() < 1e-12
    assert np.abs(uhat_M[: basis.n_modes(N)] - uhat_N).max() < 1e-12


def test_identity_and_state_shape():
    for N in (2, 3, 4):
        assert np.abs(prolongation(N, N) - np.eye(basis.n_modes(N))).max() < 1e-12
    U = np.random.default_rng(3).standard_normal((5, 4, 6))
    assert prolong_state(U, 2, 4).shape == (5, 4, 15)
    with pytest.raises(ValueError):
        prolongation(4, 3)


def poly3(c, r, s, t, N):
    return sum(c[a, b, d] * r ** a * s ** b * t ** d
               for a in range(N + 1) for b in range(N + 1 - a) for d in range(N + 1 - a - b))


@pytest.mark.parametrize("N,M", [(2, 3), (2, 4), (3, 4), (1, 3)])
def test_tet_exact_on_degree_n_polynomials(N, M):
    rng = np.random.default_rng(100 + N * 10 + M)
    c = rng.standard_normal((N + 1, N + 1, N + 1))
    rN, sN, tN = tet.warp_blend_nodes_3d(N)
    rM, sM, tM = tet.warp_blend_nodes_3d(M)
    assert np.abs(prolongation3(N, M) @ poly3(c, rN, sN, tN, N) - poly3(c, rM, sM, tM, N)).max() < 1e-11


@pytest.mark.parametrize("N,M", [(2, 3), (2, 4), (3, 4)])
def test_tet_hierarchical_modes(N, M):
    u = np.random.default_rng(8).standard_normal(tet.n_modes(N))
    rN, sN, tN = tet.warp_blend_nodes_3d(N)
    rM, sM, tM = tet.warp_blend_nodes_3d(M)
    uhat_N = np.linalg.solve(tet.vandermonde(N, rN, sN, tN), u)
    uhat_M = np.linalg.solve(tet.vandermonde(M, rM, sM, tM), prolongation3(N, M) @ u)
    deg = tet.mode_degrees(M)
    assert np.abs(uhat_M[deg > N]).max() < 1e-11
    assert np.abs(uhat_M[: tet.n_modes(N)] - uhat_N).max() < 1e-11


def test_tet_identity_and_state_shape():
    for N in (2, 3, 4):
        assert np.abs(prolongation3(N, N) - np.eye(tet.n_modes(N))).max() < 1e-11
    U = np.random.default_rng(4).standard_normal((3, 5, 10))
    assert prolong_state3(U, 2, 4).shape == (3, 5, 35)
    with pytest.raises(ValueError):
        prolongation3(3, 2)

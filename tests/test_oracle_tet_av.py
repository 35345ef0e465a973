"""Pins of the tetrahedral oracle's artificial viscosity (paper Sec. 2 with
d = 3), each against a fact fixed by the mathematics rather than by the
oracle's code:

* the sensor's ratio: for a density a psi_0 + b psi_top on an affine element
  the orthonormal basis gives S = b^2 / (a^2 + b^2) exactly; the three
  regimes of the ramp follow;
* a density of degree <= N - 1 has no top-degree modes: eps = 0;
* BR1 is exact on linear states: with one eps everywhere, q_m = sqrt(eps)
  dU/dx_m on every element whose faces are all interior (affine and curved);
* a constant viscous flux sqrt(eps) q has zero discrete divergence, so the
  viscous terms then leave L(U) unchanged on every element, boundary faces
  included (q+ = q-, eps+ = eps- there);
* eps = 0 gives the inviscid right-hand side exactly.
"""
import numpy as np
import pytest

from oracle import tet
from oracle.dg3 import Oracle3
from paper_1208_4772_gb300.inputs import meshes3d, states
from cases import minimal_tet_mesh


def bump_case(N):
    m = meshes3d.bump_channel(6, 3, 4, seed=2000)
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    return m, X, ref


def linear_state(X, rng):
    """A + B x, constant along y (the channel is periodic in y, so this
    state is continuous across the periodic faces)."""
    A = np.array([1.0, 0.2, -0.1, 0.05, 2.5])
    Bm = 0.1 * rng.standard_normal((5, 3))
    Bm[:, 1] = 0.0
    U = A[None, :, None] + np.einsum('vm,kpm->kvp', Bm, X)
    return U, Bm


@pytest.mark.parametrize("N", [2, 3, 4])
def test_sensor_ratio_from_orthonormal_modes(N):
    m = minimal_tet_mesh("single")
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    o = Oracle3(N, m.EToV, m.bc, X, u_inf=states.freestream3(0.5, 0.0), av=True)
    top = int(np.nonzero(tet.mode_degrees(N) == N)[0][0])
    lo, hi = o.s0 - o.kappa, o.s0 + o.kappa
    for b in (1e-6, 10 ** ((o.s0) / 2.0), 1.0, 10.0):
        a = 1.0
        coef = np.zeros(ref.Np)
        coef[0], coef[top] = a, b
        U = np.zeros((1, 5, ref.Np))
        U[0, 0] = ref.V @ coef
        S = b * b / (a * a + b * b)
        s = np.log10(S)
        eps = o.sensor(U)[0]
        if s < lo:
            assert eps == 0.0
        elif s > hi:
            assert eps == o.eps0
        else:
            assert eps == pytest.approx(0.5 * o.eps0 * (1 + np.sin(np.pi * (s - o.s0) / (2 * o.kappa))), rel=1e-12)


def test_sensor_zero_for_low_degree_density():
    N = 3
    m, X, ref = bump_case(N)
    o = Oracle3(N, m.EToV, m.bc, X, u_inf=states.freestream3(0.5, 0.0), av=True)
    affine = np.nonzero(~meshes3d.mapped_elements(m, ref.r, ref.s, ref.t))[0][:40]
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    U = states.uniform_state3(m.K, ref.Np, states.freestream3(0.5, 0.0))
    U[:, 0] = 1.0 + 0.1 * x + 0.05 * y * z - 0.02 * x * x        # degree 2 = N - 1
    assert np.all(o.sensor(U, affine) == 0.0)


@pytest.mark.parametrize("N", [2, 3])
def test_gradient_exact_on_linear_states(N):
    m, X, ref = bump_case(N)
    o = Oracle3(N, m.EToV, m.bc, X, u_inf=states.freestream3(0.5, 0.0), av=True)
    U, Bm = linear_state(X, np.random.default_rng(N))
    eps = np.full(m.K, 0.04)
    inner = np.nonzero(np.all(m.bc == 0, axis=1))[0]
    curved = meshes3d.mapped_elements(m, ref.r, ref.s, ref.t)
    assert np.any(curved[inner]) and np.any(~curved[inner])
    q = o.gradient_q(U, eps, inner)
    exact = 0.2 * Bm.T[None, :, :, None]                        # sqrt(eps) dU_v/dx_m
    assert np.abs(q - exact).max() < 1e-10 * np.abs(Bm).max()


@pytest.mark.parametrize("N", [2, 3])
def test_constant_viscous_flux_leaves_rhs_unchanged(N):
    m, X, ref = bump_case(N)
    ui = states.freestream3(0.5, 0.0)
    o_av = Oracle3(N, m.EToV, m.bc, X, u_inf=ui, av=True)
    o = Oracle3(N, m.EToV, m.bc, X, u_inf=ui)
    rng = np.random.default_rng(5)
    U = states.uniform_state3(m.K, ref.Np, ui) * (1 + 0.02 * rng.standard_normal((m.K, 5, ref.Np)))
    eps = np.full(m.K, 0.09)
    q = np.broadcast_to(rng.standard_normal((1, 3, 5, 1)), (m.K, 3, 5, ref.Np)).copy()
    L0, vol, _ = o.rhs(U, parts=True)
    L1 = o_av.rhs(U, eps=eps, q=q)
    scale = np.abs(vol @ o.geometry().Minv.transpose(0, 2, 1)).max()
    assert np.abs(L1 - L0).max() < 1e-10 * scale
    # and a non-constant q does change it (the terms are live)
    q2 = q + 0.1 * rng.standard_normal(q.shape)
    assert np.abs(o_av.rhs(U, eps=eps, q=q2) - L0).max() > 1e-4 * scale


def test_zero_eps_is_the_inviscid_rhs():
    N = 2
    m, X, ref = bump_case(N)
    ui = states.freestream3(0.5, 0.0)
    rng = np.random.default_rng(9)
    U = states.uniform_state3(m.K, ref.Np, ui) * (1 + 0.02 * rng.standard_normal((m.K, 5, ref.Np)))
    q = rng.standard_normal((m.K, 3, 5, ref.Np))
    L1 = Oracle3(N, m.EToV, m.bc, X, u_inf=ui, av=True).rhs(U, eps=np.zeros(m.K), q=q)
    L0 = Oracle3(N, m.EToV, m.bc, X, u_inf=ui).rhs(U)
    assert np.array_equal(L1, L0)

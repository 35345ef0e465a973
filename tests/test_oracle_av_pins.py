"""Closed-form pins of the triangle oracle's artificial viscosity (paper
Sec. 2), each against a fact fixed by the mathematics rather than by the
oracle's code:

* the sensor's ratio: for a density a psi_0 + b psi_top on an affine
  element the orthonormal basis gives S = b^2 / (a^2 + b^2) exactly, across
  the three regimes of the ramp; a density of degree <= N - 1 gives eps = 0;
* BR1 is exact on linear states: with one eps everywhere, q_m = sqrt(eps)
  dU/dx_m on every element whose faces are all interior;
* a constant viscous flux sqrt(eps) q has zero discrete divergence, so the
  viscous terms leave L(U) unchanged on every element -- curved wall
  elements and boundary faces included (q+ = q-, eps+ = eps- there) --
  while a varying q changes it;
* eps = 0 gives the inviscid right-hand side exactly.
"""
import numpy as np
import pytest

from oracle import basis, nodes
from oracle.dg import Oracle
from paper_1208_4772_gb300.inputs import curving, meshes, states


def cyl_case(N):
    m = meshes.cylinder_channel(n_t=32, n_r=5, seed=1002)
    r, s = nodes.warp_blend_nodes(N)
    xy, curved = curving.curve_mesh(m, N, r, s)
    return m, xy, curved, r, s


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_sensor_ratio_from_orthonormal_modes(N):
    m, xy, curved, r, s = cyl_case(N)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=states.freestream(0.38, 0.0), av=True)
    V = basis.vandermonde(N, r, s)
    top = int(np.nonzero(basis.mode_degrees(N) == N)[0][0])
    k = np.nonzero(~curved)[0][:1]
    lo, hi = o.s0 - o.kappa, o.s0 + o.kappa
    for b in (1e-6, 10 ** (o.s0 / 2.0), 1.0, 10.0):
        coef = np.zeros(len(r))
        coef[0], coef[top] = 1.0, b
        U = states.uniform_state(m.K, len(r), states.freestream(0.38, 0.0))
        U[k, 0] = V @ coef
        S = b * b / (1.0 + b * b)
        sk = np.log10(S)
        eps = o.sensor(U, k)[0]
        if sk < lo:
            assert eps == 0.0
        elif sk > hi:
            assert eps == o.eps0
        else:
            assert eps == pytest.approx(0.5 * o.eps0 * (1 + np.sin(np.pi * (sk - o.s0) / (2 * o.kappa))), rel=1e-12)


def test_sensor_zero_for_low_degree_density():
    N = 4
    m, xy, curved, r, s = cyl_case(N)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=states.freestream(0.38, 0.0), av=True)
    x, y = xy[..., 0], xy[..., 1]
    U = states.uniform_state(m.K, len(r), states.freestream(0.38, 0.0))
    U[:, 0] = 1.0 + 0.01 * x + 0.02 * x * y - 0.003 * y ** 3        # degree 3 = N - 1
    affine = np.nonzero(~curved)[0]
    assert np.all(o.sensor(U, affine) == 0.0)


@pytest.mark.parametrize("N", [2, 4])
def test_gradient_exact_on_linear_states(N):
    m, xy, curved, r, s = cyl_case(N)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=states.freestream(0.38, 0.0), av=True)
    Bm = 0.1 * np.random.default_rng(N).standard_normal((4, 2))
    A = np.array([1.0, 0.1, -0.05, 2.5])
    U = A[None, :, None] + np.einsum('vm,kpm->kvp', Bm, xy)
    eps = np.full(m.K, 0.04)
    inner = np.nonzero(np.all(m.bc == 0, axis=1))[0]
    q = o.gradient_q(U, eps, inner)                              # [n, 2, 4, Np]
    exact = 0.2 * Bm.T[None, :, :, None]
    assert np.abs(q - exact).max() < 1e-10 * np.abs(Bm).max()


@pytest.mark.parametrize("N", [2, 4])
def test_constant_viscous_flux_leaves_rhs_unchanged(N):
    m, xy, curved, r, s = cyl_case(N)
    ui = states.freestream(0.38, 0.0)
    o_av = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=ui, av=True)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=ui)
    rng = np.random.default_rng(3)
    U = states.uniform_state(m.K, len(r), ui) * (1 + 0.02 * rng.standard_normal((m.K, 4, len(r))))
    eps = np.full(m.K, 0.09)
    q = np.broadcast_to(rng.standard_normal((1, 2, 4, 1)), (m.K, 2, 4, len(r))).copy()
    L0, vol, _ = o.rhs(U, parts=True)
    L1 = o_av.rhs(U, eps=eps, q=q)
    scale = np.abs(vol @ o.geometry(None).Minv.transpose(0, 2, 1)).max()
    assert np.any(curved)
    assert np.abs(L1 - L0).max() < 1e-10 * scale
    q2 = q + 0.1 * rng.standard_normal(q.shape)
    assert np.abs(o_av.rhs(U, eps=eps, q=q2) - L0).max() > 1e-4 * scale


def test_zero_eps_is_the_inviscid_rhs():
    N = 3
    m, xy, curved, r, s = cyl_case(N)
    ui = states.freestream(0.38, 0.0)
    rng = np.random.default_rng(4)
    U = states.uniform_state(m.K, len(r), ui) * (1 + 0.02 * rng.standard_normal((m.K, 4, len(r))))
    q = rng.standard_normal((m.K, 2, 4, len(r)))
    L1 = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=ui, av=True).rhs(U, eps=np.zeros(m.K), q=q)
    L0 = Oracle(N, m.EToE, m.EToF, m.bc, xy, u_inf=ui).rhs(U)
    assert np.array_equal(L1, L0)

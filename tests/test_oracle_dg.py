"""Pins of the oracle's right-hand side, mass, sensor, SSP-RK3 and residual
against what the paper and the mathematics fix: free-stream preservation on
curved meshes, discrete conservation on periodic meshes, isentropic-vortex
convergence order, flux symmetries, closed forms and invariances.  The last
tests plant mistakes in the oracle and check that a pin catches each."""
import numpy as np
import pytest

from oracle import euler
from oracle.dg import Oracle
from oracle.operators import ReferenceElement
from paper_1208_4772_gb300.inputs import curving, meshes, states

GAMMA = 1.4


def periodic_case(N, n=6, length=10.0, av=False, seed=11, **kw):
    ref = ReferenceElement(N)
    m = meshes.periodic_square(n, length=length, seed=seed)
    xy = meshes.straight_nodes(m.verts, ref.r, ref.s)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=av, **kw)
    return m, xy, o


def curved_case(N, kind="naca", bc_all_farfield=False, av=False, mach=0.8, aoa=1.25):
    ref = ReferenceElement(N)
    m = meshes.naca_omesh(n_t=32, n_r=5) if kind == "naca" else meshes.cylinder_channel(n_t=28, n_r=5)
    xy, curved = curving.curve_mesh(m, N, ref.r, ref.s)
    bc = np.where(m.bc != 0, 2, 0) if bc_all_farfield else m.bc
    ui = states.freestream(mach, aoa)
    o = Oracle(N, m.EToE, m.EToF, bc, xy, u_inf=ui, av=av)
    return m, xy, curved, o, ui


# ------------------------------------------------------------------ flux
def test_euler_flux_hand_values():
    # rho = 2, u = 3, v = -1, p = 5 -> E = 5/0.4 + 0.5*2*10 = 22.5
    U = np.array([2.0, 6.0, -2.0, 22.5])[:, None]
    F, G = euler.flux(U, GAMMA)
    np.testing.assert_allclose(euler.pressure(U, GAMMA), [5.0])
    np.testing.assert_allclose(F[:, 0], [6.0, 23.0, -6.0, 82.5])
    np.testing.assert_allclose(G[:, 0], [-2.0, -6.0, 7.0, -27.5])


def test_llf_consistency_and_conservation():
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.5, 2, 7)
    U1 = states.conserved(rho, rng.normal(size=7), rng.normal(size=7), rng.uniform(0.5, 2, 7))
    U2 = states.conserved(rng.uniform(0.5, 2, 7), rng.normal(size=7), rng.normal(size=7), rng.uniform(0.5, 2, 7))
    th = rng.uniform(0, 2 * np.pi, 7)
    nx, ny = np.cos(th), np.sin(th)
    F, G = euler.flux(U1, GAMMA)
    assert np.abs(euler.llf(U1, U1, nx, ny, GAMMA) - (F * nx + G * ny)).max() < 1e-14
    a = euler.llf(U1, U2, nx, ny, GAMMA)
    b = euler.llf(U2, U1, -nx, -ny, GAMMA)
    assert np.abs(a + b).max() < 1e-14


def _hllc_states(seed, n=9):
    rng = np.random.default_rng(seed)
    mk = lambda: states.conserved(rng.uniform(0.5, 2, n), rng.normal(size=n), rng.normal(size=n),
                                  rng.uniform(0.5, 2, n))
    th = rng.uniform(0, 2 * np.pi, n)
    return mk(), mk(), np.cos(th), np.sin(th)


def test_hllc_consistency_and_antisymmetry():
    U1, U2, nx, ny = _hllc_states(3)
    F, G = euler.flux(U1, GAMMA)
    assert np.abs(euler.hllc(U1, U1, nx, ny, GAMMA) - (F * nx + G * ny)).max() < 1e-13
    a = euler.hllc(U1, U2, nx, ny, GAMMA)
    b = euler.hllc(U2, U1, -nx, -ny, GAMMA)
    assert np.abs(a + b).max() < 1e-13


def test_hllc_resolves_stationary_contact_and_shear():
    """Two states with the same pressure and zero normal velocity but
    different densities and tangential velocities: HLLC carries no mass,
    tangential momentum or energy across (flux (0, p n, 0)); LLF does."""
    n = 5
    rng = np.random.default_rng(4)
    th = rng.uniform(0, 2 * np.pi, n)
    nx, ny = np.cos(th), np.sin(th)
    tx, ty = -ny, nx
    p = rng.uniform(0.5, 2, n)
    wl, wr = rng.normal(size=n), rng.normal(size=n)
    UL = states.conserved(rng.uniform(0.5, 2, n), wl * tx, wl * ty, p)
    UR = states.conserved(rng.uniform(0.5, 2, n), wr * tx, wr * ty, p)
    fh = euler.hllc(UL, UR, nx, ny, GAMMA)
    exact = np.stack([np.zeros(n), p * nx, p * ny, np.zeros(n)])
    assert np.abs(fh - exact).max() < 1e-13
    assert np.abs(euler.llf(UL, UR, nx, ny, GAMMA)[0]).max() > 1e-3


def test_hllc_supersonic_upwinding():
    """u.n > c on both sides: the flux is F(U-).n; u.n < -c: F(U+).n."""
    n = 6
    rng = np.random.default_rng(5)
    th = rng.uniform(0, 2 * np.pi, n)
    nx, ny = np.cos(th), np.sin(th)
    for sgn, pick in ((1.0, 0), (-1.0, 1)):
        U = [states.conserved(rng.uniform(0.5, 2, n), sgn * 3.0 * nx, sgn * 3.0 * ny, rng.uniform(0.2, 0.5, n))
             for _ in range(2)]
        F, G = euler.flux(U[pick], GAMMA)
        assert np.abs(euler.hllc(U[0], U[1], nx, ny, GAMMA) - (F * nx + G * ny)).max() < 1e-13


def test_hllc_wall_and_operator_pins():
    """No mass or energy through a slip wall; with HLLC in the operator,
    free stream on a curved mesh and conservation on a periodic one."""
    U, _, nx, ny = _hllc_states(6)
    fn = euler.hllc(U, euler.wall_ghost(U, nx, ny), nx, ny, GAMMA)
    assert np.abs(fn[0]).max() < 1e-13 and np.abs(fn[3]).max() < 1e-13
    N = 4
    ref = ReferenceElement(N)
    m = meshes.naca_omesh(n_t=32, n_r=5)
    xy, curved = curving.curve_mesh(m, N, ref.r, ref.s)
    ui = states.freestream(0.8, 1.25)
    o = Oracle(N, m.EToE, m.EToF, np.where(m.bc != 0, 2, 0), xy, u_inf=ui, flux="hllc")
    assert _relative(o, states.uniform_state(m.K, o.ref.Np, ui)) < 1e-12
    m, xy, o = periodic_case(3, flux="hllc")
    Uv = states.vortex_state(xy, period=(10.0, 10.0))
    L, vol, surf = o.rhs(Uv, parts=True)
    total = np.einsum('kij,kvj->v', o.geometry(None).M, L)
    assert np.all(np.abs(total) < 1e-12 * np.sum(np.abs(surf), axis=(0, 2)))


def test_wall_ghost_no_mass_flux():
    rng = np.random.default_rng(1)
    U = states.conserved(rng.uniform(0.5, 2, 9), rng.normal(size=9), rng.normal(size=9), rng.uniform(0.5, 2, 9))
    th = rng.uniform(0, 2 * np.pi, 9)
    nx, ny = np.cos(th), np.sin(th)
    fn = euler.llf(U, euler.wall_ghost(U, nx, ny), nx, ny, GAMMA)
    assert np.abs(fn[0]).max() < 1e-14          # no mass through the wall
    assert np.abs(fn[3]).max() < 1e-14          # no energy through the wall


# ------------------------------------------------------------------ geometry / mass
def test_affine_geometry_and_mass():
    N = 4
    m, xy, o = periodic_case(N)
    g = o.geometry(None)
    v = m.verts
    xr, xs = 0.5 * (v[:, 1] - v[:, 0]), 0.5 * (v[:, 2] - v[:, 0])
    J = xr[:, 0] * xs[:, 1] - xs[:, 0] * xr[:, 1]
    assert np.abs(g.J - J[:, None]).max() < 1e-13
    assert np.abs(g.rx - (xs[:, 1] / J)[:, None]).max() < 1e-12
    # face 0 length / 2 = sJ, normal orthogonal to the edge
    e0 = v[:, 1] - v[:, 0]
    assert np.abs(g.sJ[:, 0] - 0.5 * np.linalg.norm(e0, axis=1)[:, None]).max() < 1e-13
    assert np.abs(g.nx[:, 0] * e0[:, 0:1] + g.ny[:, 0] * e0[:, 1:2]).max() < 1e-13
    # M_k = J_k M_ref, M_ref = (V V^T)^-1
    Mref = np.linalg.inv(o.ref.V @ o.ref.V.T)
    assert np.abs(g.M - J[:, None, None] * Mref).max() < 1e-12 * np.abs(g.M).max()
    # total area of the periodic box
    assert abs(np.sum(g.J * o.ref.wq) - 100.0) < 1e-11


# ------------------------------------------------------------------ free stream
def _relative(o, U):
    L, vol, surf = o.rhs(U, parts=True)
    scale = np.abs(vol).max()
    return np.abs(vol - surf).max() / scale


@pytest.mark.parametrize("N", [2, 4, 6])
def test_free_stream_periodic(N):
    m, xy, o = periodic_case(N)
    U = states.uniform_state(m.K, o.ref.Np, states.freestream(0.5, 30.0))
    assert _relative(o, U) < 1e-12


@pytest.mark.parametrize("N,kind,av", [(2, "naca", False), (4, "naca", False), (4, "naca", True),
                                       (5, "cyl", False), (6, "cyl", True)])
def test_free_stream_curved(N, kind, av):
    """L(U_inf) = 0 on curved meshes: J r_x etc. are polynomial minors of the
    isoparametric map and the face n sJ is exact, so every integrand is
    within the rules' degree."""
    m, xy, curved, o, ui = curved_case(N, kind, bc_all_farfield=True, av=av)
    assert curved.sum() > 0
    U = states.uniform_state(m.K, o.ref.Np, ui)
    assert _relative(o, U) < 1e-12


# ------------------------------------------------------------------ conservation
@pytest.mark.parametrize("N,av", [(2, False), (3, False), (4, True), (6, False)])
def test_conservation_periodic(N, av):
    """sum_k 1^T M_k L_k = 0: volume terms sum to zero (sum_i grad l_i = 0)
    and face fluxes cancel pairwise."""
    m, xy, o = periodic_case(N, av=av)
    U = states.vortex_state(xy, period=(10.0, 10.0))
    L, vol, surf = o.rhs(U, parts=True)
    g = o.geometry(None)
    total = np.einsum('kij,kvj->v', g.M, L)
    scale = np.sum(np.abs(surf), axis=(0, 2))
    assert np.all(np.abs(total) < 1e-12 * scale)


# ------------------------------------------------------------------ consistency and convergence
def vortex_dudt(xy, length):
    """Central difference in time of the closed form, with the periodic image
    fixed at t = 0 so that no node changes image between t - d and t + d."""
    d = 1e-5
    c = np.array([length / 2, length / 2])
    xs = xy - length * np.round((xy - c) / length)
    return (states.vortex_state(xs, t=d, center=c) - states.vortex_state(xs, t=-d, center=c)) / (2 * d)


def rhs_consistency_error(N, n, oracle_cls=Oracle, length=15.0):
    """Max |L(I U) - dU/dt| for the vortex on a box wide enough (15) that
    its tail at the periodic seam is below 1e-11."""
    ref = ReferenceElement(N)
    m = meshes.periodic_square(n, length=length, seed=5)
    xy = meshes.straight_nodes(m.verts, ref.r, ref.s)
    o = oracle_cls(N, m.EToE, m.EToF, m.bc, xy)
    c = (length / 2, length / 2)
    U = states.vortex_state(xy, period=(length, length), center=c)
    return np.abs(o.rhs(U) - vortex_dudt(xy, length)).max()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_rhs_consistency(N):
    """L(I U) approaches dU/dt of the exact vortex as h -> 0; the pointwise
    truncation error of the DG operator falls at about order N (here > N-1)."""
    e1, e2 = rhs_consistency_error(N, 18), rhs_consistency_error(N, 36)
    assert np.log2(e1 / e2) > N - 1


def vortex_error(N, n, T=0.2, length=10.0):
    ref = ReferenceElement(N)
    m = meshes.periodic_square(n, length=length, seed=7)
    xy = meshes.straight_nodes(m.verts, ref.r, ref.s)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy)
    U = states.vortex_state(xy, period=(length, length))
    dt0 = states.time_step(m.verts, U, N, cfl=0.3)
    nst = int(np.ceil(T / dt0))
    for _ in range(nst):
        U = o.ssp_rk3_step(U, T / nst)
    Ue = states.vortex_state(xy, t=T, period=(length, length))
    e = (U - Ue)[:, 0, :] @ ref.Icub.T
    return np.sqrt(np.sum(o.geometry(None).J * ref.wq * e * e))


@pytest.mark.parametrize("N,n1", [(2, 16), (3, 8), (4, 8)])
def test_vortex_convergence_order(N, n1):
    """Density L2 error at T = 0.2 on n and 2n periodic meshes converges at
    order >= N + 1/2."""
    e1, e2 = vortex_error(N, n1), vortex_error(N, 2 * n1)
    assert np.log2(e1 / e2) >= N + 0.5


# ------------------------------------------------------------------ RK3
def test_ssp_rk3_stability_polynomial():
    class Linear(Oracle):
        lam = -0.7 + 0.4j

        def rhs(self, U, idx=None, eps=None, q=None, parts=False):
            return self.lam * U
    m, xy, _ = periodic_case(2, n=3)
    o = Linear(2, m.EToE, m.EToF, m.bc, xy)
    U = np.ones((m.K, 4, 6), dtype=complex)
    dt = 0.9
    z = Linear.lam * dt
    assert np.abs(o.ssp_rk3_step(U, dt) - (1 + z + z * z / 2 + z ** 3 / 6)).max() < 1e-15


def test_lserk54_is_fourth_order_on_linear_problems():
    """One LSERK(5,4) step on u' = lam u multiplies u by a degree-5
    polynomial R(z), z = lam dt; a fourth-order method has R(z) = 1 + z +
    z^2/2 + z^3/6 + z^4/24 + c5 z^5.  R is recovered exactly from six values
    of z and its coefficients compared with those of exp."""
    m, xy, _ = periodic_case(2, n=3)
    zs = np.array([0.3, -0.5, 0.8 + 0.2j, -1.1 - 0.4j, 0.6j, -0.2 + 0.9j])   # well inside the stability region
    vals = []
    for z in zs:
        class Linear(Oracle):
            def rhs(self, U, idx=None, eps=None, q=None, parts=False):
                return z * U
        o = Linear(2, m.EToE, m.EToF, m.bc, xy)
        vals.append(o.lserk54_step(np.ones((m.K, 4, 6), dtype=complex), 1.0)[0, 0, 0])
    c = np.linalg.solve(np.vander(zs, 6, increasing=True), np.array(vals))
    assert np.abs(c[:5] - np.array([1, 1, 1 / 2, 1 / 6, 1 / 24])).max() < 1e-12
    assert abs(c[5] - 1 / 120) > 1e-4          # fourth, not fifth order


def test_lserk54_temporal_order_on_the_vortex():
    """Nonlinear check: the time error of LSERK(5,4) on a vortex mesh
    (fixed spatial discretisation) falls by ~16 when dt halves."""
    N = 2
    m, xy, o = periodic_case(N, n=4)
    U0 = states.vortex_state(xy, period=(10.0, 10.0))
    T = 0.4

    def run(nst):
        U = U0.copy()
        for _ in range(nst):
            U = o.lserk54_step(U, T / nst)
        return U
    ref = run(64)
    e1 = np.abs(run(4) - ref).max()
    e2 = np.abs(run(8) - ref).max()
    assert np.log2(e1 / e2) >= 3.5, np.log2(e1 / e2)


# ------------------------------------------------------------------ sensor
def test_sensor_closed_forms():
    N = 4
    m, xy, o = periodic_case(N, av=True, kappa=4.0, eps0=0.3)
    ref = o.ref
    K = m.K
    U = states.uniform_state(K, ref.Np, states.freestream(0.3, 0.0))
    # degree <= N-1 density: S = 0 -> eps = 0
    x, y = xy[..., 0], xy[..., 1]
    U[:, 0, :] = 1.0 + 0.01 * x ** 3 + 0.02 * x * y ** 2
    assert np.all(o.sensor(U) == 0.0)
    # pure top-degree mode on an affine element: S = 1 -> s = 0
    top = np.nonzero(ref.degrees == N)[0][1]
    U[:, 0, :] = ref.V[:, top][None, :]
    o2 = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=True, kappa=4.0, eps0=0.3, s0=-0.5)
    eps = o2.sensor(U)
    want = 0.5 * 0.3 * (1 + np.sin(np.pi * (0.0 + 0.5) / 8.0))
    assert np.abs(eps - want).max() < 1e-12
    # ramp values at s0 and the ends
    for s0, want in ((0.0, 0.15), (-4.0, 0.3), (4.0, 0.0)):
        o3 = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=True, kappa=4.0, eps0=0.3, s0=s0)
        assert np.abs(o3.sensor(U) - want).max() < 1e-12
    # affine element: the cubature form equals sum_top u^2 / sum u^2
    rng = np.random.default_rng(2)
    U[:, 0, :] = 1.0 + 0.1 * rng.normal(size=(K, ref.Np))
    modal = U[:, 0, :] @ ref.Vinv.T
    S = np.sum(modal[:, ref.degrees == N] ** 2, 1) / np.sum(modal ** 2, 1)
    s = np.log10(S)
    o4 = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=True, kappa=4.0, eps0=0.3, s0=-2.0)
    want = np.where(s < -6, 0, np.where(s > 2, 0.3, 0.15 * (1 + np.sin(np.pi * (s + 2) / 8))))
    assert np.abs(o4.sensor(U) - want).max() < 1e-12


# ------------------------------------------------------------------ invariances
def test_renumbering_invariance():
    N = 3
    ref = ReferenceElement(N)
    m = meshes.periodic_square(6, seed=4)
    rng = np.random.default_rng(9)
    perm = rng.permutation(m.K)
    _, m2 = meshes.renumber(m, perm)
    xy = meshes.straight_nodes(m.verts, ref.r, ref.s)
    xy2 = meshes.straight_nodes(m2.verts, ref.r, ref.s)
    U = states.vortex_state(xy, period=(10, 10))
    for av in (False, True):
        L1 = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=av).rhs(U)
        L2 = Oracle(N, m2.EToE, m2.EToF, m2.bc, xy2, av=av).rhs(U[perm])
        assert np.abs(L1[perm] - L2).max() < 1e-12 * np.abs(L1).max()


def test_rotation_invariance():
    """Rotating the mesh and the flow by 90 degrees rotates L."""
    N = 3
    m, xy, curved, o, ui = curved_case(N, "cyl", mach=0.38, aoa=20.0)
    ref = o.ref
    rng = np.random.default_rng(5)
    U = states.uniform_state(m.K, ref.Np, ui) * (1 + 0.01 * rng.normal(size=(m.K, 1, ref.Np)))
    L = o.rhs(U)
    R = np.array([[0.0, -1.0], [1.0, 0.0]])
    xy_r = xy @ R.T
    Ur = U.copy()
    Ur[:, 1], Ur[:, 2] = -U[:, 2], U[:, 1]
    ui_r = ui.copy()
    ui_r[1], ui_r[2] = -ui[2], ui[1]
    o_r = Oracle(N, m.EToE, m.EToF, m.bc, xy_r, u_inf=ui_r)
    Lr = o_r.rhs(Ur)
    want = L.copy()
    want[:, 1], want[:, 2] = -L[:, 2], L[:, 1]
    assert np.abs(Lr - want).max() < 1e-10 * np.abs(L).max()


def test_residual_and_subset():
    N = 2
    m, xy, o = periodic_case(N, av=True)
    U = states.vortex_state(xy, period=(10, 10))
    L = o.rhs(U)
    linf, l2 = o.residual(U)
    assert np.allclose(linf, np.abs(L).max(axis=(0, 2)))
    assert np.allclose(l2, np.sqrt((L * L).sum(axis=(0, 2))))
    idx = np.array([0, 5, 17, 40])
    assert np.abs(o.rhs(U, idx) - L[idx]).max() < 1e-12 * np.abs(L).max()


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible mistake below breaks at least one pin above."""
    N = 3
    # (1) neighbour trace not reversed along the shared edge: consistency
    base = rhs_consistency_error(N, 18)

    class NoReverse(Oracle):
        def _exterior(self, V, idx, own, fill):
            out = super()._exterior(V, idx, own, fill)
            return out[..., ::-1]
    assert rhs_consistency_error(N, 18, NoReverse) > 10 * base
    # (2) sign of the lift flipped: free stream
    m, xy, o = periodic_case(N)
    U = states.uniform_state(m.K, o.ref.Np, states.freestream(0.5, 30.0))

    class LiftSign(Oracle):
        def lift(self, Fs):
            return -super().lift(Fs)
    o2 = LiftSign(N, m.EToE, m.EToF, m.bc, xy)
    assert _relative(o2, U) > 1e-3
    # (3) D_r and D_s swapped: free stream
    o3 = Oracle(N, m.EToE, m.EToF, m.bc, xy)
    o3.geometry(None)            # geometry first, then swap in the volume term only
    o3.ref.Dr, o3.ref.Ds = o3.ref.Ds.copy(), o3.ref.Dr.copy()
    assert _relative(o3, U) > 1e-3
    # (4) pressure with the printed rho E - |u|^2/(2 rho): flux hand values
    Ut = np.array([2.0, 6.0, -2.0, 22.5])[:, None]
    rho, mx, my, E = Ut
    wrong = (GAMMA - 1) * (E - ((mx / rho) ** 2 + (my / rho) ** 2) / (2 * rho))
    assert abs(wrong[0] - euler.pressure(Ut, GAMMA)[0]) > 0.1

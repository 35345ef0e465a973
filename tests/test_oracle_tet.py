"""Pins of the tetrahedral oracle (oracle/tet.py, oracle/euler3.py,
oracle/dg3.py) against facts fixed by the mathematics: exact integrals of
monomials, orthonormality, finite differences, the triangle node set and
GLL points, symmetry, the divergence theorem, free-stream preservation,
discrete conservation, the consistency order on an exact Euler solution,
rotation invariance, and planted mistakes."""
from fractions import Fraction
from itertools import permutations
from math import comb, factorial

import numpy as np
import pytest

from oracle import euler3, tet
from oracle import nodes as nodes2
from oracle.dg3 import Oracle3, TetGeometry, connectivity
from paper_1208_4772_gb300.inputs import meshes3d, states

L_BOX = 10.0


def exact_monomial(a, b, c):
    """int_T3 r^a s^b t^c with r = 2x - 1 etc. on the unit simplex, where
    int x^i y^j z^k = i! j! k! / (i + j + k + 3)!  (Dirichlet)."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            for k in range(c + 1):
                coef = comb(a, i) * comb(b, j) * comb(c, k) * 2 ** (i + j + k) * (-1) ** (a - i + b - j + c - k)
                tot += coef * Fraction(factorial(i) * factorial(j) * factorial(k), factorial(i + j + k + 3))
    return 8 * tot


@pytest.mark.parametrize("q", [2, 3, 4, 5, 7])
def test_tet_cubature_exactness(q):
    r, s, t, w = tet.tet_cubature(q)
    worst = 0.0
    for d in range(2 * q):
        for a in range(d + 1):
            for b in range(d - a + 1):
                c = d - a - b
                worst = max(worst, abs(np.sum(w * r ** a * s ** b * t ** c) - float(exact_monomial(a, b, c))))
    assert worst < 1e-13
    # not exact one degree higher (the degree claim is sharp)
    d = 2 * q
    errs = [abs(np.sum(w * r ** a * s ** b * t ** (d - a - b)) - float(exact_monomial(a, b, d - a - b)))
            for a in range(d + 1) for b in range(d - a + 1)]
    assert max(errs) > 1e-8


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_basis_orthonormal_and_hierarchical(N):
    r, s, t, w = tet.tet_cubature(N + 1)
    V = tet.vandermonde(N, r, s, t)
    assert np.allclose(V.T @ (w[:, None] * V), np.eye(tet.n_modes(N)), atol=1e-12)
    # the modes of degree <= N-1 span exactly the polynomials of degree <= N-1:
    # each is a combination of monomials of that degree (least squares exact)
    deg = tet.mode_degrees(N)
    mons = np.stack([r ** a * s ** b * t ** c for d in range(N) for a in range(d + 1) for b in range(d - a + 1)
                     for c in [d - a - b]], axis=1)
    for j in np.nonzero(deg <= N - 1)[0]:
        coef, *_ = np.linalg.lstsq(mons, V[:, j], rcond=None)
        assert np.abs(mons @ coef - V[:, j]).max() < 1e-11


@pytest.mark.parametrize("N", [1, 3, 4])
def test_basis_gradient_finite_differences(N):
    rng = np.random.default_rng(N)
    lam = rng.dirichlet(np.ones(4), size=20) * 0.9 + 0.025
    P = lam @ tet.VERTS
    r, s, t = P.T
    Vr, Vs, Vt = tet.grad_vandermonde(N, r, s, t)
    h = 1e-6
    for G, e in ((Vr, (h, 0, 0)), (Vs, (0, h, 0)), (Vt, (0, 0, h))):
        fd = (tet.vandermonde(N, r + e[0], s + e[1], t + e[2]) - tet.vandermonde(N, r - e[0], s - e[1], t - e[2])) / (2 * h)
        assert np.abs(fd - G).max() < 1e-6 * max(1.0, np.abs(G).max())


def _bary(r, s, t):
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_nodes(N):
    r, s, t = tet.warp_blend_nodes_3d(N)
    Np = tet.n_modes(N)
    assert len(r) == Np
    lam = _bary(r, s, t)
    # inside the element
    assert lam.min() > -1e-12
    # N = 1, 2: the equidistant lattice (GLL = equidistant up to N = 2)
    if N <= 2:
        assert np.allclose(lam, tet.lattice_3d(N), atol=1e-14)
    # every edge carries the GLL points
    gll = nodes2.gll_points(N)
    for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        others = [v for v in range(4) if v not in (a, b)]
        on = np.all(lam[:, others] < 1e-12, axis=1)
        pts = np.sort(lam[on, b] - lam[on, a])
        assert np.allclose(pts, gll, atol=1e-12)
    # every face carries the triangle's warp & blend nodes
    r2, s2 = nodes2.warp_blend_nodes(N)
    lam2 = np.stack([-(r2 + s2) / 2, (1 + r2) / 2, (1 + s2) / 2], axis=1)
    for fv in tet.FACE_VERTS:
        opp = [v for v in range(4) if v not in fv][0]
        on = lam[:, opp] < 1e-12
        F = lam[on][:, list(fv)]
        assert len(F) == len(lam2)
        for x in lam2:
            assert np.min(np.abs(F - x).sum(axis=1)) < 1e-11
    # the set is invariant under the 24 vertex permutations
    for p in permutations(range(4)):
        Q = lam[:, list(p)]
        for x in Q:
            assert np.min(np.abs(lam - x).sum(axis=1)) < 1e-11
    # unisolvent
    assert np.linalg.cond(tet.vandermonde(N, r, s, t)) < 1e3


@pytest.mark.parametrize("N", [2, 3, 4])
def test_operators_exact_on_polynomials(N):
    ref = tet.ReferenceTet(N)
    rng = np.random.default_rng(10 + N)
    terms = [(a, b, d - a - b) for d in range(N + 1) for a in range(d + 1) for b in range(d - a + 1)]
    coef = rng.standard_normal(len(terms))

    def f(r, s, t):
        return sum(c * r ** a * s ** b * t ** e for c, (a, b, e) in zip(coef, terms))

    def grad(r, s, t):
        gr = sum(c * a * r ** max(a - 1, 0) * s ** b * t ** e for c, (a, b, e) in zip(coef, terms))
        gs = sum(c * b * r ** a * s ** max(b - 1, 0) * t ** e for c, (a, b, e) in zip(coef, terms))
        gt = sum(c * e * r ** a * s ** b * t ** max(e - 1, 0) for c, (a, b, e) in zip(coef, terms))
        return gr, gs, gt

    u = f(ref.r, ref.s, ref.t)
    assert np.allclose(ref.Icub @ u, f(ref.rq, ref.sq, ref.tq), atol=1e-11)
    gr, gs, gt = grad(ref.rq, ref.sq, ref.tq)
    assert np.allclose(ref.Dr @ u, gr, atol=1e-10)
    assert np.allclose(ref.Ds @ u, gs, atol=1e-10)
    assert np.allclose(ref.Dt @ u, gt, atol=1e-10)
    for fc in range(4):
        for o in range(6):
            P = ref.face_xyz[fc, o]
            assert np.allclose(ref.Ig[fc, o] @ u, f(*P.T), atol=1e-11)
            gr, gs, gt = grad(*P.T)
            assert np.allclose(ref.Drg[fc, o] @ u, gr, atol=1e-10)
            assert np.allclose(ref.Dtg[fc, o] @ u, gt, atol=1e-10)


def test_face_points_lie_on_their_face():
    ref = tet.ReferenceTet(3)
    planes = [lambda P: P[:, 2] + 1, lambda P: P[:, 1] + 1, lambda P: P.sum(axis=1) + 1, lambda P: P[:, 0] + 1]
    for fc in range(4):
        for o in range(6):
            assert np.abs(planes[fc](ref.face_xyz[fc, o])).max() < 1e-14
    # the weights integrate the face area (reference triangle of area 2)
    assert abs(ref.wg.sum() - 2.0) < 1e-14


def warped_box(n, N, amp=0.3, seed=1000):
    m = meshes3d.box(n, L=L_BOX, seed=seed)
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    k = 2 * np.pi / L_BOX
    d = amp * np.sin(k * X[..., [0]] + 0.3) * np.sin(k * X[..., [1]]) * np.sin(k * X[..., [2]])
    return m, ref, X + d * np.array([1.0, 0.5, -0.7])


@pytest.mark.parametrize("N", [2, 3])
def test_geometry_divergence_theorem(N):
    """Volume = 1/3 of the flux of x through the surface and the closed
    surface integral of n vanishes, on curved elements; the matched face
    points of two neighbours coincide physically."""
    m, ref, X = warped_box(3, N)
    EToE, EToF, orient = connectivity(m.EToV)
    geo = TetGeometry(ref, X, orient)
    vol = np.sum(geo.J * ref.wq[None, :], axis=1)
    xf = np.zeros((m.K, 4, ref.Ng, 3))
    for fc in range(4):
        xf[:, fc] = np.einsum('kgj,kjd->kgd', ref.Ig[fc][orient[:, fc]], X)
    wsJ = ref.wg[None, None, :] * geo.sJ
    flux_x = np.sum(wsJ * np.sum(xf * geo.nrm, axis=-1), axis=(1, 2)) / 3.0
    assert np.allclose(vol, flux_x, rtol=1e-11)
    assert np.abs(np.sum(wsJ[..., None] * geo.nrm, axis=(1, 2))).max() < 1e-11 * vol.max() ** (2 / 3)
    # neighbours see the same points, opposite normals, equal area factors
    for k in range(m.K):
        for fc in range(4):
            k2, f2 = EToE[k, fc], EToF[k, fc]
            d = xf[k, fc] - xf[k2, f2]
            d -= L_BOX * np.round(d / L_BOX)          # periodic images
            assert np.abs(d).max() < 1e-11
            assert np.allclose(geo.nrm[k, fc], -geo.nrm[k2, f2], atol=1e-11)
            assert np.allclose(geo.sJ[k, fc], geo.sJ[k2, f2], rtol=1e-11)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("warp", [0.0, 0.3])
def test_free_stream_and_conservation(N, warp):
    m, ref, X = warped_box(3, N, amp=warp)
    o = Oracle3(N, m.EToV, m.bc, X)
    uinf = states.freestream3(0.5, 10.0)
    assert np.abs(o.rhs(states.uniform_state3(m.K, ref.Np, uinf))).max() < 1e-12
    rng = np.random.default_rng(3)
    U = states.vortex3_state(X, period=(L_BOX, L_BOX))
    U = U + 0.01 * rng.standard_normal(U.shape)
    for flux in ("llf", "hllc"):
        o.numflux = {"llf": euler3.llf, "hllc": euler3.hllc}[flux]
        _, vol, surf = o.rhs(U, parts=True)
        # 1^T M_k L_k summed over the periodic mesh (M L = vol - surf)
        assert np.abs((vol - surf).sum(axis=(0, 2))).max() < 1e-11 * np.abs(vol).max()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_consistency_order_on_extruded_vortex(N):
    """|L(U_exact) - dU_exact/dt| at the nodes falls at order >= N - 1 + 1/2
    between n = 12 and n = 16 cells per side (measured: 1.97, 2.67, 3.60),
    on 300 sampled elements near the vortex core."""
    ref = tet.ReferenceTet(N)
    errs = []
    for n in (12, 16):
        m = meshes3d.box(n, L=L_BOX)
        X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
        o = Oracle3(N, m.EToV, m.bc, X)
        c = m.verts.mean(axis=1)
        near = np.where(np.hypot(c[:, 0] - 5, c[:, 1] - 5) < 2.5)[0]
        idx = np.random.default_rng(0).choice(near, 300, replace=False)
        U = states.vortex3_state(X, period=(L_BOX, L_BOX))
        d = 1e-5
        Ut = (states.vortex3_state(X[idx], t=d, period=(L_BOX, L_BOX))
              - states.vortex3_state(X[idx], t=-d, period=(L_BOX, L_BOX))) / (2 * d)
        errs.append(np.sqrt(np.mean((o.rhs(U, idx) - Ut) ** 2)))
    rate = np.log(errs[0] / errs[1]) / np.log(16 / 12)
    assert rate > N - 0.5, (N, errs, rate)


def _rot(a, b, c):
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    Ry = np.array([[np.cos(c), 0, np.sin(c)], [0, 1, 0], [-np.sin(c), 0, np.cos(c)]])
    return Rz @ Rx @ Ry


def test_rotation_invariance_with_walls():
    """Rotating the mesh and the flow rotates the right-hand side (curved
    walls, farfield, both fluxes)."""
    N = 3
    m = meshes3d.bump_channel(4, 2, 3)
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    uinf = states.freestream3(0.5, 3.0)
    rng = np.random.default_rng(5)
    U = states.uniform_state3(m.K, ref.Np, uinf)
    U[:, 1:4] += 0.05 * rng.standard_normal(U[:, 1:4].shape)
    U[:, 0] += 0.02 * rng.standard_normal(U[:, 0].shape)
    R = _rot(0.7, -0.4, 1.1)
    for flux in ("llf", "hllc"):
        L0 = Oracle3(N, m.EToV, m.bc, X, u_inf=uinf, flux=flux).rhs(U)
        Ur = U.copy()
        Ur[:, 1:4] = np.einsum('ij,kjp->kip', R, U[:, 1:4])
        uinf_r = uinf.copy()
        uinf_r[1:4] = R @ uinf[1:4]
        Lr = Oracle3(N, m.EToV, m.bc, X @ R.T, u_inf=uinf_r, flux=flux).rhs(Ur)
        L0r = L0.copy()
        L0r[:, 1:4] = np.einsum('ij,kjp->kip', R, L0[:, 1:4])
        assert np.abs(Lr - L0r).max() < 1e-10 * np.abs(L0).max()


def _rand_states(rng, n):
    rho = 0.5 + rng.random(n)
    vel = rng.standard_normal((3, n))
    p = 0.5 + rng.random(n)
    return states.conserved3(rho, vel[0], vel[1], vel[2], p)


def test_fluxes_consistency_antisymmetry_wall():
    rng = np.random.default_rng(2)
    nv = rng.standard_normal((3, 50))
    nx, ny, nz = nv / np.linalg.norm(nv, axis=0)
    A, B = _rand_states(rng, 50), _rand_states(rng, 50)
    for fl in (euler3.llf, euler3.hllc):
        assert np.allclose(fl(A, A, nx, ny, nz, 1.4), euler3.normal_flux(A, nx, ny, nz, 1.4), atol=1e-13)
        assert np.allclose(fl(A, B, nx, ny, nz, 1.4), -fl(B, A, -nx, -ny, -nz, 1.4), atol=1e-12)
        W = fl(A, euler3.wall_ghost(A, nx, ny, nz), nx, ny, nz, 1.4)
        assert np.abs(W[0]).max() < 1e-13 and np.abs(W[4]).max() < 1e-12
        # the momentum flux through a wall is along n
        mom = W[1:4]
        tang = mom - np.sum(mom * np.stack([nx, ny, nz]), axis=0) * np.stack([nx, ny, nz])
        assert np.abs(tang).max() < 1e-12


def test_hllc_resolves_contact_and_shear():
    """A stationary contact with a shear jump in both tangential directions
    gives exactly the one-sided flux (pressure only)."""
    n = np.array([[0.0], [0.6], [0.8]])
    t1 = np.array([1.0, 0.0, 0.0])
    t2 = np.cross(n[:, 0], t1)
    Um = states.conserved3(np.array([1.0]), *(0.3 * t1 + 0.1 * t2)[:, None], np.array([0.9]))
    Up = states.conserved3(np.array([0.4]), *(-0.5 * t1 + 0.7 * t2)[:, None], np.array([0.9]))
    F = euler3.hllc(Um, Up, *n, 1.4)
    assert abs(F[0, 0]) < 1e-14 and abs(F[4, 0]) < 1e-14
    assert np.allclose(F[1:4, 0], 0.9 * n[:, 0], atol=1e-14)
    assert np.abs(euler3.llf(Um, Up, *n, 1.4)[0]).max() > 0.1


@pytest.mark.parametrize("mistake", ["orientation", "lift_sign", "swap_st"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    N = 2
    m, ref, X = warped_box(3, N)
    o = Oracle3(N, m.EToV, m.bc, X)
    rng = np.random.default_rng(3)
    U = states.vortex3_state(X, period=(L_BOX, L_BOX)) + 0.01 * rng.standard_normal((m.K, 5, ref.Np))
    uinf = states.freestream3(0.5, 10.0)
    U0 = states.uniform_state3(m.K, ref.Np, uinf)
    if mistake == "orientation":
        monkeypatch.setattr(o, "_face_interp", lambda faces, orient: o.ref.Ig[faces, 0 * orient])
    elif mistake == "lift_sign":
        orig = euler3.llf
        o.numflux = lambda *a: -orig(*a)
    else:   # in the volume term only (the geometry is computed first)
        o.geometry()
        o.ref.Ds, o.ref.Dt = o.ref.Dt, o.ref.Ds
    fs = np.abs(o.rhs(U0)).max()
    _, vol, surf = o.rhs(U, parts=True)
    cons = np.abs((vol - surf).sum(axis=(0, 2))).max() / np.abs(vol).max()
    assert fs > 1e-6 or cons > 1e-6, (mistake, fs, cons)


def test_time_steppers_agree():
    """SSP-RK3 and LSERK(5,4) agree to O(dt^4) on one small step of the
    vortex (both are at least third order)."""
    N = 2
    m = meshes3d.box(3, L=L_BOX)
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    o = Oracle3(N, m.EToV, m.bc, X)
    U = states.vortex3_state(X, period=(L_BOX, L_BOX))
    d = []
    for dt in (0.02, 0.01):
        d.append(np.abs(o.ssp_rk3_step(U, dt) - o.lserk54_step(U, dt)).max())
    assert d[1] < d[0] / 12.0, d

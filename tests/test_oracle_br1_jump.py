"""Pins of the BR1 central fluxes of the artificial viscosity where eps jumps
across a face (paper Sec. 2: the first-order system q = sqrt(eps) grad U and
the viscous flux sqrt(eps) q, read with central fluxes (sqrt(eps) U)* and
(sqrt(eps) q)*), on triangles and tetrahedra.

Each eps_k is drawn per element, so every interior face carries a jump.
With the state constant (U = Ubar everywhere) the weak derivative of the
element's own sqrt(eps_k) Ubar equals its boundary integral exactly, so

  int_k q_m = 1^T M_k q_m,k
            = sum_f 1/2 (sqrt(eps_nb(f)) - sqrt(eps_k)) Ubar N_m(f)

and, with q given as a constant c_k per element, the viscous terms of L add

  1^T M_k (L_av - L)_k = sum_f 1/2 (sqrt(eps_nb(f)) c_nb - sqrt(eps_k) c_k) . N(f),

where N(f) is the outward normal times the length (area) of face f.  Both
sides are computed here from the vertex coordinates (N(f) from the edge or
face vectors, int_k from J_k and the reference mass (V V^T)^-1), not from the
oracle's geometry.  Planted mistakes -- the element's own sqrt(eps) on both
sides, or eps instead of sqrt(eps) on the neighbour's side -- break both
identities.
"""
import numpy as np
import pytest

from oracle import basis, nodes, tet
from oracle.dg import Oracle
from oracle.dg3 import Oracle3
from paper_1208_4772_gb300.inputs import meshes, meshes3d

UBAR = np.array([1.1, 0.3, -0.2, 2.7])
UBAR3 = np.array([1.1, 0.3, -0.2, 0.15, 2.7])


# ---------------------------------------------------------------- triangles
def tri_case(N, n=5, seed=7):
    m = meshes.periodic_square(n, length=10.0, seed=1000 + seed)
    r, s = nodes.warp_blend_nodes(N)
    xy = meshes.straight_nodes(m.verts, r, s)
    V = basis.vandermonde(N, r, s)
    mref = np.linalg.inv(V @ V.T)                                # reference mass on T (area 2)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.01, 0.3, m.K)
    return m, xy, mref, eps, rng


def tri_face_normals(m):
    """Outward normal times length of face f (vertices f -> f+1, CCW): [K,3,2]."""
    a = m.verts
    b = np.roll(m.verts, -1, axis=1)
    d = b - a
    return np.stack([d[..., 1], -d[..., 0]], axis=-1)


def tri_jacobian(m):
    d1 = m.verts[:, 1] - m.verts[:, 0]
    d2 = m.verts[:, 2] - m.verts[:, 0]
    return 0.5 * (d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]) / 2.0   # area / area(T)


def tri_integrals(m, mref, f):
    """int_k f for nodal fields f [K, ..., Np] on affine elements."""
    return tri_jacobian(m).reshape((-1,) + (1,) * (f.ndim - 1))[..., 0] * (f @ mref.sum(axis=0))


def tri_gradient_identity(o, m, mref, eps):
    U = np.broadcast_to(UBAR[None, :, None], (m.K, 4, o.ref.Np)).copy()
    q = o.gradient_q(U, eps, np.arange(m.K))                     # [K, 2, 4, Np]
    got = tri_integrals(m, mref, q)                              # [K, 2, 4]
    Nf = tri_face_normals(m)
    jump = 0.5 * (np.sqrt(eps[m.EToE]) - np.sqrt(eps)[:, None])  # [K, 3]
    want = np.einsum('kf,kfm,v->kmv', jump, Nf, UBAR)
    return got, want


def tri_viscous_identity(o_av, o, m, mref, eps, rng):
    U = np.broadcast_to(UBAR[None, :, None], (m.K, 4, o.ref.Np)).copy()
    c = rng.standard_normal((m.K, 2, 4))
    q = np.broadcast_to(c[..., None], (m.K, 2, 4, o.ref.Np)).copy()
    dL = o_av.rhs(U, eps=eps, q=q) - o.rhs(U)
    got = tri_integrals(m, mref, dL)                             # [K, 4]
    Nf = tri_face_normals(m)
    sc = np.sqrt(eps)[:, None, None] * c                         # [K, 2, 4]
    flux = 0.5 * (sc[m.EToE] - sc[:, None])                      # [K, 3, 2, 4]
    want = np.einsum('kfmv,kfm->kv', flux, Nf)
    return got, want


@pytest.mark.parametrize("N", [2, 3, 4])
def test_tri_br1_gradient_across_eps_jumps(N):
    m, xy, mref, eps, _ = tri_case(N)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=True)
    got, want = tri_gradient_identity(o, m, mref, eps)
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_tri_br1_viscous_flux_across_eps_jumps(N):
    m, xy, mref, eps, rng = tri_case(N)
    o_av = Oracle(N, m.EToE, m.EToF, m.bc, xy, av=True)
    o = Oracle(N, m.EToE, m.EToF, m.bc, xy)
    got, want = tri_viscous_identity(o_av, o, m, mref, eps, rng)
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def _planted_tri(kind):
    class Planted(Oracle):
        def _sqrt_eps_faces(self, eps, idx):
            se, sep = super()._sqrt_eps_faces(eps, idx)
            if kind == "own":        # the element's own sqrt(eps) on both sides
                return se, np.broadcast_to(se[:, None], sep.shape)
            return se, sep ** 2      # eps, not sqrt(eps), on the neighbour's side
    return Planted


@pytest.mark.parametrize("kind", ["own", "eps"])
def test_tri_planted_weighting_mistakes_are_caught(kind):
    N = 2
    m, xy, mref, eps, rng = tri_case(N)
    P = _planted_tri(kind)
    got, want = tri_gradient_identity(P(N, m.EToE, m.EToF, m.bc, xy, av=True), m, mref, eps)
    assert np.abs(got - want).max() > 1e-3 * np.abs(want).max()
    got, want = tri_viscous_identity(P(N, m.EToE, m.EToF, m.bc, xy, av=True),
                                     Oracle(N, m.EToE, m.EToF, m.bc, xy), m, mref, eps, rng)
    assert np.abs(got - want).max() > 1e-3 * np.abs(want).max()


# ---------------------------------------------------------------- tetrahedra
def tet_case(N, n=3, seed=5):
    m = meshes3d.box(n, L=10.0, seed=1000 + seed)
    ref = tet.ReferenceTet(N)
    X = meshes3d.node_coords(m, ref.r, ref.s, ref.t)
    mref = np.linalg.inv(ref.V @ ref.V.T)                        # reference mass (volume 4/3)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.01, 0.3, m.K)
    return m, X, mref, eps, rng


def tet_faces(m):
    """For each element and each neighbour sharing three vertex numbers: the
    neighbour's index and the outward normal times area of the shared face,
    from the element's own (unwrapped) vertex coordinates.  Returns lists of
    (k, nb, N) triples."""
    owners = {}
    for k, ids in enumerate(m.EToV):
        for skip in range(4):
            key = tuple(sorted(int(v) for j, v in enumerate(ids) if j != skip))
            owners.setdefault(key, []).append((k, skip))
    out = []
    for key, pair in owners.items():
        assert len(pair) == 2, "periodic box: every face is shared by two elements"
        for (k, skip), (nb, _) in (pair, pair[::-1]):
            P = m.verts[k]
            face = [P[j] for j in range(4) if j != skip]
            nrm = 0.5 * np.cross(face[1] - face[0], face[2] - face[0])
            if np.dot(nrm, P[skip] - face[0]) > 0:              # point away from the fourth vertex
                nrm = -nrm
            out.append((k, nb, nrm))
    return out


def tet_integrals(m, mref, f):
    d = m.verts[:, 1:] - m.verts[:, :1]
    J = np.abs(np.linalg.det(d)) / 6.0 / (4.0 / 3.0)              # volume / volume of the reference tet
    return J.reshape((-1,) + (1,) * (f.ndim - 2)) * (f @ mref.sum(axis=0))


def tet_gradient_identity(o, m, mref, eps):
    U = np.broadcast_to(UBAR3[None, :, None], (m.K, 5, o.ref.Np)).copy()
    q = o.gradient_q(U, eps, np.arange(m.K))                     # [K, 3, 5, Np]
    got = tet_integrals(m, mref, q)                              # [K, 3, 5]
    want = np.zeros_like(got)
    for k, nb, nrm in tet_faces(m):
        want[k] += 0.5 * (np.sqrt(eps[nb]) - np.sqrt(eps[k])) * nrm[:, None] * UBAR3[None, :]
    return got, want


def tet_viscous_identity(o_av, o, m, mref, eps, rng):
    U = np.broadcast_to(UBAR3[None, :, None], (m.K, 5, o.ref.Np)).copy()
    c = rng.standard_normal((m.K, 3, 5))
    q = np.broadcast_to(c[..., None], (m.K, 3, 5, o.ref.Np)).copy()
    dL = o_av.rhs(U, eps=eps, q=q) - o.rhs(U)
    got = tet_integrals(m, mref, dL)                             # [K, 5]
    want = np.zeros_like(got)
    sc = np.sqrt(eps)[:, None, None] * c
    for k, nb, nrm in tet_faces(m):
        want[k] += 0.5 * np.einsum('mv,m->v', sc[nb] - sc[k], nrm)
    return got, want


@pytest.mark.parametrize("N", [2, 3])
def test_tet_br1_gradient_across_eps_jumps(N):
    m, X, mref, eps, _ = tet_case(N)
    o = Oracle3(N, m.EToV, m.bc, X, av=True)
    got, want = tet_gradient_identity(o, m, mref, eps)
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("N", [2, 3])
def test_tet_br1_viscous_flux_across_eps_jumps(N):
    m, X, mref, eps, rng = tet_case(N)
    o_av = Oracle3(N, m.EToV, m.bc, X, av=True)
    o = Oracle3(N, m.EToV, m.bc, X)
    got, want = tet_viscous_identity(o_av, o, m, mref, eps, rng)
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("kind", ["own", "eps"])
def test_tet_planted_weighting_mistakes_are_caught(kind):
    N = 2
    m, X, mref, eps, rng = tet_case(N)

    class Planted(Oracle3):
        def _sqrt_eps_faces(self, eps, idx):
            se, sep = super()._sqrt_eps_faces(eps, idx)
            if kind == "own":
                return se, np.broadcast_to(se[:, None], sep.shape)
            return se, sep ** 2
    got, want = tet_gradient_identity(Planted(N, m.EToV, m.bc, X, av=True), m, mref, eps)
    assert np.abs(got - want).max() > 1e-3 * np.abs(want).max()
    got, want = tet_viscous_identity(Planted(N, m.EToV, m.bc, X, av=True), Oracle3(N, m.EToV, m.bc, X),
                                     m, mref, eps, rng)
    assert np.abs(got - want).max() > 1e-3 * np.abs(want).max()

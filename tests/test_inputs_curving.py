"""Pins of the FP64 host curving step (paper Sec. 3 in 2D) and of the
synthetic meshes: wall nodes on the exact curve, other faces untouched, the
elasticity solve reproduces affine fields (patch test), positive Jacobians,
and the domain area converging with the degree."""
import numpy as np
import pytest

from oracle.geometry import ElementGeometry
from oracle.operators import ReferenceElement
from paper_1208_4772_gb300.inputs import curving, meshes


def _face_mask(ref, f):
    return curving._on_face(ref.r, ref.s, f)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_cylinder_wall_nodes_on_circle(N):
    ref = ReferenceElement(N)
    m = meshes.cylinder_channel(n_t=24, n_r=4)
    xy, curved = curving.curve_mesh(m, N, ref.r, ref.s)
    straight = meshes.straight_nodes(m.verts, ref.r, ref.s)
    for k, f in zip(*np.nonzero(m.bc == meshes.BC_WALL)):
        on = _face_mask(ref, f)
        assert np.abs(np.linalg.norm(xy[k, on], axis=1) - 0.5).max() < 1e-12
        for g in range(3):
            if g != f:
                other = _face_mask(ref, g)
                assert np.abs(xy[k, other] - straight[k, other]).max() == 0.0
    assert np.all(xy[~curved] == straight[~curved])


def test_naca_wall_nodes_on_curve():
    N = 4
    ref = ReferenceElement(N)
    m = meshes.naca_omesh(n_t=40, n_r=4)
    xy, curved = curving.curve_mesh(m, N, ref.r, ref.s)
    curve = m.curve
    dense = curve.point(np.linspace(-1, 1, 200001))
    for k, f in zip(*np.nonzero(m.bc == meshes.BC_WALL)):
        P = xy[k, _face_mask(ref, f)]
        # on the curve: refine the nearest dense sample by Gauss-Newton
        i = np.argmin(np.linalg.norm(P[:, None, :] - dense[None, :, :], axis=-1), axis=1)
        sg0 = np.linspace(-1, 1, 200001)[i]
        C, sg = curve.project(P, sg0, -1.0, 1.0)
        assert np.abs(C - P).max() < 1e-12


def test_elasticity_patch_test():
    """A degree-N elasticity solve with affine Dirichlet data returns the
    affine field at the interior nodes (linear fields are exact FE solutions)."""
    for N in (3, 4, 6):
        ref = ReferenceElement(N)
        Lr, Ls, qw = curving.basis_pieces(N, ref.r, ref.s)
        verts = np.array([[0.2, 0.1], [1.3, 0.4], [0.5, 1.7]])
        X = meshes.straight_nodes(verts[None], ref.r, ref.s)[0]
        A = np.array([[0.01, -0.03], [0.02, 0.015]])
        g = X @ A.T + np.array([0.005, -0.002])
        interior = ~(_face_mask(ref, 0) | _face_mask(ref, 1) | _face_mask(ref, 2))
        gin = g.copy()
        gin[interior] = 0.0
        u = curving.elastic_fill(verts, gin, interior, Lr, Ls, qw, 0.45)
        assert np.abs(u - g).max() < 1e-13


@pytest.mark.parametrize("kind", ["naca", "cyl"])
def test_curved_jacobian_positive(kind):
    for N in (2, 4, 6):
        ref = ReferenceElement(N)
        m = meshes.naca_omesh(n_t=60, n_r=6) if kind == "naca" else meshes.cylinder_channel(n_t=40, n_r=6)
        xy, curved = curving.curve_mesh(m, N, ref.r, ref.s)
        geo = ElementGeometry(ref, xy[curved])
        assert geo.J.min() > 0


def test_cylinder_area_converges_with_degree():
    """Sum of int 1 over the curved mesh -> area of (outer polygon minus the
    disc); the error falls as the wall representation gains degree."""
    m = meshes.cylinder_channel(n_t=16, n_r=3)
    outer = []
    far = np.nonzero(m.bc == meshes.BC_FARFIELD)
    # outer polygon area by the shoelace formula over the farfield edges
    area_outer = 0.0
    for k, f in zip(*far):
        a, b = m.verts[k, f], m.verts[k, (f + 1) % 3]
        area_outer += 0.5 * (a[0] * b[1] - a[1] * b[0])
    exact = area_outer - np.pi * 0.25
    errs = []
    for N in (1, 2, 3, 4, 5, 6):
        ref = ReferenceElement(N)
        xy, _ = curving.curve_mesh(m, N, ref.r, ref.s)
        geo = ElementGeometry(ref, xy)
        errs.append(abs(np.sum(geo.J * ref.wq) - exact))
    errs = np.array(errs)
    assert errs[0] > 1e-3                      # straight-sided (N = 1) misses the disc
    assert np.all(errs[1:] < errs[0])
    assert errs[-1] < 1e-6 * errs[0]


def test_mesh_sizes_and_boundaries():
    m = meshes.naca_omesh(n_t=300, n_r=100)
    assert m.K == 60000
    assert np.sum(m.bc == meshes.BC_WALL) == 300
    assert np.sum(m.bc == meshes.BC_FARFIELD) == 300
    v = m.verts
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    assert np.all(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0] > 0)
    p = meshes.periodic_square(16)
    assert p.K == 512 and np.all(p.bc == 0)
    # connectivity is symmetric
    for mm in (m, p):
        k = np.arange(mm.K)[:, None].repeat(3, 1)
        f = np.arange(3)[None, :].repeat(mm.K, 0)
        inner = mm.bc == 0
        assert np.all(mm.EToE[mm.EToE[inner], mm.EToF[inner]] == k[inner])
        assert np.all(mm.EToF[mm.EToE[inner], mm.EToF[inner]] == f[inner])

"""Seeded synthetic tetrahedral meshes (inputs only; none of the
discretisation's arithmetic).

Stand-ins for the paper's tetrahedral workloads (Sec. 5: sphere, NACA 0012
extrusion, ONERA M6, none of which is available):

* ``box``: the periodic cube [0, L]^3 cut into n^3 cells, each cell split
  into six tetrahedra along its main diagonal (the Kuhn split, conforming
  between cells), every lattice vertex jittered uniformly in
  [-j h, j h]^3 with its periodic images moved together.  For the
  extruded isentropic vortex (exact solution, convergence and parity).
* ``bump_channel``: the channel [0, Lx] x [0, Ly] x [0, H] (y periodic) of
  nx x ny x nz Kuhn-split cells, interior vertices jittered, whose floor
  carries the smooth bump z = A cos^2(pi rho / (2 R)) (rho < R, the
  distance from the bump centre).  The map
      (x, y, z) -> (x, y, z + bump(x, y) g(z)),  g(z) = (1 - z/Zd)^2 for
      z < Zd, 0 above,
  is applied to every collocation node, so elements inside the bump's
  footprint below z = Zd are curved (the floor nodes lie on the bump
  surface exactly) and all others stay affine.  Boundary codes: floor and
  ceiling slip walls, inflow and outflow planes farfield.

Elements are positively oriented: det[v1-v0, v2-v0, v3-v0] > 0 for the
local vertex order, matching the reference tetrahedron
(-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1).  Global vertex numbers identify
periodic images.  ``node_coords(mesh, r, s, t)`` returns the collocation
node coordinates [K, Np, 3] for a reference node set passed in by the
caller.
"""
from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2
FACES = ((0, 2, 1), (0, 1, 3), (1, 2, 3), (0, 3, 2))   # local vertices of each face


@dataclass
class TetMesh:
    name: str
    verts: np.ndarray          # [K, 4, 3] vertex coordinates (unwrapped, before the map)
    EToV: np.ndarray           # [K, 4] global vertex numbers
    bc: np.ndarray             # [K, 4] per face
    mapping: object = None     # smooth map applied to the nodes, or None
    meta: dict = field(default_factory=dict)

    @property
    def K(self):
        return self.EToV.shape[0]


def _kuhn(n_cells, vid, coord):
    """Six tetrahedra per cell, cells ordered l (z) outer, j, i inner, the six
    paths through each cell in the order of the axis permutations.
    vid(I, J, L) -> global numbers and coord(I, J, L) -> [..., 3] coordinates
    of lattice points (unwrapped), both on integer arrays."""
    nx, ny, nz = n_cells
    L, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([I.ravel(), J.ravel(), L.ravel()], axis=1)            # [C, 3]
    paths = []
    for perm in permutations(range(3)):
        p = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            q = p[-1].copy()
            q[ax] += 1
            p.append(q)
        paths.append(np.stack(p))                                           # [4, 3]
    pts = cells[:, None, None, :] + np.stack(paths)[None]                   # [C, 6, 4, 3]
    pts = pts.reshape(-1, 4, 3)
    EToV = vid(pts[..., 0], pts[..., 1], pts[..., 2]).astype(np.int64)
    verts = coord(pts[..., 0], pts[..., 1], pts[..., 2]).astype(np.float64)
    vol = np.einsum('ki,ki->k', np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0]),
                    verts[:, 3] - verts[:, 0])
    flip = vol < 0
    EToV[flip] = EToV[flip][:, [0, 1, 3, 2]]
    verts[flip] = verts[flip][:, [0, 1, 3, 2]]
    return EToV, verts


def box(n, L=10.0, jitter=0.1, seed=1000):
    rng = np.random.default_rng(seed)
    h = L / n
    jit = rng.uniform(-jitter * h, jitter * h, size=(n, n, n, 3))

    def vid(i, j, l):
        return (i % n) + n * ((j % n) + n * (l % n))

    def coord(i, j, l):
        return np.stack([i * h, j * h, l * h], axis=-1) + jit[i % n, j % n, l % n]

    EToV, verts = _kuhn((n, n, n), vid, coord)
    bc = np.zeros((len(EToV), 4), dtype=np.int8)
    return TetMesh("box", verts, EToV, bc, meta=dict(n=n, L=L, jitter=jitter, seed=seed, period=(L, L, L)))


def bump_channel(nx, ny, nz, Lx=3.0, Ly=1.5, H=0.8, A=0.1, R=0.4, Zd=0.4, jitter=0.1, seed=2000):
    # dz'/dz = 1 - 2 bump (1 - z/Zd) / Zd >= 1 - 2 A / Zd: keep it >= 1/2
    if Zd < 4.0 * A:
        raise ValueError("the bump map needs Zd >= 4 A to stay well inside one-to-one")
    rng = np.random.default_rng(seed)
    hx, hy, hz = Lx / nx, Ly / ny, H / nz
    jit = rng.uniform(-jitter, jitter, size=(nx + 1, ny, nz + 1, 3)) * np.array([hx, hy, hz])
    jit[0, :, :, 0] = jit[nx, :, :, 0] = 0.0          # inflow / outflow planes stay planar
    jit[:, :, 0, 2] = jit[:, :, nz, 2] = 0.0          # floor / ceiling stay planar

    def vid(i, j, l):
        return i + (nx + 1) * ((j % ny) + ny * l)

    def coord(i, j, l):
        return np.stack([i * hx, j * hy, l * hz], axis=-1) + jit[i, j % ny, l]

    EToV, verts = _kuhn((nx, ny, nz), vid, coord)
    K = len(EToV)
    bc = np.zeros((K, 4), dtype=np.int8)
    tol = 1e-9
    for f, fv in enumerate(FACES):
        P = verts[:, fv, :]
        floor = np.all(np.abs(P[..., 2]) < tol, axis=1)
        ceil = np.all(np.abs(P[..., 2] - H) < tol, axis=1)
        inflow = np.all(np.abs(P[..., 0]) < tol, axis=1)
        outflow = np.all(np.abs(P[..., 0] - Lx) < tol, axis=1)
        bc[floor | ceil, f] = BC_WALL
        bc[inflow | outflow, f] = BC_FARFIELD
    xc, yc = 0.5 * Lx, 0.5 * Ly

    def mapping(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        rho = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
        bump = np.where(rho < R, A * np.cos(0.5 * np.pi * np.minimum(rho, R) / R) ** 2, 0.0)
        g = np.where(z < Zd, (1.0 - np.minimum(z, Zd) / Zd) ** 2, 0.0)
        out = X.copy()
        out[..., 2] = z + bump * g
        return out

    return TetMesh("bump_channel", verts, EToV, bc, mapping=mapping,
                   meta=dict(n=(nx, ny, nz), L=(Lx, Ly, H), A=A, R=R, Zd=Zd, jitter=jitter, seed=seed))


def node_coords(mesh, r, s, t):
    """Collocation nodes [K, Np, 3]: the affine image of the reference nodes
    through each element's vertices, then the mesh's map (if any)."""
    r, s, t = (np.asarray(a, dtype=np.float64) for a in (r, s, t))
    lam = np.stack([-(1.0 + r + s + t) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0, (1.0 + t) / 2.0], axis=1)
    X = np.einsum('pv,kvd->kpd', lam, mesh.verts)
    if mesh.mapping is not None:
        X = mesh.mapping(X)
    return X


def mapped_elements(mesh, r, s, t):
    """Mask of the elements whose nodes the mesh's map moves (the curved
    ones); all False without a map."""
    r, s, t = (np.asarray(a, dtype=np.float64) for a in (r, s, t))
    lam = np.stack([-(1.0 + r + s + t) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0, (1.0 + t) / 2.0], axis=1)
    X = np.einsum('pv,kvd->kpd', lam, mesh.verts)
    if mesh.mapping is None:
        return np.zeros(mesh.K, dtype=bool)
    return np.any(np.abs(mesh.mapping(X) - X) > 0.0, axis=(1, 2))

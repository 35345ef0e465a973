"""Seeded synthetic triangular meshes.

Stand-ins for the paper's workloads (Sec. 5 uses 3D sphere / NACA0012 /
ONERA M6 tetrahedral meshes that are not available): a jittered periodic
square for the isentropic vortex, an O-type mesh around the NACA 0012
profile in a radius-20 farfield, and an O-type mesh around a cylinder in a
rectangular channel.  Every element is counter-clockwise; face f joins local
vertices f and (f+1) mod 3.  Boundary codes: 0 interior, 1 slip wall,
2 farfield.

This module generates inputs only; it contains none of the discretisation's
arithmetic.  Node coordinates are produced from a reference node set that the
caller passes in (``straight_nodes``).
"""
from dataclasses import dataclass, field

import numpy as np

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


@dataclass
class TriMesh:
    name: str
    verts: np.ndarray          # [K, 3, 2] element vertex coordinates (unwrapped)
    EToV: np.ndarray           # [K, 3] vertex ids (periodic images share ids)
    EToE: np.ndarray = None    # [K, 3]
    EToF: np.ndarray = None    # [K, 3]
    bc: np.ndarray = None      # [K, 3]
    curve: object = None       # wall curve (closest-point projection), or None
    meta: dict = field(default_factory=dict)

    @property
    def K(self):
        return self.EToV.shape[0]

    def wall_elements(self):
        return np.nonzero(np.any(self.bc == BC_WALL, axis=1))[0]


def _orient(verts, EToV):
    a = verts[:, 1] - verts[:, 0]
    b = verts[:, 2] - verts[:, 0]
    area2 = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    flip = area2 < 0
    verts[flip] = verts[flip][:, [0, 2, 1]]
    EToV[flip] = EToV[flip][:, [0, 2, 1]]
    return verts, EToV


def connect(mesh, boundary_code=None):
    """Face-to-face connectivity from shared vertex pairs.  Unmatched faces
    are boundary faces: EToE = self, EToF = own face, bc from
    boundary_code(k, f, midpoint) (default farfield)."""
    K = mesh.K
    EToE = np.repeat(np.arange(K)[:, None], 3, axis=1)
    EToF = np.repeat(np.arange(3)[None, :], K, axis=0).copy()
    bc = np.zeros((K, 3), dtype=np.int8)
    a = mesh.EToV
    b = np.roll(mesh.EToV, -1, axis=1)
    lo, hi = np.minimum(a, b).ravel(), np.maximum(a, b).ravel()
    key = lo.astype(np.int64) * (int(mesh.EToV.max()) + 1) + hi
    order = np.argsort(key, kind='stable')
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    f1, f2 = order[same], order[same + 1]
    if np.any(np.bincount(np.concatenate([f1, f2]), minlength=3 * K) > 1):
        raise ValueError("non-manifold face")
    EToE.ravel()[f1], EToF.ravel()[f1] = f2 // 3, f2 % 3
    EToE.ravel()[f2], EToF.ravel()[f2] = f1 // 3, f1 % 3
    matched = np.zeros(3 * K, dtype=bool)
    matched[f1] = True
    matched[f2] = True
    for g in np.nonzero(~matched)[0]:
        k, f = divmod(int(g), 3)
        mid = 0.5 * (mesh.verts[k, f] + mesh.verts[k, (f + 1) % 3])
        bc[k, f] = BC_FARFIELD if boundary_code is None else boundary_code(k, f, mid)
    mesh.EToE, mesh.EToF, mesh.bc = EToE.astype(np.int32), EToF.astype(np.int8), bc
    return mesh


def straight_nodes(verts, r, s):
    """Affine images of reference nodes (r, s) on T = (-1,-1),(1,-1),(-1,1)."""
    l1, l2, l3 = -(r + s) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0
    return (l1[None, :, None] * verts[:, None, 0] + l2[None, :, None] * verts[:, None, 1]
            + l3[None, :, None] * verts[:, None, 2])


# ---------------------------------------------------------------- periodic
def periodic_square(n, length=10.0, jitter=0.1, seed=1000, origin=(0.0, 0.0)):
    """[0, L]^2 (shifted by origin) split into n x n squares, each cut along
    the same diagonal (2 n^2 triangles); every lattice vertex moved uniformly
    within [-jitter h, jitter h]^2, periodic images together."""
    rng = np.random.default_rng(seed)
    h = length / n
    shift = rng.uniform(-jitter * h, jitter * h, size=(n * n, 2))
    verts, ids = [], []

    def vid(i, j):
        return (i % n) + n * (j % n)

    def pos(i, j):
        return np.array([origin[0] + i * h, origin[1] + j * h]) + shift[vid(i, j)]

    for j in range(n):
        for i in range(n):
            a, b, c, d = (i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)
            for tri in ((a, b, c), (a, c, d)):
                verts.append([pos(*p) for p in tri])
                ids.append([vid(*p) for p in tri])
    m = TriMesh("periodic_square", np.array(verts), np.array(ids, dtype=np.int64),
                meta=dict(n=n, length=length, h=h, origin=origin, seed=seed))
    m.verts, m.EToV = _orient(m.verts, m.EToV)
    connect(m)
    if np.any(m.bc != BC_INTERIOR):
        raise ValueError("periodic mesh has boundary faces")
    return m


# ---------------------------------------------------------------- curves
class NacaCurve:
    """NACA 00tt thickness curve, chord 1, closed trailing edge, parametrised
    by sigma in [-1, 1]: x = sigma^2, y = sign(sigma) t(|sigma|) with
    t(c) = 5 tau (0.2969 c - 0.1260 c^2 - 0.3516 c^4 + 0.2843 c^6 - 0.1036 c^8).
    sigma = 1 is the upper trailing edge, 0 the leading edge, -1 the lower
    trailing edge."""

    def __init__(self, tau=0.12):
        self.tau = tau

    def point(self, sg):
        sg = np.asarray(sg, dtype=np.float64)
        c = np.abs(sg)
        t = 5 * self.tau * (0.2969 * c - 0.1260 * c ** 2 - 0.3516 * c ** 4 + 0.2843 * c ** 6 - 0.1036 * c ** 8)
        return np.stack([sg * sg, np.sign(sg) * t], axis=-1)

    def dpoint(self, sg):
        sg = np.asarray(sg, dtype=np.float64)
        c = np.abs(sg)
        dt = 5 * self.tau * (0.2969 - 2 * 0.1260 * c - 4 * 0.3516 * c ** 3 + 6 * 0.2843 * c ** 5 - 8 * 0.1036 * c ** 7)
        return np.stack([2 * sg, dt], axis=-1)

    def project(self, x, sg0, lo, hi, iters=60):
        """Closest point on the curve (Gauss-Newton on the parameter, kept in
        [lo, hi]); paper Sec. 3 closest-point problem in 1D."""
        sg = np.array(sg0, dtype=np.float64)
        for _ in range(iters):
            c, dc = self.point(sg), self.dpoint(sg)
            step = np.sum(dc * (x - c), axis=-1) / np.sum(dc * dc, axis=-1)
            sg = np.clip(sg + step, lo, hi)
            if np.max(np.abs(step)) < 1e-15:
                break
        return self.point(sg), sg


class CircleCurve:
    """Circle of radius R about x0: the exact closest point is
    x0 + R (x - x0) / |x - x0| (paper Sec. 5, sphere displacement g)."""

    def __init__(self, center=(0.0, 0.0), radius=0.5):
        self.x0 = np.asarray(center, dtype=np.float64)
        self.R = float(radius)

    def project(self, x, *unused):
        d = x - self.x0
        return self.x0 + self.R * d / np.linalg.norm(d, axis=-1, keepdims=True), None


def _omesh(name, surf, outer, n_r, ratio, jitter, rng, curve, wall_param=None):
    """Structured O-grid between a closed inner curve surf [n_t, 2] and an
    outer curve outer [n_t, 2], geometric radial spacing, random diagonal per
    quad (wall-adjacent quads: the better-shaped wall triangle), interior
    vertices jittered by up to jitter * local spacing."""
    n_t = surf.shape[0]
    g = (ratio ** np.arange(n_r + 1) - 1.0) / (ratio ** n_r - 1.0)
    P = surf[None, :, :] + (outer - surf)[None, :, :] * g[:, None, None]   # [n_r+1, n_t, 2]
    # local spacing for jitter
    dr = np.linalg.norm(np.diff(P, axis=0), axis=-1)
    dt = np.linalg.norm(np.roll(P, -1, axis=1) - P, axis=-1)
    hloc = np.full(P.shape[:2], np.inf)
    hloc[:-1] = np.minimum(hloc[:-1], dr)
    hloc[1:] = np.minimum(hloc[1:], dr)
    hloc = np.minimum(hloc, dt)
    hloc = np.minimum(hloc, np.roll(dt, 1, axis=1))
    jit = rng.uniform(-jitter, jitter, size=P.shape) * hloc[..., None]
    jit[0] = 0.0
    jit[-1] = 0.0
    P = P + jit

    def vid(l, i):
        return l * n_t + (i % n_t)

    verts, ids, diag = [], [], rng.integers(0, 2, size=(n_r, n_t))

    def wall_quality(p0, p1, p2):   # 2 area / longest edge^2 of a wall triangle
        e = [np.sum((P[q[0], q[1] % n_t] - P[r[0], r[1] % n_t]) ** 2) for q, r in ((p0, p1), (p1, p2), (p2, p0))]
        u, w = P[p1[0], p1[1] % n_t] - P[p0[0], p0[1] % n_t], P[p2[0], p2[1] % n_t] - P[p0[0], p0[1] % n_t]
        return abs(u[0] * w[1] - u[1] * w[0]) / max(e)

    # wall-adjacent quads: the diagonal whose wall triangle is better shaped
    # (where a grid line leaves a corner of the wall, e.g. a trailing edge,
    # the other choice gives a sliver that curving the wall edge inverts)
    for i in range(n_t):
        a, b, c, d = (0, i), (0, i + 1), (1, i + 1), (1, i)
        diag[0, i] = 0 if wall_quality(a, b, c) >= wall_quality(a, b, d) else 1
    for l in range(n_r):
        for i in range(n_t):
            a, b, c, d = (l, i), (l, i + 1), (l + 1, i + 1), (l + 1, i)
            tris = ((a, b, c), (a, c, d)) if diag[l, i] == 0 else ((a, b, d), (b, c, d))
            for tri in tris:
                verts.append([P[p[0], p[1] % n_t] for p in tri])
                ids.append([vid(*p) for p in tri])
    m = TriMesh(name, np.array(verts), np.array(ids, dtype=np.int64), curve=curve)
    m.verts, m.EToV = _orient(m.verts, m.EToV)
    inner_ids = set(range(n_t))

    def code(k, f, mid):
        v0, v1 = m.EToV[k, f], m.EToV[k, (f + 1) % 3]
        return BC_WALL if (v0 in inner_ids and v1 in inner_ids) else BC_FARFIELD

    connect(m, code)
    m.meta.update(n_t=n_t, n_r=n_r, ratio=ratio)
    if wall_param is not None:
        m.meta["wall_param"] = wall_param
    return m


def naca_omesh(n_t=300, n_r=100, radius=20.0, ratio=1.06, jitter=0.1, seed=1001, tau=0.12):
    """O-mesh around NACA 00(100 tau), chord 1, farfield circle of the given
    radius about (0.5, 0); 2 n_t n_r triangles."""
    rng = np.random.default_rng(seed)
    curve = NacaCurve(tau)
    # sigma uniform from 1 to -1 (counter-clockwise); x = sigma^2 clusters
    # points at the leading edge and keeps the trailing-edge cells regular
    sg = 1.0 - 2.0 * np.arange(n_t) / n_t
    surf = curve.point(sg)
    # grid lines leave the wall along its outward normal (the bisector at the
    # trailing-edge corner) and end on the farfield circle about (0.5, 0)
    tang = -curve.dpoint(sg)                  # traversal direction (sigma decreasing)
    nrm = np.stack([tang[:, 1], -tang[:, 0]], axis=-1)
    nrm[0] = (1.0, 0.0)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    rel = surf - np.array([0.5, 0.0])
    b = np.sum(rel * nrm, axis=-1)
    t = -b + np.sqrt(b * b - (np.sum(rel * rel, axis=-1) - radius ** 2))
    outer = surf + t[:, None] * nrm
    # the parameter of surface vertex i, with the wrap to sigma = -1 at i = n_t
    param = np.concatenate([sg, [-1.0]])
    return _omesh("naca0012", surf, outer, n_r, ratio, jitter, rng, curve, wall_param=param)


def cylinder_channel(n_t=500, n_r=250, radius=0.5, box=(-10.0, 20.0, -10.0, 10.0),
                     ratio=1.02, jitter=0.1, seed=1002):
    """O-mesh between a cylinder of the given radius at the origin and the
    rectangle box = (x0, x1, y0, y1) reached along rays; 2 n_t n_r triangles."""
    rng = np.random.default_rng(seed)
    th = 2 * np.pi * np.arange(n_t) / n_t
    d = np.stack([np.cos(th), np.sin(th)], axis=-1)
    surf = radius * d
    x0, x1, y0, y1 = box
    with np.errstate(divide='ignore'):
        tx = np.where(d[:, 0] > 0, x1 / d[:, 0], np.where(d[:, 0] < 0, x0 / d[:, 0], np.inf))
        ty = np.where(d[:, 1] > 0, y1 / d[:, 1], np.where(d[:, 1] < 0, y0 / d[:, 1], np.inf))
    outer = d * np.minimum(tx, ty)[:, None]
    return _omesh("cylinder_channel", surf, outer, n_r, ratio, jitter, rng, CircleCurve((0.0, 0.0), radius))


def locality_order(mesh):
    """A permutation of elements that keeps neighbours close in memory
    (breadth-first order from element 0).  Returns (perm, mesh') where
    mesh' has elements renumbered as perm."""
    K = mesh.K
    seen = np.zeros(K, dtype=bool)
    order = []
    for start in range(K):
        if seen[start]:
            continue
        seen[start] = True
        frontier = [start]
        while frontier:
            nxt = []
            for k in frontier:
                order.append(k)
                for nb in mesh.EToE[k]:
                    if not seen[nb]:
                        seen[nb] = True
                        nxt.append(int(nb))
            frontier = nxt
    perm = np.array(order, dtype=np.int64)
    return renumber(mesh, perm)


def renumber(mesh, perm):
    """New element i is old element perm[i]."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    m = TriMesh(mesh.name, mesh.verts[perm].copy(), mesh.EToV[perm].copy(), curve=mesh.curve,
                meta=dict(mesh.meta))
    m.EToE = inv[mesh.EToE[perm]].astype(np.int32)
    m.EToF = mesh.EToF[perm].copy()
    m.bc = mesh.bc[perm].copy()
    return perm, m

"""Shared seeded test cases: a mesh, its node coordinates on the library's
reference nodes, parameters, and a perturbed state.  Inputs only."""
import numpy as np

from paper_1208_4772_gb300.inputs import curving, meshes, states


def rel_l2_per_var(a, b):
    """||a - b|| / ||b|| per conserved variable (arrays [K, 4, Np])."""
    return np.linalg.norm((a - b).transpose(1, 0, 2).reshape(4, -1), axis=1) / \
        np.linalg.norm(b.transpose(1, 0, 2).reshape(4, -1), axis=1)


def make_case(kind, N, r, s, seed=0, av=False, size="small", perturb=0.02):
    """Returns dict(mesh, xy, curved, u_inf, U, av, name)."""
    rng = np.random.default_rng(seed)
    if kind == "vortex":
        n = {"tiny": 3, "small": 6, "config": 16}.get(size, size) if isinstance(size, str) else size
        m = meshes.periodic_square(n, length=10.0, seed=1000 + seed)
        xy = meshes.straight_nodes(m.verts, r, s)
        curved = np.zeros(m.K, bool)
        ui = states.freestream(0.5, 45.0)
        U = states.vortex_state(xy, period=(10.0, 10.0))
    elif kind in ("naca", "cyl"):
        if kind == "naca":
            nt, nr = {"tiny": (12, 2), "small": (40, 5), "config": (300, 100)}[size]
            m = meshes.naca_omesh(n_t=nt, n_r=nr, seed=1001 + seed)
            ui = states.freestream(0.8, 1.25)
        else:
            nt, nr = {"tiny": (12, 2), "small": (32, 5), "config": (500, 250)}[size]
            m = meshes.cylinder_channel(n_t=nt, n_r=nr, seed=1002 + seed)
            ui = states.freestream(0.38, 0.0)
        xy, curved = curving.curve_mesh(m, N, r, s)
        x = xy[..., 0]
        y = xy[..., 1]
        U = states.uniform_state(m.K, len(r), ui)
        # smooth perturbation plus a little noise so that every term is exercised
        U[:, 0] *= 1.0 + perturb * np.sin(1.3 * x) * np.cos(0.7 * y)
        U[:, 3] *= 1.0 + perturb * np.cos(0.9 * x + 0.4 * y)
        U[:, 1] += perturb * np.sin(y)
        U *= 1.0 + 0.1 * perturb * rng.standard_normal(U.shape)
    else:
        raise ValueError(kind)
    return dict(mesh=m, xy=xy, curved=curved, u_inf=ui, U=U, av=av, name=kind, N=N)


# ------------------------------------------------------------------ tetrahedra
def warp_box_nodes(X, L, amp=0.3):
    """Smooth periodic displacement of the box nodes (every element curved)."""
    k = 2 * np.pi / L
    d = amp * np.sin(k * X[..., [0]] + 0.3) * np.sin(k * X[..., [1]]) * np.sin(k * X[..., [2]])
    return X + d * np.array([1.0, 0.5, -0.7])


def make_case3(kind, N, r, s, t, seed=0, size="small", perturb=0.02):
    """Tetrahedral cases.  Returns dict(mesh, xyz, u_inf, U, name, N).
      box   periodic jittered cube (affine), extruded vortex plus noise
      wbox  the same cube with a smooth periodic warp (every element curved)
      bump  channel with a curved bump on the floor: slip walls, farfield
            inflow/outflow, uniform flow with smooth perturbations and noise"""
    from paper_1208_4772_gb300.inputs import meshes3d
    rng = np.random.default_rng(seed)
    if kind in ("box", "wbox"):
        n = {"tiny": 2, "small": 3, "medium": 5}.get(size, size) if isinstance(size, str) else size
        L = 10.0
        m = meshes3d.box(n, L=L, seed=1000 + seed)
        X = meshes3d.node_coords(m, r, s, t)
        if kind == "wbox":
            X = warp_box_nodes(X, L)
        ui = states.freestream3(0.5, 10.0)
        U = states.vortex3_state(X, period=(L, L))
        U *= 1.0 + 0.1 * perturb * rng.standard_normal(U.shape)
    elif kind in ("single", "pair"):
        m = minimal_tet_mesh(kind)
        X = meshes3d.node_coords(m, r, s, t)
        ui = states.freestream3(0.5, 10.0)
        U = states.uniform_state3(m.K, len(r), ui)
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        U[:, 0] *= 1.0 + perturb * np.sin(2.1 * x + y) * np.cos(1.7 * z)
        U[:, 4] *= 1.0 + perturb * np.cos(1.9 * y - z)
        U[:, 3] += perturb * np.sin(3 * x)
        U *= 1.0 + 0.1 * perturb * rng.standard_normal(U.shape)
    elif kind == "bump":
        if size == "config":     # the 300,000-tetrahedron bump channel of the benchmark
            m = meshes3d.bump_channel(50, 25, 40, Zd=0.4, seed=2000 + seed)
        else:
            nx, ny, nz = {"tiny": (4, 2, 2), "small": (6, 3, 4), "medium": (12, 6, 8)}[size]
            m = meshes3d.bump_channel(nx, ny, nz, seed=2000 + seed)
        X = meshes3d.node_coords(m, r, s, t)
        ui = states.freestream3(0.5, 0.0)
        U = states.uniform_state3(m.K, len(r), ui)
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        U[:, 0] *= 1.0 + perturb * np.sin(1.3 * x) * np.cos(0.7 * y + z)
        U[:, 4] *= 1.0 + perturb * np.cos(0.9 * x + 0.4 * y)
        U[:, 2] += perturb * np.sin(2 * z)
        U[:, 3] += perturb * np.cos(x + y)
        U *= 1.0 + 0.1 * perturb * rng.standard_normal(U.shape)
    else:
        raise ValueError(kind)
    return dict(mesh=m, xyz=X, u_inf=ui, U=U, name=kind, N=N)


def minimal_tet_mesh(kind):
    """One tetrahedron ("single"), or two sharing one face with their vertices
    numbered in different orders ("pair"); faces 0 and 1 of each element are
    slip walls, the other outer faces farfield."""
    from paper_1208_4772_gb300.inputs import meshes3d
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 1.1, 0.1], [0.1, 0.2, 0.9], [1.0, 1.0, 1.0]])
    EToV = np.array([[0, 1, 2, 3]] if kind == "single" else [[0, 1, 2, 3], [4, 3, 2, 1]])
    for k in range(len(EToV)):       # positive orientation
        v = P[EToV[k]]
        if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]])) < 0:
            EToV[k, [1, 2]] = EToV[k, [2, 1]]
    bc = np.zeros((len(EToV), 4), dtype=np.int8)
    sets = [[frozenset(EToV[k, list(f)]) for f in meshes3d.FACES] for k in range(len(EToV))]
    count = {}
    for row in sets:
        for f in row:
            count[f] = count.get(f, 0) + 1
    for k, row in enumerate(sets):
        for j, f in enumerate(row):
            bc[k, j] = 0 if count[f] == 2 else (1 if j < 2 else 2)
    return meshes3d.TetMesh(kind, P[EToV], EToV, bc)


def rel_l2_per_var5(a, b):
    nv = a.shape[1]
    return np.linalg.norm((a - b).transpose(1, 0, 2).reshape(nv, -1), axis=1) / \
        np.linalg.norm(b.transpose(1, 0, 2).reshape(nv, -1), axis=1)

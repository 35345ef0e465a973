"""Initial and reference states on the collocation nodes (inputs only).

* freestream(M, aoa): rho = 1, p = 1/gamma (so c = 1), velocity M (cos a, sin a);
* isentropic vortex (strength beta = 5, gamma = 1.4): about centre (xc, yc)
  moving with the mean flow (u0, v0),
      r^2 = (x - xc - u0 t)^2 + (y - yc - v0 t)^2,
      du = -beta/(2 pi) exp((1 - r^2)/2) (y - yc - v0 t),
      dv = +beta/(2 pi) exp((1 - r^2)/2) (x - xc - u0 t),
      T  = 1 - (gamma - 1) beta^2 / (8 gamma pi^2) exp(1 - r^2),
      rho = T^(1/(gamma-1)), p = rho^gamma,
  which the Euler equations carry unchanged with the mean flow.  On a
  periodic box the centre is taken at its nearest periodic image;
* the time step rule used by the workloads,
      dt = CFL h_min / ((N+1)^2 max(|u| + c)),
  h_k = 2 area / perimeter (the inradius); with artificial viscosity also
      dt <= 0.5 CFL h_min^2 / ((N+1)^4 eps0).
  The rule is an input to both sides of every parity check.
"""
import numpy as np


def conserved(rho, u, v, p, gamma=1.4):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-2)


def freestream(mach, aoa_deg=0.0, gamma=1.4):
    a = np.deg2rad(aoa_deg)
    rho, p = 1.0, 1.0 / gamma
    u, v = mach * np.cos(a), mach * np.sin(a)
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def vortex(x, y, t=0.0, beta=5.0, gamma=1.4, center=(5.0, 5.0), mean=(1.0, 1.0), period=None):
    xc = center[0] + mean[0] * t
    yc = center[1] + mean[1] * t
    dx, dy = x - xc, y - yc
    if period is not None:
        Lx, Ly = period
        dx = dx - Lx * np.round(dx / Lx)
        dy = dy - Ly * np.round(dy / Ly)
    r2 = dx * dx + dy * dy
    e = np.exp(0.5 * (1.0 - r2))
    u = mean[0] - beta / (2 * np.pi) * e * dy
    v = mean[1] + beta / (2 * np.pi) * e * dx
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8 * gamma * np.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return conserved(rho, u, v, p, gamma)


def vortex_state(node_xy, t=0.0, **kw):
    """U [K, 4, Np] at the nodes."""
    return vortex(node_xy[..., 0], node_xy[..., 1], t, **kw)


def uniform_state(K, Np, u_inf):
    return np.broadcast_to(np.asarray(u_inf, dtype=np.float64)[None, :, None], (K, 4, Np)).copy()


def inradius(verts):
    a = np.linalg.norm(verts[:, 1] - verts[:, 0], axis=-1)
    b = np.linalg.norm(verts[:, 2] - verts[:, 1], axis=-1)
    c = np.linalg.norm(verts[:, 0] - verts[:, 2], axis=-1)
    e1, e2 = verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0]
    area = 0.5 * np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    return 2.0 * area / (a + b + c)


def max_wave_speed(U, gamma=1.4):
    rho = U[:, 0]
    u, v = U[:, 1] / rho, U[:, 2] / rho
    p = (gamma - 1.0) * (U[:, 3] - 0.5 * rho * (u * u + v * v))
    return float(np.max(np.sqrt(u * u + v * v) + np.sqrt(gamma * p / rho)))


def time_step(verts, U, N, cfl=0.3, gamma=1.4, eps0=None):
    h = float(np.min(inradius(verts)))
    dt = cfl * h / ((N + 1) ** 2 * max_wave_speed(U, gamma))
    if eps0:
        dt = min(dt, 0.5 * cfl * h * h / ((N + 1) ** 4 * eps0))
    return dt


# ------------------------------------------------------------------ 3D
# Five conserved variables (rho, rho u, rho v, rho w, E).  The extruded
# isentropic vortex (the 2D vortex above with w = 0, independent of z) is an
# exact solution of the 3D Euler equations.

def conserved3(rho, u, v, w, p, gamma=1.4):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=-2)


def freestream3(mach, aoa_deg=0.0, gamma=1.4):
    """rho = 1, p = 1/gamma, velocity M (cos a, 0, sin a) (angle in the x-z plane)."""
    a = np.deg2rad(aoa_deg)
    u, w = mach * np.cos(a), mach * np.sin(a)
    p = 1.0 / gamma
    return np.array([1.0, u, 0.0, w, p / (gamma - 1.0) + 0.5 * (u * u + w * w)])


def vortex3_state(node_xyz, t=0.0, **kw):
    """U [K, 5, Np]: the 2D isentropic vortex in (x, y), w = 0."""
    U2 = vortex(node_xyz[..., 0], node_xyz[..., 1], t, **kw)
    out = np.zeros(U2.shape[:-2] + (5,) + U2.shape[-1:])
    out[..., 0, :], out[..., 1, :], out[..., 2, :], out[..., 4, :] = U2[..., 0, :], U2[..., 1, :], U2[..., 2, :], U2[..., 3, :]
    return out


def uniform_state3(K, Np, u_inf):
    return np.broadcast_to(np.asarray(u_inf, dtype=np.float64)[None, :, None], (K, 5, Np)).copy()


def inradius3(verts):
    """3 volume / surface area of each tetrahedron [K, 4, 3]."""
    e1, e2, e3 = verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0], verts[:, 3] - verts[:, 0]
    vol = np.abs(np.einsum('ki,ki->k', np.cross(e1, e2), e3)) / 6.0
    area = 0.0
    for (a, b, c) in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
        area = area + 0.5 * np.linalg.norm(np.cross(verts[:, b] - verts[:, a], verts[:, c] - verts[:, a]), axis=1)
    return 3.0 * vol / area


def time_step3(verts, U, N, cfl=0.3, gamma=1.4, eps0=None):
    """dt = CFL h_min / ((N+1)^2 max(|u| + c)) with h the inradius; with
    artificial viscosity up to eps0 also at most CFL h_min^2 / (2 (N+1)^4
    eps0), the limit of the triangle path."""
    rho = U[:, 0]
    vel2 = (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / rho ** 2
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * vel2)
    smax = float(np.max(np.sqrt(vel2) + np.sqrt(gamma * p / rho)))
    h = float(np.min(inradius3(verts)))
    dt = cfl * h / ((N + 1) ** 2 * smax)
    if eps0:
        dt = min(dt, 0.5 * cfl * h * h / ((N + 1) ** 4 * eps0))
    return dt

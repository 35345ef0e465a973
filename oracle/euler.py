"""2D Euler system (paper Sec. 5, with the z-momentum dropped) and the
approximate Riemann solver of Sec. 2.

U = (rho, rho u, rho v, E).  The paper prints the pressure as
(gamma-1)(rho E - (u^2+v^2+w^2)/(2 rho)); the dimensionally consistent
reading used here is p = (gamma-1)(E - |m|^2/(2 rho)) with m = rho u.

Numerical flux (Sec. 2 names local Lax-Friedrichs): for the outward unit
normal n,
  F*.n = 1/2 (F(U-).n + F(U+).n) - 1/2 lam (U+ - U-),
  lam  = max(|u-.n| + c-, |u+.n| + c+) evaluated pointwise, c = sqrt(gamma p/rho).

Boundary ghost states (the paper does not state them):
  slip wall  U+ = (rho, m - 2 (m.n) n, E);
  farfield   U+ = U_inf.

Test infrastructure only.
"""
import numpy as np


def pressure(U, gamma):
    rho, mx, my, E = U[..., 0, :], U[..., 1, :], U[..., 2, :], U[..., 3, :]
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)


def flux(U, gamma):
    """Cartesian fluxes F (x) and G (y); U has the variable axis at -2."""
    rho, mx, my, E = U[..., 0, :], U[..., 1, :], U[..., 2, :], U[..., 3, :]
    u, v = mx / rho, my / rho
    p = pressure(U, gamma)
    F = np.stack([mx, mx * u + p, my * u, u * (E + p)], axis=-2)
    G = np.stack([my, mx * v, my * v + p, v * (E + p)], axis=-2)
    return F, G


def llf(Um, Up, nx, ny, gamma):
    """F*.n for states with the variable axis at -2 and normals broadcastable
    to the remaining axes."""
    Fm, Gm = flux(Um, gamma)
    Fp, Gp = flux(Up, gamma)
    n_x, n_y = nx[..., None, :], ny[..., None, :]
    fn_m = Fm * n_x + Gm * n_y
    fn_p = Fp * n_x + Gp * n_y

    def wave_speed(U):
        rho = U[..., 0, :]
        un = (U[..., 1, :] * nx + U[..., 2, :] * ny) / rho
        c = np.sqrt(gamma * pressure(U, gamma) / rho)
        return np.abs(un) + c

    lam = np.maximum(wave_speed(Um), wave_speed(Up))
    return 0.5 * (fn_m + fn_p) - 0.5 * lam[..., None, :] * (Up - Um)


def wall_ghost(Um, nx, ny):
    mn = Um[..., 1, :] * nx + Um[..., 2, :] * ny
    Up = Um.copy()
    Up[..., 1, :] = Um[..., 1, :] - 2.0 * mn * nx
    Up[..., 2, :] = Um[..., 2, :] - 2.0 * mn * ny
    return Up

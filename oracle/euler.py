"""2D Euler system (paper Sec. 5, with the z-momentum dropped) and the
approximate Riemann solver of Sec. 2.

U = (rho, rho u, rho v, E).  The paper prints the pressure as
(gamma-1)(rho E - (u^2+v^2+w^2)/(2 rho)); the dimensionally consistent
reading used here is p = (gamma-1)(E - |m|^2/(2 rho)) with m = rho u.

Numerical flux (Sec. 2 names local Lax-Friedrichs): for the outward unit
normal n,
  F*.n = 1/2 (F(U-).n + F(U+).n) - 1/2 lam (U+ - U-),
  lam  = max(|u-.n| + c-, |u+.n| + c+) evaluated pointwise, c = sqrt(gamma p/rho).

HLLC (the alternative the paper names) is `hllc` below.

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


def hllc(Um, Up, nx, ny, gamma):
    """The HLLC numerical flux (Sec. 2 names it as the alternative to LLF),
    along the normal n, after Toro, Spruce and Speares: Davis wave-speed
    estimates S_L = min(u_n- - c-, u_n+ - c+), S_R = max(u_n- + c-, u_n+ + c+),
    contact speed
        S_M = (p+ - p- + rho- u_n- (S_L - u_n-) - rho+ u_n+ (S_R - u_n+))
              / (rho- (S_L - u_n-) - rho+ (S_R - u_n+)),
    star states U*_K = rho_K (S_K - u_nK)/(S_K - S_M) (1, u_K + (S_M - u_nK) n,
    E_K/rho_K + (S_M - u_nK)(S_M + p_K / (rho_K (S_K - u_nK)))), and
        F* = F- if 0 <= S_L;  F- + S_L (U*- - U-) if S_L <= 0 <= S_M;
             F+ + S_R (U*+ - U+) if S_M <= 0 <= S_R;  F+ if S_R <= 0,
    with F+- = F(U+-).n.  Shapes as in llf."""
    Fm, Gm = flux(Um, gamma)
    Fp, Gp = flux(Up, gamma)
    n_x, n_y = nx[..., None, :], ny[..., None, :]
    fm = Fm * n_x + Gm * n_y
    fp = Fp * n_x + Gp * n_y

    def prim(U):
        rho = U[..., 0, :]
        u, v = U[..., 1, :] / rho, U[..., 2, :] / rho
        p = pressure(U, gamma)
        return rho, u, v, u * nx + v * ny, p, np.sqrt(gamma * p / rho)

    rl, ul, vl, unl, pl, cl = prim(Um)
    rr, ur, vr, unr, pr, cr = prim(Up)
    SL = np.minimum(unl - cl, unr - cr)
    SR = np.maximum(unl + cl, unr + cr)
    SM = (pr - pl + rl * unl * (SL - unl) - rr * unr * (SR - unr)) / (rl * (SL - unl) - rr * (SR - unr))

    def star(U, rho, u, v, un, p, S):
        f = rho * (S - un) / (S - SM)
        return np.stack([f, f * (u + (SM - un) * nx), f * (v + (SM - un) * ny),
                         f * (U[..., 3, :] / rho + (SM - un) * (SM + p / (rho * (S - un))))], axis=-2)

    Fsl = fm + SL[..., None, :] * (star(Um, rl, ul, vl, unl, pl, SL) - Um)
    Fsr = fp + SR[..., None, :] * (star(Up, rr, ur, vr, unr, pr, SR) - Up)
    return np.where((SL >= 0)[..., None, :], fm,
                    np.where((SM >= 0)[..., None, :], Fsl, np.where((SR > 0)[..., None, :], Fsr, fp)))


def wall_ghost(Um, nx, ny):
    mn = Um[..., 1, :] * nx + Um[..., 2, :] * ny
    Up = Um.copy()
    Up[..., 1, :] = Um[..., 1, :] - 2.0 * mn * nx
    Up[..., 2, :] = Um[..., 2, :] - 2.0 * mn * ny
    return Up

"""3D Euler system (paper Sec. 5) and the numerical fluxes of Sec. 2 for the
tetrahedral form of the method.

U = (rho, rho u, rho v, rho w, E), p = (gamma-1)(E - |m|^2/(2 rho)) (the
dimensionally consistent reading of the printed pressure).

Local Lax-Friedrichs, for the outward unit normal n:
  F*.n = 1/2 (F(U-).n + F(U+).n) - 1/2 lam (U+ - U-),
  lam  = max(|u-.n| + c-, |u+.n| + c+) pointwise.
HLLC (Toro, Spruce and Speares, Davis wave speeds), as in 2D with the
tangential velocity a 2-vector.
Ghost states: slip wall (rho, m - 2 (m.n) n, E); farfield U_inf.

Test infrastructure only.
"""
import numpy as np


def pressure(U, gamma):
    rho, mx, my, mz, E = (U[..., v, :] for v in range(5))
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)


def flux(U, gamma):
    """Cartesian fluxes (F, G, H); U has the variable axis at -2."""
    rho, mx, my, mz, E = (U[..., v, :] for v in range(5))
    u, v, w = mx / rho, my / rho, mz / rho
    p = pressure(U, gamma)
    F = np.stack([mx, mx * u + p, my * u, mz * u, u * (E + p)], axis=-2)
    G = np.stack([my, mx * v, my * v + p, mz * v, v * (E + p)], axis=-2)
    H = np.stack([mz, mx * w, my * w, mz * w + p, w * (E + p)], axis=-2)
    return F, G, H


def normal_flux(U, nx, ny, nz, gamma):
    F, G, H = flux(U, gamma)
    return F * nx[..., None, :] + G * ny[..., None, :] + H * nz[..., None, :]


def llf(Um, Up, nx, ny, nz, gamma):
    fm = normal_flux(Um, nx, ny, nz, gamma)
    fp = normal_flux(Up, nx, ny, nz, gamma)

    def speed(U):
        rho = U[..., 0, :]
        un = (U[..., 1, :] * nx + U[..., 2, :] * ny + U[..., 3, :] * nz) / rho
        return np.abs(un) + np.sqrt(gamma * pressure(U, gamma) / rho)

    lam = np.maximum(speed(Um), speed(Up))
    return 0.5 * (fm + fp) - 0.5 * lam[..., None, :] * (Up - Um)


def hllc(Um, Up, nx, ny, nz, gamma):
    """HLLC: S_L = min(un- - c-, un+ - c+), S_R = max(un- + c-, un+ + c+),
    S_M from the momentum balance, star states
    U*_K = rho_K (S_K - un_K)/(S_K - S_M) (1, u_K + (S_M - un_K) n,
           E_K/rho_K + (S_M - un_K)(S_M + p_K/(rho_K (S_K - un_K))))."""
    fm = normal_flux(Um, nx, ny, nz, gamma)
    fp = normal_flux(Up, nx, ny, nz, gamma)

    def prim(U):
        rho = U[..., 0, :]
        vel = [U[..., 1 + d, :] / rho for d in range(3)]
        p = pressure(U, gamma)
        un = vel[0] * nx + vel[1] * ny + vel[2] * nz
        return rho, vel, un, p, np.sqrt(gamma * p / rho)

    rl, vl, unl, pl, cl = prim(Um)
    rr, vr, unr, pr, cr = prim(Up)
    SL = np.minimum(unl - cl, unr - cr)
    SR = np.maximum(unl + cl, unr + cr)
    SM = (pr - pl + rl * unl * (SL - unl) - rr * unr * (SR - unr)) / (rl * (SL - unl) - rr * (SR - unr))

    def star(U, rho, vel, un, p, S):
        fac = rho * (S - un) / (S - SM)
        E = U[..., 4, :]
        n = (nx, ny, nz)
        comps = [fac] + [fac * (vel[d] + (SM - un) * n[d]) for d in range(3)]
        comps.append(fac * (E / rho + (SM - un) * (SM + p / (rho * (S - un)))))
        return np.stack(comps, axis=-2)

    Fl = fm + SL[..., None, :] * (star(Um, rl, vl, unl, pl, SL) - Um)
    Fr = fp + SR[..., None, :] * (star(Up, rr, vr, unr, pr, SR) - Up)
    out = np.where((SL >= 0.0)[..., None, :], fm,
                   np.where((SM >= 0.0)[..., None, :], Fl,
                            np.where((SR > 0.0)[..., None, :], Fr, fp)))
    return out


def wall_ghost(U, nx, ny, nz):
    """Mirror state of a slip wall; U [..., 5, n], normals [..., n]."""
    out = U.copy()
    mn = U[..., 1, :] * nx + U[..., 2, :] * ny + U[..., 3, :] * nz
    out[..., 1, :] = U[..., 1, :] - 2.0 * mn * nx
    out[..., 2, :] = U[..., 2, :] - 2.0 * mn * ny
    out[..., 3, :] = U[..., 3, :] - 2.0 * mn * nz
    return out

"""Isoparametric element geometry (paper Sec. 2 change of variables with
D Psi and J = |det D Psi|; Sec. 3: the curved map lives in the same Lagrange
basis as the solution, so only the collocation-node coordinates are needed).

For element k with node coordinates (x_j, y_j), x(r,s) = sum_j x_j l_j(r,s):
  at cubature nodes  x_r = D_r x, x_s = D_s x, y_r, y_s,
                     J = x_r y_s - x_s y_r,
                     r_x = y_s/J, r_y = -x_s/J, s_x = -y_r/J, s_y = x_r/J;
  at face f points   (x_t, y_t) = (dr/dt) (x_r, y_r) + (ds/dt) (x_s, y_s),
                     sJ = |(x_t, y_t)|, outward n = (y_t, -x_t) / sJ
                     (elements are counter-clockwise).
A non-positive J anywhere is an error.

Test infrastructure only.
"""
import numpy as np


class ElementGeometry:
    """Geometric factors for a set of elements (arrays lead with element)."""

    def __init__(self, ref, node_xy):
        x = node_xy[..., 0]
        y = node_xy[..., 1]
        xr, xs = x @ ref.Dr.T, x @ ref.Ds.T
        yr, ys = y @ ref.Dr.T, y @ ref.Ds.T
        J = xr * ys - xs * yr
        if np.any(J <= 0.0):
            raise ValueError("non-positive Jacobian at a cubature node")
        self.J = J
        self.rx, self.ry = ys / J, -xs / J
        self.sx, self.sy = -yr / J, xr / J

        K = node_xy.shape[0]
        self.nx = np.zeros((K, 3, ref.Ng))
        self.ny = np.zeros((K, 3, ref.Ng))
        self.sJ = np.zeros((K, 3, ref.Ng))
        for f in range(3):
            xt = (x @ ref.Drg[f].T) * ref.drdt[f] + (x @ ref.Dsg[f].T) * ref.dsdt[f]
            yt = (y @ ref.Drg[f].T) * ref.drdt[f] + (y @ ref.Dsg[f].T) * ref.dsdt[f]
            sJ = np.sqrt(xt * xt + yt * yt)
            self.sJ[:, f] = sJ
            self.nx[:, f] = yt / sJ
            self.ny[:, f] = -xt / sJ

        # mass matrix, paper eq. (mass): M = I_cub^T diag(J W) I_cub
        WJ = J * ref.wq[None, :]
        self.M = np.einsum('qi,kq,qj->kij', ref.Icub, WJ, ref.Icub)
        # factored once at set-up (paper Sec. 2: LU / Cholesky in an initial
        # step); kept as the explicit inverse obtained from that LU
        self.Minv = np.linalg.inv(self.M)

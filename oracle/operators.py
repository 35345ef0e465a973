"""Reference-element operators (paper Sec. 2).

  V        = [psi_j(r_i)]                        nodal <-> modal, f = V f^
  I_cub    = V_cub V^-1      (N_cub x N_p)        interpolation to cubature
  D_r, D_s = V_r V^-1, V_s V^-1 at cubature      derivative matrices
  I_g^f    = V_g^f V^-1      (N_g x N_p)          interpolation to face f
  D_r^f, D_s^f                                   derivatives at face points
                                                 (for curved face normals)

Test infrastructure only.
"""
import numpy as np

from . import basis, nodes, quadrature


class ReferenceElement:
    def __init__(self, N, q=None):
        self.N = N
        self.Np = basis.n_modes(N)
        self.q = quadrature.default_q(N) if q is None else q
        self.r, self.s = nodes.warp_blend_nodes(N)
        self.V = basis.vandermonde(N, self.r, self.s)
        self.Vinv = np.linalg.inv(self.V)
        self.degrees = basis.mode_degrees(N)

        self.rq, self.sq, self.wq = quadrature.triangle_cubature(self.q)
        self.Nq = len(self.wq)
        Vq = basis.vandermonde(N, self.rq, self.sq)
        Vrq, Vsq = basis.grad_vandermonde(N, self.rq, self.sq)
        self.Vq = Vq
        self.Icub = Vq @ self.Vinv
        self.Dr = Vrq @ self.Vinv
        self.Ds = Vsq @ self.Vinv

        self.tg, self.wg = quadrature.gauss_legendre(self.q)
        self.Ng = len(self.wg)
        fr, fs, self.drdt, self.dsdt = quadrature.face_points(self.tg)
        self.Ig = np.zeros((3, self.Ng, self.Np))
        self.Drg = np.zeros((3, self.Ng, self.Np))
        self.Dsg = np.zeros((3, self.Ng, self.Np))
        for f in range(3):
            self.Ig[f] = basis.vandermonde(N, fr[f], fs[f]) @ self.Vinv
            Vr, Vs = basis.grad_vandermonde(N, fr[f], fs[f])
            self.Drg[f] = Vr @ self.Vinv
            self.Dsg[f] = Vs @ self.Vinv
        self.face_r, self.face_s = fr, fs

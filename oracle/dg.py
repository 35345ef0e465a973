"""Semi-discrete DG right-hand side, artificial viscosity, SSP-RK3, residual.

Paper Sec. 2, eq. (semidiscrete), in 2D:

  dU/dt = M_k^-1 sum_m S_{k,x_m} F_m(U^cub) - M_k^-1 M_dOmega (F*(U^g).n)

with, per element k (quantities at cubature nodes q, face points (f,g)):
  U^cub   = I_cub U
  S_x F + S_y G = D_r^T [W J (r_x F + r_y G)] + D_s^T [W J (s_x F + s_y G)]
                                                       (eq. stiffness)
  M_dOmega (F*.n) = sum_f (I_g^f)^T [w_g sJ (F*.n)]    (eq. face_mass)
  M_k = I_cub^T diag(J W) I_cub, solved by LU         (eq. mass)

U- is this element's trace I_g^f U; U+ is the neighbour's trace on its face
f' at the reversed point index g' = N_g - 1 - g (the neighbour runs the
shared edge the other way), or a ghost state on a boundary face.

Artificial viscosity (Sec. 2, Persson & Peraire): sensor on the density,
  u^ = V^-1 rho,  rho~ keeps the modes of degree <= N-1,
  S_k = int (rho - rho~)^2 / int rho^2   (cubature with J),
  s_k = log10 S_k, s_0 = log10(1/N^4) unless given,
  eps_k = 0 | eps0/2 (1 + sin(pi (s_k - s_0) / (2 kappa))) | eps0
            for s_k < s0-kappa | |s_k-s0| <= kappa | s_k > s0+kappa
  (S_k = 0 or int rho^2 = 0 gives eps_k = 0).
The first-order system U_t + div F - div(sqrt(eps) q) = 0, q = sqrt(eps) grad U
is discretised with central (Bassi-Rebay 1) fluxes; the printed q equation
has a sign / M^-1 slip, read here as
  M q_m = - sum_n S-type product with sqrt(eps) U^cub  (weak derivative)
          + sum_f (I_g^f)^T [w_g sJ n_m (sqrt(eps) U)*],
  (sqrt(eps) U)* = 1/2 (sqrt(eps-) U- + sqrt(eps+) U+),
  (sqrt(eps) q)* = 1/2 (sqrt(eps-) q- + sqrt(eps+) q+),
and on wall / farfield faces eps+ = eps-, U+ = ghost state, q+ = q-.

SSP-RK3 (Shu-Osher form; the paper uses a five-stage low-storage RK4, the
workload fixes SSP-RK3):
  U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
  U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)).

Residual (Sec. 5 checks the residual norm): L(U^n) per variable, infinity
norm and Euclidean norm over all nodal values.

Parity: the Euler right-hand side, mass, sensor, SSP-RK3 and residual are
pinned by tests/test_oracle_*.py (free stream, conservation, LLF symmetries,
vortex convergence order, sensor closed forms, stability polynomial).  The
artificial-viscosity right-hand side (the paper prints no values for it) is
pinned by free stream, conservation and the closed forms of
tests/test_oracle_av_pins.py: the gradient exact on linear states, a
constant viscous flux cancelling, eps = 0 giving the inviscid right-hand
side; the sqrt(eps) weighting of both central fluxes where eps jumps across
a face by the discrete divergence identities of
tests/test_oracle_br1_jump.py.

Test infrastructure only.
"""
import numpy as np

from . import euler
from .geometry import ElementGeometry
from .operators import ReferenceElement

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


class Oracle:
    """Plain FP64 evaluation of the method on one mesh.

    EToE, EToF, bc: [K, 3] integer arrays (face f joins element vertices f
    and f+1); node_xy: [K, N_p, 2] collocation-node coordinates in the
    canonical node order; U arrays are [K, 4, N_p].
    """

    def __init__(self, N, EToE, EToF, bc, node_xy, gamma=1.4, u_inf=None,
                 av=False, kappa=4.0, eps0=0.3, s0=None, q=None, flux="llf"):
        self.ref = ReferenceElement(N, q)
        self.N = N
        self.EToE = np.asarray(EToE, dtype=np.int64)
        self.EToF = np.asarray(EToF, dtype=np.int64)
        self.bc = np.asarray(bc, dtype=np.int64)
        self.node_xy = np.asarray(node_xy, dtype=np.float64)
        self.K = self.EToE.shape[0]
        self.gamma = float(gamma)
        self.numflux = {"llf": euler.llf, "hllc": euler.hllc}[flux]
        self.u_inf = None if u_inf is None else np.asarray(u_inf, dtype=np.float64)
        self.av = bool(av)
        self.kappa, self.eps0 = float(kappa), float(eps0)
        self.s0 = np.log10(1.0 / N ** 4) if s0 is None else float(s0)
        self._geo_all = None
        ref = self.ref
        self._IgT = ref.Ig.reshape(3 * ref.Ng, ref.Np).T          # [Np, 3Ng]

    # ------------------------------------------------------------ helpers
    def geometry(self, idx):
        if idx is None or len(idx) == self.K and np.all(idx == np.arange(self.K)):
            if self._geo_all is None:
                self._geo_all = ElementGeometry(self.ref, self.node_xy)
            return self._geo_all
        return ElementGeometry(self.ref, self.node_xy[idx])

    def neighbours(self, idx):
        nb = self.EToE[idx].ravel()
        return np.unique(np.concatenate([idx, nb]))

    def _sqrt_eps_faces(self, eps, idx):
        """sqrt(eps) of each element (own, [n]) and of the other side of each
        of its faces ([n, 3]): the neighbour's, or the element's own on a
        boundary face (eps+ = eps- there)."""
        se = np.sqrt(eps[idx])
        sep = np.where(self.bc[idx] == BC_INTERIOR, np.sqrt(eps[self.EToE[idx]]), se[:, None])
        return se, sep

    def traces(self, V):
        """Own traces I_g^f V on all three faces: [n, nv, 3, Ng]."""
        n, nv, _ = V.shape
        return (V @ self._IgT).reshape(n, nv, 3, self.ref.Ng)

    def lift(self, Fs):
        """sum_f (I_g^f)^T Fs_f for Fs [n, nv, 3, Ng] -> [n, nv, Np]."""
        n, nv = Fs.shape[:2]
        return Fs.reshape(n, nv, -1) @ self._IgT.T

    def _ghost(self, Um, bc, nx, ny):
        """Exterior state on boundary faces; Um [n,4,3,Ng], bc [n,3]."""
        Up = Um.transpose(0, 2, 1, 3).copy()          # [n,3,4,Ng]
        wall = bc == BC_WALL
        if np.any(wall):
            Up[wall] = euler.wall_ghost(Up[wall], nx[wall], ny[wall])
        far = bc == BC_FARFIELD
        if np.any(far):
            Up[far] = self.u_inf[None, :, None]
        return Up.transpose(0, 2, 1, 3)

    def _exterior(self, V, idx, own_traces, bc_fill):
        """Neighbour traces of field V ([K, nv, Np]) on the faces of elements
        idx, taken on the neighbour's face f' and reversed along the shared
        edge; boundary faces take bc_fill(own_traces)."""
        ref = self.ref
        nb = self.EToE[idx]                                   # [n,3]
        fn = self.EToF[idx]
        T = np.matmul(V[nb], ref.Ig[fn].transpose(0, 1, 3, 2))  # [n,3,nv,Ng]
        out = np.ascontiguousarray(T[..., ::-1].transpose(0, 2, 1, 3))
        bnd = self.bc[idx] != BC_INTERIOR
        if np.any(bnd):
            out = np.where(bnd[:, None, :, None], bc_fill(own_traces), out)
        return out

    # ------------------------------------------------------------ sensor
    def sensor(self, U, idx=None):
        """Persson-Peraire viscosity eps_k for elements idx (Sec. 2)."""
        idx = np.arange(self.K) if idx is None else np.asarray(idx)
        ref = self.ref
        geo = self.geometry(idx)
        rho = U[idx, 0, :]
        modal = rho @ ref.Vinv.T
        low = np.where(ref.degrees[None, :] <= self.N - 1, modal, 0.0)
        rho_low = low @ ref.V.T
        WJ = geo.J * ref.wq[None, :]
        num = np.sum(WJ * ((rho - rho_low) @ ref.Icub.T) ** 2, axis=1)
        den = np.sum(WJ * (rho @ ref.Icub.T) ** 2, axis=1)
        eps = np.zeros(len(idx))
        ok = (num > 0.0) & (den > 0.0)
        s = np.full(len(idx), -np.inf)
        s[ok] = np.log10(num[ok] / den[ok])
        lo, hi = self.s0 - self.kappa, self.s0 + self.kappa
        mid = ok & (s >= lo) & (s <= hi)
        eps[mid] = 0.5 * self.eps0 * (1.0 + np.sin(np.pi * (s[mid] - self.s0) / (2.0 * self.kappa)))
        eps[ok & (s > hi)] = self.eps0
        return eps

    # ------------------------------------------------------------ AV q
    def gradient_q(self, U, eps, idx):
        """q = sqrt(eps) grad U by the DG weak form for elements idx.
        eps: array over all elements (only idx and neighbours are read).
        Returns q [n, 2, 4, Np] (m = x, y)."""
        ref = self.ref
        geo = self.geometry(idx)
        se, sep = self._sqrt_eps_faces(eps, idx)
        Ui = U[idx]
        Uc = (Ui @ ref.Icub.T) * se[:, None, None]
        WJ = (ref.wq[None, :] * geo.J)[:, None, :]
        Um = self.traces(Ui)
        nx, ny = geo.nx, geo.ny
        bci = self.bc[idx]
        Up = self._exterior(U, idx, Um, lambda T: self._ghost(T, bci, nx, ny))
        ustar = 0.5 * (se[:, None, None, None] * Um + sep[:, None, :, None] * Up)
        wsJ = (ref.wg[None, None, :] * geo.sJ)[:, None]
        q = np.zeros((len(idx), 2, 4, ref.Np))
        for m, (dr, ds, nm) in enumerate(((geo.rx, geo.sx, nx), (geo.ry, geo.sy, ny))):
            vol = (WJ * dr[:, None, :] * Uc) @ ref.Dr + (WJ * ds[:, None, :] * Uc) @ ref.Ds
            surf = self.lift(wsJ * nm[:, None] * ustar)
            q[:, m] = (-vol + surf) @ geo.Minv.transpose(0, 2, 1)
        return q

    # ------------------------------------------------------------ RHS
    def rhs(self, U, idx=None, eps=None, q=None, parts=False):
        """L(U) on elements idx (all by default).  With AV on, eps and q are
        computed on the neighbourhood that idx needs unless given over all
        elements.  parts=True also returns (vol, surf) before M^-1."""
        idx = np.arange(self.K) if idx is None else np.asarray(idx)
        ref = self.ref
        U = np.asarray(U, dtype=np.float64)
        g = self.gamma
        geo = self.geometry(idx)
        Ui = U[idx]
        Uc = Ui @ ref.Icub.T                                   # U^cub = I_cub U
        F, G = euler.flux(Uc, g)

        if self.av:
            if eps is None or q is None:
                ring1 = self.neighbours(idx)
                ring2 = self.neighbours(ring1)
                eps_full = np.zeros(self.K)
                eps_full[ring2] = self.sensor(U, ring2)
                q_full = np.zeros((self.K, 2, 4, ref.Np))
                q_full[ring1] = self.gradient_q(U, eps_full, ring1)
                eps, q = eps_full, q_full
            se = np.sqrt(eps[idx])
            qc = q[idx] @ ref.Icub.T                           # [n,2,4,Nq]
            F = F - se[:, None, None] * qc[:, 0]
            G = G - se[:, None, None] * qc[:, 1]

        WJ = (ref.wq[None, :] * geo.J)[:, None, :]
        Ft = WJ * (geo.rx[:, None, :] * F + geo.ry[:, None, :] * G)
        Gt = WJ * (geo.sx[:, None, :] * F + geo.sy[:, None, :] * G)
        vol = Ft @ ref.Dr + Gt @ ref.Ds                        # D_r^T Ft + D_s^T Gt

        Um = self.traces(Ui)
        nx, ny = geo.nx, geo.ny
        bci = self.bc[idx]
        Up = self._exterior(U, idx, Um, lambda T: self._ghost(T, bci, nx, ny))
        Fs = self.numflux(Um.transpose(0, 2, 1, 3), Up.transpose(0, 2, 1, 3), nx, ny, g)
        Fs = Fs.transpose(0, 2, 1, 3)                          # [n,4,3,Ng]
        if self.av:
            n = len(idx)
            qm = self.traces(q[idx].reshape(n, 8, ref.Np))
            qp = self._exterior(q.reshape(self.K, 8, ref.Np), idx, qm, lambda T: T)
            qm = qm.reshape(n, 2, 4, 3, ref.Ng)
            qp = qp.reshape(n, 2, 4, 3, ref.Ng)
            se, sep = self._sqrt_eps_faces(eps, idx)
            qn_m = qm[:, 0] * nx[:, None] + qm[:, 1] * ny[:, None]
            qn_p = qp[:, 0] * nx[:, None] + qp[:, 1] * ny[:, None]
            Fs = Fs - 0.5 * (se[:, None, None, None] * qn_m + sep[:, None, :, None] * qn_p)
        surf = self.lift((ref.wg[None, None, :] * geo.sJ)[:, None] * Fs)
        L = (vol - surf) @ geo.Minv.transpose(0, 2, 1)          # M_k^-1 (vol - surf)
        if parts:
            return L, vol, surf
        return L

    # ------------------------------------------------------------ time
    def ssp_rk3_step(self, U, dt):
        U1 = U + dt * self.rhs(U)
        U2 = 0.75 * U + 0.25 * (U1 + dt * self.rhs(U1))
        return U / 3.0 + 2.0 / 3.0 * (U2 + dt * self.rhs(U2))

    # The paper's integrator (Sec. 2): Carpenter and Kennedy's five-stage,
    # fourth-order Runge-Kutta in 2N storage (NASA TM 109112, 1994, the
    # (5,4) coefficient set).  For i = 1..5:
    #     dU <- A_i dU + dt L(U),   U <- U + B_i dU,   with A_1 = 0.
    LSERK_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
    LSERK_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
               2277821191437.0 / 14882151754819.0)

    def lserk54_step(self, U, dt):
        dU = np.zeros_like(U)
        for a, b in zip(self.LSERK_A, self.LSERK_B):
            dU = a * dU + dt * self.rhs(U)
            U = U + b * dU
        return U

    def residual(self, U):
        L = self.rhs(U)
        linf = np.max(np.abs(L), axis=(0, 2))
        l2 = np.sqrt(np.sum(L * L, axis=(0, 2)))
        return linf, l2

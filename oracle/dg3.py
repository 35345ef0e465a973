"""The method on tetrahedra (paper Sec. 2 as printed, d = 3): semi-discrete
DG right-hand side for the 3D Euler equations on isoparametric curved
elements, SSP-RK3 and the five-stage low-storage RK, residual norms.

Per element k (cubature points q, face f with face-rule points g):
  U^cub = I_cub U
  vol   = D_r^T [W J (r_x F + r_y G + r_z H)] + D_s^T [...] + D_t^T [...]
  surf  = sum_f (I_g^f)^T [w_g sJ (F*.n)]
  L(U)  = M_k^-1 (vol - surf),  M_k = I_cub^T diag(J W) I_cub
with (r_x, ...) the inverse of the Jacobian matrix of the isoparametric map
at each cubature point, and at each face point the outward normal and area
factor from the cross product of the physical tangents of the face.

U- is this element's polynomial at the face points; U+ is the neighbour's
polynomial at the same physical points: the face rule sits in the face's
canonical frame (vertices ordered by global number, oracle/tet.py), so the
point with index g is the same point seen from both sides.  Boundary faces
take the slip-wall or farfield ghost state.

The mesh is given by EToV [K, 4] (global vertex numbers; periodic images
share a number), bc [K, 4] per face (0 interior, 1 slip wall, 2 farfield)
and the collocation-node coordinates node_xyz [K, Np, 3] in the canonical
node order.  States are [K, 5, Np].

With artificial viscosity (av=True) the Persson-Peraire sensor and the BR1
gradient q = sqrt(eps) grad U of the triangle oracle carry over to three
directions (same readings).

Parity: pinned by tests/test_oracle_tet.py (rules, basis, nodes, operators,
geometry identities, free stream, conservation, convergence order on the
extruded isentropic vortex, flux properties, planted mistakes; the sensor's
modal ratio, the gradient exact on linear states, the viscous terms of a
constant viscous flux cancelling).

Test infrastructure only.
"""
import numpy as np

from . import euler3
from .dg import Oracle as _Oracle2
from .tet import FACE_VERTS, PERMS3, ReferenceTet, mode_degrees

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


def connectivity(EToV):
    """Face matching from global vertex numbers.  Returns EToE, EToF (-1 on
    unmatched faces) and the orientation code [K, 4]: the index in PERMS3 of
    the local positions of the face's vertices taken in increasing global
    number."""
    EToV = np.asarray(EToV, dtype=np.int64)
    K = EToV.shape[0]
    EToE = -np.ones((K, 4), dtype=np.int64)
    EToF = -np.ones((K, 4), dtype=np.int64)
    orient = np.zeros((K, 4), dtype=np.int64)
    seen = {}
    for k in range(K):
        for f, fv in enumerate(FACE_VERTS):
            G = [int(EToV[k, v]) for v in fv]
            order = tuple(sorted(range(3), key=lambda p: G[p]))
            orient[k, f] = PERMS3.index(order)
            key = tuple(sorted(G))
            if key in seen:
                k2, f2 = seen.pop(key)
                EToE[k, f], EToF[k, f] = k2, f2
                EToE[k2, f2], EToF[k2, f2] = k, f
            else:
                seen[key] = (k, f)
    return EToE, EToF, orient


class TetGeometry:
    """Geometric factors of a set of elements (arrays lead with element)."""

    def __init__(self, ref, node_xyz, orient):
        X = [node_xyz[..., d] for d in range(3)]                  # [n, Np]
        Dm = (ref.Dr, ref.Ds, ref.Dt)
        Jm = np.stack([np.stack([x @ D.T for D in Dm], axis=-1) for x in X], axis=-2)  # [n,Nq,3,3]
        J = np.linalg.det(Jm)
        if np.any(J <= 0.0):
            raise ValueError("non-positive Jacobian at a cubature point")
        self.J = J
        self.inv = np.linalg.inv(Jm)          # inv[..., a, d] = d r_a / d x_d
        n = node_xyz.shape[0]
        self.nrm = np.zeros((n, 4, ref.Ng, 3))
        self.sJ = np.zeros((n, 4, ref.Ng))
        for f in range(4):
            o = orient[:, f]
            Jf = np.stack([np.stack([np.einsum('ngj,nj->ng', D[f, o], x) for D in (ref.Drg, ref.Dsg, ref.Dtg)],
                                    axis=-1) for x in X], axis=-2)    # [n,Ng,3,3]
            au = Jf @ ref.tan_u[f]
            av = Jf @ ref.tan_v[f]
            nr = np.cross(au, av)
            sJ = np.linalg.norm(nr, axis=-1)
            self.sJ[:, f] = sJ
            self.nrm[:, f] = nr / sJ[..., None]
        WJ = J * ref.wq[None, :]
        self.M = np.einsum('qi,kq,qj->kij', ref.Icub, WJ, ref.Icub)
        self.Minv = np.linalg.inv(self.M)


class Oracle3:
    """Plain FP64 evaluation of the tetrahedral method on one mesh."""

    LSERK_A = _Oracle2.LSERK_A
    LSERK_B = _Oracle2.LSERK_B

    def __init__(self, N, EToV, bc, node_xyz, gamma=1.4, u_inf=None, flux="llf", q=None,
                 av=False, kappa=4.0, eps0=0.3, s0=None):
        self.ref = ReferenceTet(N, q)
        self.av = bool(av)
        self.kappa, self.eps0 = float(kappa), float(eps0)
        self.s0 = np.log10(1.0 / N ** 4) if s0 is None else float(s0)
        self.degrees = mode_degrees(N)
        self.N = N
        self.EToV = np.asarray(EToV, dtype=np.int64)
        self.bc = np.asarray(bc, dtype=np.int64)
        self.node_xyz = np.asarray(node_xyz, dtype=np.float64)
        self.K = self.EToV.shape[0]
        self.gamma = float(gamma)
        self.u_inf = None if u_inf is None else np.asarray(u_inf, dtype=np.float64)
        self.numflux = {"llf": euler3.llf, "hllc": euler3.hllc}[flux]
        self.EToE, self.EToF, self.orient = connectivity(self.EToV)
        matched = self.EToE >= 0
        if np.any(matched != (self.bc == BC_INTERIOR)):
            raise ValueError("bc must mark exactly the unmatched faces as boundary faces")
        self._geo = None

    def geometry(self, idx=None):
        if idx is None:
            if self._geo is None:
                self._geo = TetGeometry(self.ref, self.node_xyz, self.orient)
            return self._geo
        return TetGeometry(self.ref, self.node_xyz[idx], self.orient[idx])

    def _face_interp(self, faces, orient):
        """I_g[f][o] for arrays of faces and orientation codes."""
        return self.ref.Ig[faces, orient]

    def _face_values(self, V, idx):
        """Face-point values of the nodal fields V [K, nv, Np] on both sides
        of every face of the elements idx: (I_g of each own face, own [n,4,
        nv,Ng], neighbour's at the same points [n,4,nv,Ng]; on boundary faces
        the neighbour's are the element's own, for the caller to replace)."""
        n = len(idx)
        fidx = np.arange(4)[None, :].repeat(n, 0)
        Igm = self._face_interp(fidx, self.orient[idx])          # [n,4,Ng,Np]
        Vm = np.einsum('nfgj,nvj->nfvg', Igm, V[idx])
        nb, fn = self.EToE[idx], self.EToF[idx]
        bnd = self.bc[idx] != BC_INTERIOR
        nbs, fns = np.where(bnd, idx[:, None], nb), np.where(bnd, 0, fn)
        Igp = self._face_interp(fns, self.orient[nbs, fns])
        Vp = np.einsum('nfgj,nfvj->nfvg', Igp, V[nbs])
        Vp = np.where(bnd[:, :, None, None], Vm, Vp)
        return Igm, Vm, Vp

    def _ghost(self, Um, Up, idx, geo):
        """Exterior states on boundary faces: slip-wall reflection, farfield."""
        nx, ny, nz = geo.nrm[..., 0], geo.nrm[..., 1], geo.nrm[..., 2]
        Up = Up.copy()
        wall = self.bc[idx] == BC_WALL
        if np.any(wall):
            Up[wall] = euler3.wall_ghost(Um[wall], nx[wall], ny[wall], nz[wall])
        far = self.bc[idx] == BC_FARFIELD
        if np.any(far):
            Up[far] = self.u_inf[None, :, None]
        return Up

    def _sqrt_eps_faces(self, eps, idx):
        """sqrt(eps) of the element (own) and of the face's other side,
        which is the element itself on boundary faces."""
        se = np.sqrt(eps[idx])
        sep = np.where(self.bc[idx] == BC_INTERIOR, np.sqrt(eps[np.maximum(self.EToE[idx], 0)]), se[:, None])
        return se, sep

    def neighbours(self, idx):
        idx = np.asarray(idx)
        nb = self.EToE[idx].ravel()
        return np.unique(np.concatenate([idx, nb[nb >= 0]]))

    # ------------------------------------------------------------ sensor
    def sensor(self, U, idx=None):
        """Persson-Peraire viscosity eps_k (Sec. 2): S_k = the L2 norm of the
        density's highest-degree modes over that of the density, both by the
        cubature rule with J; s_k = log10 S_k; the sine ramp of width kappa
        around s0 up to eps0."""
        idx = np.arange(self.K) if idx is None else np.asarray(idx)
        ref = self.ref
        geo = self.geometry(idx)
        rho = U[idx, 0, :]
        modal = rho @ ref.Vinv.T
        low = np.where(self.degrees[None, :] <= self.N - 1, modal, 0.0)
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
        """q_m = sqrt(eps) dU/dx_m by the DG weak form with central face
        values (BR1) for elements idx: M q_m = -sum_a D_a^T [W J (dr_a/dx_m)
        sqrt(eps) U^cub] + sum_f I_g^T [w_g sJ n_m (sqrt(eps) U)*], with
        (sqrt(eps) U)* the mean of the two sides' and, on boundary faces,
        the ghost state with the element's own eps.  eps over all elements
        (idx and their neighbours are read).  Returns q [n, 3, 5, Np]."""
        ref = self.ref
        idx = np.asarray(idx)
        geo = self.geometry(idx)
        U = np.asarray(U, dtype=np.float64)
        se, sep = self._sqrt_eps_faces(eps, idx)
        Uc = (U[idx] @ ref.Icub.T) * se[:, None, None]
        WJ = (ref.wq[None, :] * geo.J)[:, None, :]
        Igm, Um, Up = self._face_values(U, idx)
        Up = self._ghost(Um, Up, idx, geo)
        ustar = 0.5 * (se[:, None, None, None] * Um + sep[:, :, None, None] * Up)
        wsJ = ref.wg[None, None, :] * geo.sJ
        q = np.zeros((len(idx), 3, 5, ref.Np))
        for m in range(3):
            vol = sum((WJ * geo.inv[:, None, :, a, m] * Uc) @ D for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)))
            surf = np.einsum('nfgj,nfvg->nvj', Igm, (wsJ * geo.nrm[..., m])[:, :, None, :] * ustar)
            q[:, m] = (-vol + surf) @ geo.Minv.transpose(0, 2, 1)
        return q

    def rhs(self, U, idx=None, parts=False, eps=None, q=None):
        """L(U) on elements idx (all by default).  With artificial viscosity
        the physical fluxes lose sqrt(eps) q at the cubature points and the
        numerical flux the mean of the two sides' sqrt(eps) q.n; eps and q
        are computed on the neighbourhood idx needs unless given over all
        elements."""
        ref = self.ref
        idx = np.arange(self.K) if idx is None else np.asarray(idx)
        geo = self.geometry(None if len(idx) == self.K and np.all(idx == np.arange(self.K)) else idx)
        U = np.asarray(U, dtype=np.float64)
        g = self.gamma
        Ui = U[idx]
        Uc = Ui @ ref.Icub.T                                     # [n,5,Nq]
        F, G, H = euler3.flux(Uc, g)
        if self.av:
            if eps is None or q is None:
                ring1 = self.neighbours(idx)
                ring2 = self.neighbours(ring1)
                eps_full = np.zeros(self.K)
                eps_full[ring2] = self.sensor(U, ring2)
                q_full = np.zeros((self.K, 3, 5, ref.Np))
                q_full[ring1] = self.gradient_q(U, eps_full, ring1)
                eps, q = eps_full, q_full
            se = np.sqrt(eps[idx])
            qc = q[idx] @ ref.Icub.T                             # [n,3,5,Nq]
            F = F - se[:, None, None] * qc[:, 0]
            G = G - se[:, None, None] * qc[:, 1]
            H = H - se[:, None, None] * qc[:, 2]
        WJ = (ref.wq[None, :] * geo.J)[:, None, :]
        vol = np.zeros_like(Ui)
        for a, D in enumerate((ref.Dr, ref.Ds, ref.Dt)):
            contra = WJ * (geo.inv[:, None, :, a, 0] * F + geo.inv[:, None, :, a, 1] * G
                           + geo.inv[:, None, :, a, 2] * H)
            vol += contra @ D                                    # D^T [W J (grad r_a . Fvec)]

        Igm, Um, Up = self._face_values(U, idx)                  # [n,4,5,Ng]
        Up = self._ghost(Um, Up, idx, geo)
        nx, ny, nz = geo.nrm[..., 0], geo.nrm[..., 1], geo.nrm[..., 2]
        Fs = self.numflux(Um, Up, nx, ny, nz, g)                 # [n,4,5,Ng]
        if self.av:
            n = len(idx)
            _, qm, qp = self._face_values(q.reshape(self.K, 15, ref.Np), idx)   # q+ = q- on boundary faces
            qm = qm.reshape(n, 4, 3, 5, ref.Ng)
            qp = qp.reshape(n, 4, 3, 5, ref.Ng)
            se, sep = self._sqrt_eps_faces(eps, idx)
            qn_m = sum(qm[:, :, m] * geo.nrm[..., m][:, :, None, :] for m in range(3))
            qn_p = sum(qp[:, :, m] * geo.nrm[..., m][:, :, None, :] for m in range(3))
            Fs = Fs - 0.5 * (se[:, None, None, None] * qn_m + sep[:, :, None, None] * qn_p)
        wsJ = ref.wg[None, None, :] * geo.sJ                      # [n,4,Ng]
        surf = np.einsum('nfgj,nfvg->nvj', Igm, wsJ[:, :, None, :] * Fs)
        L = (vol - surf) @ geo.Minv.transpose(0, 2, 1)
        if parts:
            return L, vol, surf
        return L

    def ssp_rk3_step(self, U, dt):
        U1 = U + dt * self.rhs(U)
        U2 = 0.75 * U + 0.25 * (U1 + dt * self.rhs(U1))
        return U / 3.0 + 2.0 / 3.0 * (U2 + dt * self.rhs(U2))

    def lserk54_step(self, U, dt):
        dU = np.zeros_like(U)
        for a, b in zip(self.LSERK_A, self.LSERK_B):
            dU = a * dU + dt * self.rhs(U)
            U = U + b * dU
        return U

    def residual(self, U):
        L = self.rhs(U)
        return np.max(np.abs(L), axis=(0, 2)), np.sqrt(np.sum(L * L, axis=(0, 2)))

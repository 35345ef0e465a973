// Device helpers shared by the tetrahedral stage kernels (CUDA-core and
// tensor-core volume terms): 16-byte operand loads, the Euler fluxes on a
// face, the stage combination, and the face phases of a tile that both
// kernels run on the CUDA cores (paper Sec. 2 with d = 3).
#pragma once
#include "dg3_device.h"

namespace dgc {
namespace {

// Four consecutive reals by one 16-byte access (two for double).
template <typename Real>
struct V4 {
    Real x, y, z, w;
};
__device__ __forceinline__ V4<float> lds4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> lds4(const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ V4<float> ldg4(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ldg4(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p + 2));
    return {a.x, a.y, b.x, b.y};
}
template <typename Real>
__device__ __forceinline__ Real dot4(const V4<Real>& a, const V4<Real>& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// outward reference face vectors (t_u x t_v of each face's parametrisation)
__device__ __constant__ float kFaceRef[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};

template <typename Real>
__device__ __forceinline__ void normal_flux3(const Real* u, Real nx, Real ny, Real nz, Real gamma, Real* fn,
                                             Real& un, Real& c) {
    const Real ir = recip(u[0]);
    un = (u[1] * nx + u[2] * ny + u[3] * nz) * ir;
    const Real p = (gamma - Real(1)) * (u[4] - Real(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir);
    c = fsqrt(gamma * p * ir);
    fn[0] = u[0] * un;
    fn[1] = u[1] * un + p * nx;
    fn[2] = u[2] * un + p * ny;
    fn[3] = u[3] * un + p * nz;
    fn[4] = (u[4] + p) * un;
}

template <typename Real>
__device__ __forceinline__ void llf3(const Real* um, const Real* up, Real nx, Real ny, Real nz, Real gamma,
                                     Real* F) {
    Real fm[5], fp[5], unm, cm, unp, cp;
    normal_flux3(um, nx, ny, nz, gamma, fm, unm, cm);
    normal_flux3(up, nx, ny, nz, gamma, fp, unp, cp);
    const Real lam = fmax(fabs(unm) + cm, fabs(unp) + cp);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = Real(0.5) * (fm[v] + fp[v]) - Real(0.5) * lam * (up[v] - um[v]);
}

// HLLC (Toro, Spruce and Speares) with Davis wave-speed estimates.
template <typename Real>
__device__ __forceinline__ void hllc3(const Real* um, const Real* up, Real nx, Real ny, Real nz, Real gamma,
                                      Real* F) {
    Real fm[5], fp[5], unl, cl, unr, cr;
    normal_flux3(um, nx, ny, nz, gamma, fm, unl, cl);
    normal_flux3(up, nx, ny, nz, gamma, fp, unr, cr);
    const Real SL = fmin(unl - cl, unr - cr), SR = fmax(unl + cl, unr + cr);
    if (SL >= Real(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] = fm[v];
        return;
    }
    if (SR <= Real(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] = fp[v];
        return;
    }
    const Real rl = um[0], rr = up[0];
    const Real pl = (gamma - Real(1)) * (um[4] - Real(0.5) * (um[1] * um[1] + um[2] * um[2] + um[3] * um[3]) / rl);
    const Real pr = (gamma - Real(1)) * (up[4] - Real(0.5) * (up[1] * up[1] + up[2] * up[2] + up[3] * up[3]) / rr);
    const Real SM = (pr - pl + rl * unl * (SL - unl) - rr * unr * (SR - unr)) / (rl * (SL - unl) - rr * (SR - unr));
    const bool left = SM >= Real(0);
    const Real* u = left ? um : up;
    const Real* f = left ? fm : fp;
    const Real S = left ? SL : SR, un = left ? unl : unr, p = left ? pl : pr, rho = u[0];
    const Real fac = rho * (S - un) / (S - SM);
    const Real ir = Real(1) / rho;
    const Real n[3] = {nx, ny, nz};
    Real us[5];
    us[0] = fac;
#pragma unroll
    for (int d = 0; d < 3; ++d) us[1 + d] = fac * (u[1 + d] * ir + (SM - un) * n[d]);
    us[4] = fac * (u[4] * ir + (SM - un) * (SM + p / (rho * (S - un))));
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = f[v] + S * (us[v] - u[v]);
}

template <typename Real>
__device__ __forceinline__ Real stage_value3(const StageArgs3<Real>& p, long long n, Real us, Real L) {
    if (p.rhs_only) return L;
    if (p.dU) {
        const Real d = (p.a != Real(0) ? p.a * p.dU[n] : Real(0)) + p.dt * L;
        p.dU[n] = d;
        return us + p.b * d;
    }
    return p.a * (p.a != Real(0) ? p.Un[n] : Real(0)) + p.b * (us + p.dt * L);
}


// Cofactors of the affine map (g[3 d + a] = J dr_a / dx_d) and 1/J (g[9])
// from J[3 d + a] = dx_d / dr_a.
template <typename Real>
__device__ __forceinline__ void affine_cofactors3(const Real* J, Real* g) {
    g[0] = J[4] * J[8] - J[5] * J[7];
    g[1] = J[5] * J[6] - J[3] * J[8];
    g[2] = J[3] * J[7] - J[4] * J[6];
    g[3] = J[2] * J[7] - J[1] * J[8];
    g[4] = J[0] * J[8] - J[2] * J[6];
    g[5] = J[1] * J[6] - J[0] * J[7];
    g[6] = J[1] * J[5] - J[2] * J[4];
    g[7] = J[2] * J[3] - J[0] * J[5];
    g[8] = J[0] * J[4] - J[1] * J[3];
    const Real det = J[0] * g[0] + J[1] * g[1] + J[2] * g[2];
    g[9] = Real(1) / det;
}

// Per face-frame point of the tile: U- and U+ from the face nodes by I2 of
// the face's orientation (the neighbour's with its own), ghost states on
// boundary faces, normal and area factor (affine: from the cofactors sG with
// row stride GST; curved: from the record), the numerical flux, stored as
// w_g sJ F* in sFs [e][4][5][NGP].  With Bar (the data of each
// element's mean state: ubar[5], its velocity [3], pressure, total
// enthalpy, BST reals per element) the normal flux of that state is
// subtracted first.  Items start at thread `first`, so that a phase with
// fewer items than threads before it can hand this one its idle threads.
//
// MODE 1 (artificial viscosity) also takes the q face-node rows of both
// sides (sQf, sQnb: [e][4][15][NFPP]) and sqrt(eps) of the element and of
// each face's other side (sSe [e][5]), and subtracts the mean of the two
// sides' sqrt(eps) q.n (q+ = q- and eps+ = eps- on boundary faces).
// MODE 2 (the BR1 gradient, direction gm) replaces the numerical flux by the
// central value n_gm (sqrt(eps) U)*, the exterior state being the ghost on
// boundary faces.
template <int N, typename Real, int GST, int BST, int MODE = 0>
__device__ __forceinline__ void face_points3(const StageArgs3<Real>& p, long long e0, int ne, int first,
                                             const Real* sI2, const Real* sW, const Real* sUf, const Real* sNb,
                                             const int* sCode, const Real* sG, const Real* Bar, Real* sFs,
                                             const Real* sSe = nullptr, const Real* sQf = nullptr,
                                             const Real* sQnb = nullptr, int gm = 0) {
    constexpr int NQ = nq3_of(N), NG = ng3_of(N), NFPP = pad4(nfp3_of(N)), NGP = pad4(NG);
    constexpr int CS = curved3_stride(N);
    for (int i = first; i < ne * 4 * NG; i += THREADS) {
        const int e = i / (4 * NG), r = i - e * 4 * NG, f = r / NG, g = r - f * NG;
        const int code = sCode[e * 4 + f];
        const long long eg = e0 + e;
        const Real* I2o = sI2 + (code3_own(code) * NG + g) * NFPP;
        const Real* uf = sUf + (e * 4 + f) * 5 * NFPP;
        Real um[5] = {0, 0, 0, 0, 0}, up[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int ib = 0; ib < NFPP / 4; ++ib) {
            const V4<Real> w = lds4(I2o + 4 * ib);
#pragma unroll
            for (int v = 0; v < 5; ++v) um[v] += dot4(w, lds4(uf + v * NFPP + 4 * ib));
        }
        Real nx, ny, nz, sJ;
        if (eg < p.Kaff) {
            const Real* c = sG + e * GST;
            const Real a0 = kFaceRef[f][0], a1 = kFaceRef[f][1], a2 = kFaceRef[f][2];
            const Real x = c[0] * a0 + c[1] * a1 + c[2] * a2;
            const Real y = c[3] * a0 + c[4] * a1 + c[5] * a2;
            const Real z = c[6] * a0 + c[7] * a1 + c[8] * a2;
            sJ = sqrt(x * x + y * y + z * z);
            const Real is = Real(1) / sJ;
            nx = x * is; ny = y * is; nz = z * is;
        } else {
            const Real* gf = p.geoC + (eg - p.Kaff) * CS + 9 * NQ + f * NG + g;
            nx = gf[0]; ny = gf[4 * NG]; nz = gf[8 * NG]; sJ = gf[12 * NG];
        }
        const int bc = code3_bc(code);
        if (bc == 0) {
            const Real* I2p = sI2 + (code3_nbr(code) * NG + g) * NFPP;
            const Real* nbv = sNb + (e * 4 + f) * 5 * NFPP;
#pragma unroll
            for (int ib = 0; ib < NFPP / 4; ++ib) {
                const V4<Real> w = lds4(I2p + 4 * ib);
#pragma unroll
                for (int v = 0; v < 5; ++v) up[v] += dot4(w, lds4(nbv + v * NFPP + 4 * ib));
            }
        } else if (bc == 1) {
            const Real mn = um[1] * nx + um[2] * ny + um[3] * nz;
            up[0] = um[0];
            up[1] = um[1] - Real(2) * mn * nx;
            up[2] = um[2] - Real(2) * mn * ny;
            up[3] = um[3] - Real(2) * mn * nz;
            up[4] = um[4];
        } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) up[v] = p.uinf[v];
        }
        Real F[5];
        if constexpr (MODE == 2) {
            const Real se = sSe[e * 5], sp = bc == 0 ? sSe[e * 5 + 1 + f] : se;
            const Real nm = gm == 0 ? nx : gm == 1 ? ny : nz;
#pragma unroll
            for (int v = 0; v < 5; ++v) F[v] = nm * Real(0.5) * (se * um[v] + sp * up[v]);
        } else {
            if (p.flux == 1)
                hllc3(um, up, nx, ny, nz, p.gamma, F);
            else
                llf3(um, up, nx, ny, nz, p.gamma, F);
        }
        if constexpr (MODE == 1) {   // minus the mean of the two sides' sqrt(eps) q.n
            const Real se = sSe[e * 5], sp = bc == 0 ? sSe[e * 5 + 1 + f] : se;
            const Real* qf = sQf + (e * 4 + f) * 15 * NFPP;
            const Real* qn = sQnb + (e * 4 + f) * 15 * NFPP;
            const Real* I2p = sI2 + (code3_nbr(code) * NG + g) * NFPP;
            Real qm[15], qp[15];
#pragma unroll
            for (int r = 0; r < 15; ++r) qm[r] = qp[r] = Real(0);
#pragma unroll
            for (int ib = 0; ib < NFPP / 4; ++ib) {
                const V4<Real> w = lds4(I2o + 4 * ib);
#pragma unroll
                for (int r = 0; r < 15; ++r) qm[r] += dot4(w, lds4(qf + r * NFPP + 4 * ib));
            }
            if (bc == 0) {
#pragma unroll
                for (int ib = 0; ib < NFPP / 4; ++ib) {
                    const V4<Real> w = lds4(I2p + 4 * ib);
#pragma unroll
                    for (int r = 0; r < 15; ++r) qp[r] += dot4(w, lds4(qn + r * NFPP + 4 * ib));
                }
            } else {
#pragma unroll
                for (int r = 0; r < 15; ++r) qp[r] = qm[r];
            }
#pragma unroll
            for (int v = 0; v < 5; ++v)
                F[v] -= Real(0.5) * (se * (nx * qm[v] + ny * qm[5 + v] + nz * qm[10 + v]) +
                                     sp * (nx * qp[v] + ny * qp[5 + v] + nz * qp[10 + v]));
        }
        if (Bar) {   // minus the normal flux of the element's mean state
            const Real* b = Bar + e * BST;
            const Real un = nx * b[5] + ny * b[6] + nz * b[7];
            F[0] -= b[0] * un;
            F[1] -= b[1] * un + b[8] * nx;
            F[2] -= b[2] * un + b[8] * ny;
            F[3] -= b[3] * un + b[8] * nz;
            F[4] -= b[9] * un;
        }
        const Real ws = sW[g] * sJ;
        Real* out = sFs + (e * 4 + f) * 5 * NGP + g;
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v * NGP] = ws * F[v];
    }
}

// Lift of each face's w sJ F* to its face nodes: sT [e][4][5][NFPP] =
// I2_o^T sFs, o the face's own orientation.
template <int N, typename Real>
__device__ __forceinline__ void lift3(int ne, const Real* sI2T, const Real* sFs, const int* sCode, Real* sT) {
    constexpr int NFP = nfp3_of(N), NFPP = pad4(NFP), NGP = pad4(ng3_of(N));
    for (int i = threadIdx.x; i < ne * 4 * NFP; i += THREADS) {
        const int ef = i / NFP, n = i - ef * NFP;   // ef = e * 4 + f
        const Real* I2t = sI2T + (code3_own(sCode[ef]) * NFP + n) * NGP;
        const Real* fs = sFs + ef * 5 * NGP;
        Real t[5] = {0, 0, 0, 0, 0};
#pragma unroll 2
        for (int gb = 0; gb < NGP / 4; ++gb) {
            const V4<Real> w = lds4(I2t + 4 * gb);
#pragma unroll
            for (int v = 0; v < 5; ++v) t[v] += dot4(w, lds4(fs + v * NGP + 4 * gb));
        }
        Real* out = sT + ef * 5 * NFPP + n;
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v * NFPP] = t[v];
    }
}

// R = (sum of the NPARTS volume parts, PSTRIDE reals apart) - the lifted
// face terms gathered to the element nodes, in place in sR [e][5][NP].
template <int N, typename Real, int NPARTS>
__device__ __forceinline__ void combine3(int ne, int pstride, const Real* sT, const int* sFpos, Real* sR) {
    constexpr int NP = np3_of(N), NFPP = pad4(nfp3_of(N));
    for (int i = threadIdx.x; i < ne * 5 * NP; i += THREADS) {
        const int e = i / (5 * NP), r = i - e * 5 * NP, v = r / NP, n = r - v * NP;
        Real acc = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int pos = sFpos[f * NP + n];
            if (pos >= 0) acc += sT[((e * 4 + f) * 5 + v) * NFPP + pos];
        }
        Real vol = sR[i];
#pragma unroll
        for (int k = 1; k < NPARTS; ++k) vol += sR[k * pstride + i];
        sR[i] = vol - acc;
    }
}

// L = M_k^-1 R (affine: M_ref^-1 / J, 1/J at sG[e GST + 9]; curved: the
// record's M_k^-1) and the stage update to global memory.
template <int N, typename Real, int GST>
__device__ __forceinline__ void update3(const StageArgs3<Real>& p, long long e0, int ne, const Real* sR,
                                        const Real* sMiT, const Real* sG, const Real* sU) {
    constexpr int NP = np3_of(N), NPP = pad4(NP), NQ = nq3_of(N), NG = ng3_of(N);
    constexpr int CS = curved3_stride(N);
    for (int i = threadIdx.x; i < ne * 5 * NP; i += THREADS) {
        const int e = i / (5 * NP), r = i - e * 5 * NP, v = r / NP, n = r - v * NP;
        const Real* rr = sR + (e * 5 + v) * NP;
        const long long eg = e0 + e;
        Real Lv = 0;
        if (eg < p.Kaff) {
            for (int j = 0; j < NP; ++j) Lv += sMiT[j * NP + n] * rr[j];
            Lv *= sG[e * GST + 9];
        } else {
            const Real* mi = p.geoC + (eg - p.Kaff) * CS + 9 * NQ + 16 * NG;
            for (int j = 0; j < NP; ++j) Lv += mi[j * NP + n] * rr[j];
        }
        const long long at = e0 * 5 * NP + i;
        p.Uout[at] = stage_value3(p, at, sU[(e * 5 + v) * NPP + n], Lv);
    }
}

}  // namespace
}  // namespace dgc

// CUDA-core kernels of the RKDG right-hand side and SSP-RK stage (FP32 and
// FP64), templated on the degree N.  Included by kernels_n<N>.cu only.
//
// One CTA handles a tile of E consecutive elements of one class (affine or
// curved; curved elements sit after the affine ones in device order).  The
// tile's state is one contiguous chunk of E*4*NP values, read and written
// coalesced.  Per stage (paper Sec. 4 flowchart, fused into one pass):
//   phase A  (e, cubature node):  U^cub = I_cub U, Euler flux F, G, the
//            contravariant weighted fluxes J(r_x F + r_y G), J(s_x F + s_y G)
//            (per-node factors for curved elements, Sec. 2 eq. stiffness)
//   phase C  (e, face point):     own trace I_g U, neighbour trace at the
//            reversed point (read from the neighbour's state in L2), or a
//            ghost state; local Lax-Friedrichs flux times sJ
//   phase D  (e, variable, node): weak-derivative products and lift,
//            M_k^-1 (folded into the operators for affine elements), then
//            the SSP-RK stage combination, stored coalesced.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "dg_device.h"

namespace dgc {

template <int N, typename Real>
struct Tile {
    static constexpr int NP = np_of(N), NQ = nq_of(N), NG = ng_of(N), NF = nf_of(N);
    static constexpr int E = (N == 2) ? 32 : (N == 3) ? 20 : (N == 4) ? 16 : (N == 5) ? 12 : 8;
    // shared-memory carve-up of the stage kernel (in Real elements)
    static constexpr int OPS = 3 * NP * NQ + 2 * NP * NF;
    static constexpr int PER_E = 4 * NP + 8 * NQ + 4 * NF + 16 + 4 * NP;
    static constexpr int PER_E_AV = 8 * NP + 1;
    static constexpr size_t smem_stage(bool av, int e = E) {
        return sizeof(Real) * (size_t)(OPS + e * (PER_E + (av ? PER_E_AV : 0)));
    }
    // gradient kernel: ops IcubT, DrT, DsT (curved) or QrT, QsT (affine), IgT, LT / MLT
    static constexpr int OPS_G = 3 * NP * NQ + 2 * NP * NF;
    static constexpr int PER_E_G = 4 * NP + 16 * NQ + 8 * NF + 16 + 8 * NP + 1;
    static constexpr size_t smem_grad(int e = E) { return sizeof(Real) * (size_t)(OPS_G + e * PER_E_G); }
    // the tile size of a launch: the mesh's tuned value or the default
    static __host__ __device__ int cap(int tile_e) { return tile_e > 0 ? tile_e : E; }
};


template <typename Real>
__device__ __forceinline__ void euler_flux(const Real U[4], Real gamma, Real F[4], Real G[4]) {
    const Real ir = recip(U[0]);
    const Real u = U[1] * ir, v = U[2] * ir;
    const Real p = (gamma - Real(1)) * (U[3] - Real(0.5) * (U[1] * u + U[2] * v));
    F[0] = U[1];
    F[1] = U[1] * u + p;
    F[2] = U[2] * u;
    F[3] = u * (U[3] + p);
    G[0] = U[2];
    G[1] = U[1] * v;
    G[2] = U[2] * v + p;
    G[3] = v * (U[3] + p);
}

// F*.n by local Lax-Friedrichs with the pointwise wave speed
// lam = max(|u-.n| + c-, |u+.n| + c+).  The normal flux of a state is formed
// directly, F.n = (m.n, m_x u_n + p n_x, m_y u_n + p n_y, (E + p) u_n) with
// u_n = m.n / rho, sharing p and 1/rho with the wave speed.
template <typename Real>
__device__ __forceinline__ void normal_flux(const Real U[4], Real nx, Real ny, Real gamma, Real Fn[4],
                                            Real& speed) {
    const Real ir = recip(U[0]);
    const Real mn = U[1] * nx + U[2] * ny;
    const Real un = mn * ir;
    const Real p = (gamma - Real(1)) * (U[3] - Real(0.5) * (U[1] * U[1] + U[2] * U[2]) * ir);
    Fn[0] = mn;
    Fn[1] = U[1] * un + p * nx;
    Fn[2] = U[2] * un + p * ny;
    Fn[3] = (U[3] + p) * un;
    speed = fabs(un) + fsqrt(gamma * p * ir);
}

template <typename Real>
__device__ __forceinline__ void llf_flux(const Real Um[4], const Real Up[4], Real nx, Real ny, Real gamma,
                                         Real Fn[4]) {
    Real Fm[4], Fp[4], lm, lp;
    normal_flux(Um, nx, ny, gamma, Fm, lm);
    normal_flux(Up, nx, ny, gamma, Fp, lp);
    const Real lam = fmax(lm, lp);
#pragma unroll
    for (int v = 0; v < 4; ++v) Fn[v] = Real(0.5) * (Fm[v] + Fp[v]) - Real(0.5) * lam * (Up[v] - Um[v]);
}

// F*.n by HLLC (Toro, Spruce and Speares) with Davis wave-speed estimates
// S_L = min(u_n- - c-, u_n+ - c+), S_R = max(u_n- + c-, u_n+ + c+), the
// contact speed S_M and the star states of each side; the branch order
// (S_L >= 0, S_M >= 0, S_R > 0) is the flux's upwinding.
template <typename Real>
__device__ __forceinline__ void hllc_flux(const Real Um[4], const Real Up[4], Real nx, Real ny, Real gamma,
                                          Real Fn[4]) {
    const Real g1 = gamma - Real(1);
    const Real irl = recip(Um[0]), irr = recip(Up[0]);
    const Real ul = Um[1] * irl, vl = Um[2] * irl, ur = Up[1] * irr, vr = Up[2] * irr;
    const Real unl = ul * nx + vl * ny, unr = ur * nx + vr * ny;
    const Real pl = g1 * (Um[3] - Real(0.5) * (Um[1] * ul + Um[2] * vl));
    const Real pr = g1 * (Up[3] - Real(0.5) * (Up[1] * ur + Up[2] * vr));
    const Real cl = fsqrt(gamma * pl * irl), cr = fsqrt(gamma * pr * irr);
    const Real SL = fmin(unl - cl, unr - cr), SR = fmax(unl + cl, unr + cr);
    const Real SM = (pr - pl + Um[0] * unl * (SL - unl) - Up[0] * unr * (SR - unr)) /
                    (Um[0] * (SL - unl) - Up[0] * (SR - unr));
    // the side whose flux (and star state) is used, and its wave speed
    const bool left = SM >= Real(0);
    const Real* U = left ? Um : Up;
    const Real un = left ? unl : unr, u = left ? ul : ur, v = left ? vl : vr, pk = left ? pl : pr;
    const Real S = left ? SL : SR;
    Fn[0] = U[0] * un;
    Fn[1] = U[1] * un + pk * nx;
    Fn[2] = U[2] * un + pk * ny;
    Fn[3] = (U[3] + pk) * un;
    if ((left && SL >= Real(0)) || (!left && SR <= Real(0))) return;   // supersonic: the upwind flux
    const Real f = U[0] * (S - un) / (S - SM);
    const Real us[4] = {f, f * (u + (SM - un) * nx), f * (v + (SM - un) * ny),
                        f * (U[3] / U[0] + (SM - un) * (SM + pk / (U[0] * (S - un))))};
#pragma unroll
    for (int w = 0; w < 4; ++w) Fn[w] += S * (us[w] - U[w]);
}

// The numerical flux selected by p.flux.
template <typename Real>
__device__ __forceinline__ void num_flux(int which, const Real Um[4], const Real Up[4], Real nx, Real ny, Real gamma,
                                         Real Fn[4]) {
    if (which == 1)
        hllc_flux(Um, Up, nx, ny, gamma, Fn);
    else
        llf_flux(Um, Up, nx, ny, gamma, Fn);
}

template <typename Real>
__device__ __forceinline__ void ghost_state(const Real Um[4], int bc, Real nx, Real ny, const Real* uinf,
                                            Real Up[4]) {
    if (bc == 1) {  // slip wall: reflect the normal momentum
        const Real mn = Um[1] * nx + Um[2] * ny;
        Up[0] = Um[0];
        Up[1] = Um[1] - Real(2) * mn * nx;
        Up[2] = Um[2] - Real(2) * mn * ny;
        Up[3] = Um[3];
    } else {  // farfield
#pragma unroll
        for (int v = 0; v < 4; ++v) Up[v] = uinf[v];
    }
}

template <typename Real>
__device__ __forceinline__ void copy_to_smem(Real* dst, const Real* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// The threads that run one CUDA-core tile: the whole CTA (barrier 0), or a
// warp-aligned group of a larger CTA with a named barrier of its own.
struct TileThreads {
    int tid, n;
    uint32_t bar;
    __device__ __forceinline__ void sync() const {
        if (bar == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" :: "r"(bar), "r"(n) : "memory");
    }
};
__device__ __forceinline__ TileThreads cta_threads() { return TileThreads{(int)threadIdx.x, (int)blockDim.x, 0u}; }

template <typename Real>
__device__ __forceinline__ void copy_to_smem(const TileThreads& th, Real* dst, const Real* src, int n) {
    for (int i = th.tid; i < n; i += th.n) dst[i] = src[i];
}

// Affine geometry of element k into g[16]: J r_x, J r_y, J s_x, J s_y, 1/J,
// then per face (n_x, n_y, sJ).  From x_r, x_s, y_r, y_s of the affine map:
// J r_x = y_s, J r_y = -x_s, J s_x = -y_r, J s_y = x_r; face tangents
// dx/dt = (x_r, y_r), (x_s - x_r, y_s - y_r), (-x_s, -y_s).
template <typename Real>
__device__ __forceinline__ void affine_geometry(const Real* gA, Real* g) {
    const Real xr = gA[0], xs = gA[1], yr = gA[2], ys = gA[3];
    g[0] = ys;
    g[1] = -xs;
    g[2] = -yr;
    g[3] = xr;
    g[4] = Real(1) / (xr * ys - xs * yr);
    const Real tx[3] = {xr, xs - xr, -xs}, ty[3] = {yr, ys - yr, -ys};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const Real sJ = sqrt(tx[f] * tx[f] + ty[f] * ty[f]);
        g[5 + 3 * f] = ty[f] / sJ;
        g[6 + 3 * f] = -tx[f] / sJ;
        g[7 + 3 * f] = sJ;
    }
}

// Tile bookkeeping: blocks [0, nAff) take affine tiles, the rest curved ones.
struct TileRange {
    long long e0;
    int ne;
    bool curved;
};
__device__ __forceinline__ TileRange tile_range(long long K, long long Kaff, int E) {
    TileRange t;
    const long long nAff = (Kaff + E - 1) / E;
    if ((long long)blockIdx.x < nAff) {
        t.curved = false;
        t.e0 = (long long)blockIdx.x * E;
        t.ne = (int)min((long long)E, Kaff - t.e0);
    } else {
        t.curved = true;
        t.e0 = Kaff + (long long)(blockIdx.x - nAff) * E;
        t.ne = (int)min((long long)E, K - t.e0);
    }
    return t;
}

// eps from the two sensor integrals.  s = log10(num/den) is needed only
// inside the ramp band: outside it two comparisons (in FP64, without a
// division) decide, which keeps the FP64 transcendentals off the elements
// where eps is 0 or eps0.
template <typename Real>
__device__ __forceinline__ Real sensor_eps(const StageArgs<Real>& p, Real num, Real den) {
    double eps = 0.0;
    const double dn = (double)num, dd = (double)den;
    if (dn > 0.0 && dd > 0.0 && dn >= p.S_lo * dd) {
        if (dn > p.S_hi * dd) {
            eps = p.eps0;
        } else {
            const double s = log10(dn / dd);
            if (s > p.s0 + p.kappa)
                eps = p.eps0;
            else if (s >= p.s0 - p.kappa)
                eps = 0.5 * p.eps0 * (1.0 + sin(M_PI * (s - p.s0) / (2.0 * p.kappa)));
        }
    }
    return (Real)eps;
}

// The sensor of one element of the state being written (the next stage's
// eps), by one warp: affine elements over the modes u = V^-1 rho, curved
// ones over the cubature points with J (the same integrals as the sensor
// kernel).  rho: the element's density row in the new state.
template <int N, typename Real>
__device__ __forceinline__ Real element_sensor_warp(const StageArgs<Real>& p, long long k, const Real* rho) {
    constexpr int NP = np_of(N), NQ = nq_of(N);
    constexpr int NLOW = N * (N + 1) / 2;
    constexpr OpsLayout L = ops_layout(N);
    const int lane = threadIdx.x & 31;
    Real num = 0, den = 0;
    if (k < p.Kaff) {
        for (int m = lane; m < NP; m += 32) {
            Real um = 0;
            for (int j = 0; j < NP; ++j) um += p.ops[L.vinvt + j * NP + m] * rho[j];
            den += um * um;
            if (m >= NLOW) num += um * um;
        }
    } else {
        const Real* g = p.geoC + (k - p.Kaff) * curved_stride(N);
        for (int qn = lane; qn < NQ; qn += 32) {
            Real a = 0, b = 0;
            for (int j = 0; j < NP; ++j) {
                a += p.ops[L.icub + j * NQ + qn] * rho[j];
                b += p.ops[L.itopt + j * NQ + qn] * rho[j];
            }
            const Real wj = p.ops[L.w + qn] * g[4 * NQ + qn];
            den += wj * a * a;
            num += wj * b * b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    return sensor_eps(p, num, den);
}

// The stage combination of one value: L alone, the SSP form a Un + b (Us +
// dt L), or the low-storage form dU <- a dU + dt L, Uout = Us + b dU (a = 0
// on the first stage, where dU is not read).
template <typename Real>
__device__ __forceinline__ Real stage_value(const StageArgs<Real>& p, long long n, Real us, Real L) {
    if (p.rhs_only) return L;
    if (p.dU) {
        const Real d = (p.a != Real(0) ? p.a * p.dU[n] : Real(0)) + p.dt * L;
        p.dU[n] = d;
        return us + p.b * d;
    }
    return p.a * (p.a != Real(0) ? p.Un[n] : Real(0)) + p.b * (us + p.dt * L);
}

// ---------------------------------------------------------------------------
// Stage kernel: L(Us) and the SSP-RK combination (or L alone).
// ---------------------------------------------------------------------------
template <int N, typename Real, bool AV>
__device__ __forceinline__ void stage_tile(const StageArgs<Real>& p, const TileRange& t, unsigned char* smem_raw,
                                           const TileThreads& th = cta_threads(), int cap_e = 0) {
    using T = Tile<N, Real>;
    constexpr int NP = T::NP, NQ = T::NQ, NG = T::NG, NF = T::NF;
    const int E = cap_e > 0 ? cap_e : T::cap(p.tile_e);   // capacity of this launch's layout
    constexpr OpsLayout L = ops_layout(N);
    Real* sIcubT = reinterpret_cast<Real*>(smem_raw);
    Real* sXrT = sIcubT + NP * NQ;
    Real* sXsT = sXrT + NQ * NP;
    Real* sIgT = sXsT + NQ * NP;
    Real* sXLT = sIgT + NP * NF;
    Real* sU = sXLT + NF * NP;
    Real* sF = sU + E * 4 * NP;
    Real* sFS = sF + E * 8 * NQ;
    Real* sGeo = sFS + E * 4 * NF;
    Real* sR = sGeo + E * 16;
    Real* sQ = sR + E * 4 * NP;   // AV only
    Real* sEps = sQ + E * 8 * NP; // AV only

    const Real* ops = p.ops;
    copy_to_smem(th, sIcubT, ops + L.icub, NP * NQ);
    copy_to_smem(th, sXrT, ops + (t.curved ? L.drt : L.mrt), NQ * NP);
    copy_to_smem(th, sXsT, ops + (t.curved ? L.dst : L.mst), NQ * NP);
    copy_to_smem(th, sIgT, ops + L.igt, NP * NF);
    copy_to_smem(th, sXLT, ops + (t.curved ? L.lt : L.mlt), NF * NP);
    const int nval = t.ne * 4 * NP;
    const Real* Us_tile = p.Us + t.e0 * 4 * NP;
    for (int i = th.tid; i < nval; i += th.n) sU[i] = Us_tile[i];
    if (!t.curved)
        for (int e = th.tid; e < t.ne; e += th.n) affine_geometry(p.geoA + (t.e0 + e) * 4, sGeo + e * 16);
    if constexpr (AV) {
        const Real* q_tile = p.q + t.e0 * 8 * NP;
        for (int i = th.tid; i < t.ne * 8 * NP; i += th.n) sQ[i] = q_tile[i];
        for (int e = th.tid; e < t.ne; e += th.n) sEps[e] = sqrt(p.eps[t.e0 + e]);
    }
    th.sync();

    const Real gamma = p.gamma;
    const Real* geoC = p.geoC + (t.curved ? (t.e0 - p.Kaff) * curved_stride(N) : 0);

    // phase A: cubature nodes
    for (int it = th.tid; it < t.ne * NQ; it += th.n) {
        const int e = it / NQ, qn = it - e * NQ;
        Real Uc[4] = {0, 0, 0, 0};
        const Real* u = sU + e * 4 * NP;
#pragma unroll 4
        for (int j = 0; j < NP; ++j) {
            const Real w = sIcubT[j * NQ + qn];
#pragma unroll
            for (int v = 0; v < 4; ++v) Uc[v] += w * u[v * NP + j];
        }
        Real F[4], G[4];
        euler_flux(Uc, gamma, F, G);
        if constexpr (AV) {
            const Real* qe = sQ + e * 8 * NP;
            Real qx[4] = {0, 0, 0, 0}, qy[4] = {0, 0, 0, 0};
            for (int j = 0; j < NP; ++j) {
                const Real w = sIcubT[j * NQ + qn];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    qx[v] += w * qe[v * NP + j];
                    qy[v] += w * qe[(4 + v) * NP + j];
                }
            }
            const Real se = sEps[e];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                F[v] -= se * qx[v];
                G[v] -= se * qy[v];
            }
        }
        Real jrx, jry, jsx, jsy;
        if (!t.curved) {
            const Real* g = sGeo + e * 16;
            jrx = g[0]; jry = g[1]; jsx = g[2]; jsy = g[3];
        } else {
            const Real* g = geoC + (long long)e * curved_stride(N);
            jrx = g[qn]; jry = g[NQ + qn]; jsx = g[2 * NQ + qn]; jsy = g[3 * NQ + qn];
        }
        Real* f = sF + e * 8 * NQ;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            f[v * NQ + qn] = jrx * F[v] + jry * G[v];
            f[(4 + v) * NQ + qn] = jsx * F[v] + jsy * G[v];
        }
    }

    // phase C: face points
    for (int it = th.tid; it < t.ne * NF; it += th.n) {
        const int e = it / NF, fg = it - e * NF;
        const int f = fg / NG, g = fg - f * NG;
        const long long k = t.e0 + e;
        const int4 cn = p.conn[k];
        const int code = cn.w;
        const int bc = code_bc(code, f);
        const int nb = (f == 0) ? cn.x : (f == 1) ? cn.y : cn.z;
        Real nx, ny, sJ;
        if (!t.curved) {
            const Real* gg = sGeo + e * 16 + 5 + 3 * f;
            nx = gg[0]; ny = gg[1]; sJ = gg[2];
        } else {
            const Real* gg = geoC + (long long)e * curved_stride(N) + 5 * NQ;
            nx = gg[fg]; ny = gg[NF + fg]; sJ = gg[2 * NF + fg];
        }
        Real Um[4] = {0, 0, 0, 0}, Up[4] = {0, 0, 0, 0};
        const Real* u = sU + e * 4 * NP;
        for (int j = 0; j < NP; ++j) {
            const Real w = sIgT[j * NF + fg];
#pragma unroll
            for (int v = 0; v < 4; ++v) Um[v] += w * u[v * NP + j];
        }
        const int fgn = code_face(code, f) * NG + (NG - 1 - g);
        if (bc == 0) {
            const Real* un = p.Us + (long long)nb * 4 * NP;
            for (int j = 0; j < NP; ++j) {
                const Real w = sIgT[j * NF + fgn];
#pragma unroll
                for (int v = 0; v < 4; ++v) Up[v] += w * __ldg(un + v * NP + j);
            }
        } else {
            ghost_state(Um, bc, nx, ny, p.uinf, Up);
        }
        Real Fn[4];
        num_flux(p.flux, Um, Up, nx, ny, gamma, Fn);
        if constexpr (AV) {
            const Real se = sEps[e];
            const Real* qe = sQ + e * 8 * NP;
            Real qmx[4] = {0, 0, 0, 0}, qmy[4] = {0, 0, 0, 0};
            for (int j = 0; j < NP; ++j) {
                const Real w = sIgT[j * NF + fg];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    qmx[v] += w * qe[v * NP + j];
                    qmy[v] += w * qe[(4 + v) * NP + j];
                }
            }
            Real sep = se, qpx[4], qpy[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) { qpx[v] = qmx[v]; qpy[v] = qmy[v]; }
            if (bc == 0) {
                sep = sqrt(__ldg(p.eps + nb));
                const Real* qn_ = p.q + (long long)nb * 8 * NP;
#pragma unroll
                for (int v = 0; v < 4; ++v) { qpx[v] = 0; qpy[v] = 0; }
                for (int j = 0; j < NP; ++j) {
                    const Real w = sIgT[j * NF + fgn];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        qpx[v] += w * __ldg(qn_ + v * NP + j);
                        qpy[v] += w * __ldg(qn_ + (4 + v) * NP + j);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < 4; ++v)
                Fn[v] -= Real(0.5) * (se * (qmx[v] * nx + qmy[v] * ny) + sep * (qpx[v] * nx + qpy[v] * ny));
        }
        Real* fs = sFS + e * 4 * NF;
#pragma unroll
        for (int v = 0; v < 4; ++v) fs[v * NF + fg] = Fn[v] * sJ;
    }
    th.sync();

    // phase D: products, M^-1, stage combination
    const long long base = t.e0 * 4 * NP;
    for (int it = th.tid; it < nval; it += th.n) {
        const int e = it / (4 * NP), r = it - e * 4 * NP, v = r / NP, i = r - v * NP;
        const Real* fr = sF + e * 8 * NQ + v * NQ;
        const Real* fs = sF + e * 8 * NQ + (4 + v) * NQ;
        Real acc = 0;
#pragma unroll 4
        for (int qn = 0; qn < NQ; ++qn) acc += sXrT[qn * NP + i] * fr[qn] + sXsT[qn * NP + i] * fs[qn];
        const Real* fl = sFS + (e * 4 + v) * NF;
#pragma unroll 4
        for (int fg = 0; fg < NF; ++fg) acc -= sXLT[fg * NP + i] * fl[fg];
        if (!t.curved) {
            const Real Lv = acc * sGeo[e * 16 + 4];
            p.Uout[base + it] = stage_value(p, base + it, sU[it], Lv);
        } else {
            sR[it] = acc;
        }
    }
    if (t.curved) {
        th.sync();
        for (int it = th.tid; it < nval; it += th.n) {
            const int e = it / (4 * NP), r = it - e * 4 * NP, v = r / NP, i = r - v * NP;
            const Real* mi = geoC + (long long)e * curved_stride(N) + 5 * NQ + 3 * NF;
            const Real* rr = sR + (e * 4 + v) * NP;
            Real Lv = 0;
            for (int j = 0; j < NP; ++j) Lv += mi[j * NP + i] * rr[j];
            p.Uout[base + it] = stage_value(p, base + it, sU[it], Lv);
        }
    }
    if constexpr (AV) {
        if (p.eps_next != nullptr && !p.rhs_only) {   // eps of the new state, one warp per element
            th.sync();                            // the tile's new state is written
            for (int e = th.tid >> 5; e < t.ne; e += th.n >> 5) {
                const Real eps = element_sensor_warp<N, Real>(p, t.e0 + e, p.Uout + (t.e0 + e) * 4 * NP);
                if ((th.tid & 31) == 0) {
                    p.eps_next[t.e0 + e] = eps;
                    if (p.visc && eps > Real(0)) atomicAdd(p.visc, 1);
                }
            }
        }
    }
}

// Out-of-line copies of the CUDA-core tile bodies, called from the
// persistent tensor-core kernels for curved tiles so that they do not add
// to those kernels' register allocation.
template <int N, typename Real, bool AV>
__device__ __noinline__ void stage_tile_call(const StageArgs<Real>& p, const TileRange& t, unsigned char* smem) {
    stage_tile<N, Real, AV>(p, t, smem);
}
template <int N, typename Real, bool AV>
__device__ __noinline__ void stage_tile_call(const StageArgs<Real>& p, const TileRange& t, unsigned char* smem,
                                             const TileThreads& th, int cap_e) {
    stage_tile<N, Real, AV>(p, t, smem, th, cap_e);
}

template <int N, typename Real, bool AV>
__global__ void __launch_bounds__(THREADS) stage_kernel(StageArgs<Real> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileRange t = tile_range(p.K, p.Kaff, Tile<N, Real>::cap(p.tile_e));
    if (t.ne <= 0) return;
    stage_tile<N, Real, AV>(p, t, smem_raw);
}

// ---------------------------------------------------------------------------
// Persson-Peraire sensor: eps_k from the density (paper Sec. 2).
// Affine elements: one thread per element; the block stages the densities of
// its 128 elements in shared memory with coalesced loads and reads V^-1 as
// broadcasts.  S = sum_{deg N} u^2 / sum u^2 with u = V^-1 rho (the cubature
// form for constant J and an orthonormal basis).
// Curved elements: one warp per element, lanes over the cubature points,
// both integrals by cubature with J, in blocks of their own at the front of
// the grid so that they do not form a tail.
// Sums in the state precision; ratio, log10 and the sine ramp in FP64.
// ---------------------------------------------------------------------------
constexpr int SENSOR_THREADS = 128;
constexpr int SENSOR_CURVED_PER_BLOCK = SENSOR_THREADS / 32;

template <int N, typename Real>
__global__ void __launch_bounds__(SENSOR_THREADS) sensor_kernel(StageArgs<Real> p, Real* eps_out, int ncb) {
    constexpr int NP = np_of(N), NQ = nq_of(N);
    constexpr int NLOW = N * (N + 1) / 2;  // modes of degree <= N-1 come first
    constexpr OpsLayout L = ops_layout(N);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the state comes from the previous kernel
    if ((int)blockIdx.x < ncb) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const long long k = p.Kaff + (long long)blockIdx.x * SENSOR_CURVED_PER_BLOCK + warp;
        if (k >= p.K) return;
        const Real* rho = p.Us + k * 4 * NP;
        const Real* g = p.geoC + (k - p.Kaff) * curved_stride(N);
        Real num = 0, den = 0;
        for (int qn = lane; qn < NQ; qn += 32) {
            Real a = 0, b = 0;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const Real r = __ldg(rho + j);
                a += __ldg(p.ops + L.icub + j * NQ + qn) * r;
                b += __ldg(p.ops + L.itopt + j * NQ + qn) * r;
            }
            const Real wj = p.ops[L.w + qn] * g[4 * NQ + qn];
            den += wj * a * a;
            num += wj * b * b;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (lane == 0) {
            const Real ev = sensor_eps(p, num, den);
            eps_out[k] = ev;
            if (p.visc && ev > Real(0)) atomicAdd(p.visc, 1);
        }
        return;
    }
    constexpr int RS = NP | 1;   // odd row stride: conflict-free column reads
    __shared__ Real sRho[SENSOR_THREADS * RS];
    __shared__ Real sV[NP * NP];
    const long long k0 = (long long)(blockIdx.x - ncb) * SENSOR_THREADS;
    const int nb = (int)min((long long)SENSOR_THREADS, p.Kaff - k0);
    for (int i = threadIdx.x; i < NP * NP; i += SENSOR_THREADS) sV[i] = p.ops[L.vinvt + i];
    for (int i = threadIdx.x; i < nb * NP; i += SENSOR_THREADS) {
        const int e = i / NP, j = i - e * NP;
        sRho[e * RS + j] = p.Us[(k0 + e) * 4 * NP + j];
    }
    __syncthreads();
    const int e = threadIdx.x;
    if (e >= nb) return;
    const Real* rho = sRho + e * RS;
    Real num = 0, den = 0;
#pragma unroll 1
    for (int m = 0; m < NP; ++m) {
        Real um = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) um += sV[j * NP + m] * rho[j];
        den += um * um;
        if (m >= NLOW) num += um * um;
    }
    const Real ev = sensor_eps(p, num, den);
    eps_out[k0 + e] = ev;
    if (p.visc && ev > Real(0)) atomicAdd(p.visc, 1);
}

// ---------------------------------------------------------------------------
// Gradient kernel for the artificial viscosity: q = sqrt(eps) grad U by the
// DG weak form with central fluxes,
//   M q_m = -sum (weak derivative of sqrt(eps) U) + sum_f I_g^T diag(w sJ n_m) (sqrt(eps) U)*.
// Affine elements use the folded node-to-node operators Mref^-1 D^T W I_cub
// (exact for these polynomial integrands); curved ones go through the
// cubature nodes with per-node factors and apply M_k^-1.
// ---------------------------------------------------------------------------
template <int N, typename Real>
__device__ __forceinline__ void grad_tile(const StageArgs<Real>& p, Real* q_out, const TileRange& t,
                                          unsigned char* smem_raw) {
    using T = Tile<N, Real>;
    constexpr int NP = T::NP, NQ = T::NQ, NG = T::NG, NF = T::NF;
    const int E = T::cap(p.tile_e);   // capacity of this launch's layout
    constexpr OpsLayout L = ops_layout(N);
    Real* sIcubT = reinterpret_cast<Real*>(smem_raw);   // curved only
    Real* sXrT = sIcubT + NP * NQ;                      // DrT [NQ][NP] or QrT [NP][NP]
    Real* sXsT = sXrT + NQ * NP;
    Real* sIgT = sXsT + NQ * NP;
    Real* sXLT = sIgT + NP * NF;
    Real* sU = sXLT + NF * NP;
    Real* sG = sU + E * 4 * NP;        // curved: [e][m][c][v][NQ] factors times sqrt(eps) U^cub
    Real* sUS = sG + E * 16 * NQ;      // [e][m][v][NF]  n_m sJ (sqrt(eps) U)*
    Real* sGeo = sUS + E * 8 * NF;
    Real* sR = sGeo + E * 16;          // [e][m][v][NP]
    Real* sEps = sR + E * 8 * NP;

    // q enters the stage only as sqrt(eps) q of its own element, so a tile
    // whose elements all have eps = 0 needs none: it is neither computed nor
    // written
    {
        __shared__ int s_visc;
        __syncthreads();   // a previous tile of a persistent caller is done with s_visc
        if (threadIdx.x == 0) s_visc = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x)
            if (p.eps[t.e0 + e] > Real(0)) s_visc = 1;
        __syncthreads();
        if (!s_visc) return;
    }

    const Real* ops = p.ops;
    if (t.curved) {
        copy_to_smem(sIcubT, ops + L.icub, NP * NQ);
        copy_to_smem(sXrT, ops + L.drt, NQ * NP);
        copy_to_smem(sXsT, ops + L.dst, NQ * NP);
        copy_to_smem(sXLT, ops + L.lt, NF * NP);
    } else {
        copy_to_smem(sXrT, ops + L.qrt, NP * NP);
        copy_to_smem(sXsT, ops + L.qst, NP * NP);
        copy_to_smem(sXLT, ops + L.mlt, NF * NP);
    }
    copy_to_smem(sIgT, ops + L.igt, NP * NF);
    const int nval = t.ne * 4 * NP;
    const Real* Us_tile = p.Us + t.e0 * 4 * NP;
    for (int i = threadIdx.x; i < nval; i += blockDim.x) sU[i] = Us_tile[i];
    for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
        sEps[e] = sqrt(p.eps[t.e0 + e]);
        if (!t.curved) affine_geometry(p.geoA + (t.e0 + e) * 4, sGeo + e * 16);
    }
    __syncthreads();
    const Real* geoC = p.geoC + (t.curved ? (t.e0 - p.Kaff) * curved_stride(N) : 0);

    if (t.curved) {
        for (int it = threadIdx.x; it < t.ne * NQ; it += blockDim.x) {
            const int e = it / NQ, qn = it - e * NQ;
            Real Uc[4] = {0, 0, 0, 0};
            const Real* u = sU + e * 4 * NP;
            for (int j = 0; j < NP; ++j) {
                const Real w = sIcubT[j * NQ + qn];
#pragma unroll
                for (int v = 0; v < 4; ++v) Uc[v] += w * u[v * NP + j];
            }
            const Real* g = geoC + (long long)e * curved_stride(N);
            const Real fac[4] = {g[qn], g[2 * NQ + qn], g[NQ + qn], g[3 * NQ + qn]};  // (x: Jrx, Jsx), (y: Jry, Jsy)
            const Real se = sEps[e];
            Real* gg = sG + e * 16 * NQ;
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int v = 0; v < 4; ++v) gg[(c * 4 + v) * NQ + qn] = fac[c] * se * Uc[v];
        }
    }
    for (int it = threadIdx.x; it < t.ne * NF; it += blockDim.x) {
        const int e = it / NF, fg = it - e * NF;
        const int f = fg / NG, g = fg - f * NG;
        const long long k = t.e0 + e;
        const int4 cn = p.conn[k];
        const int bc = code_bc(cn.w, f);
        const int nb = (f == 0) ? cn.x : (f == 1) ? cn.y : cn.z;
        Real nx, ny, sJ;
        if (!t.curved) {
            const Real* gg = sGeo + e * 16 + 5 + 3 * f;
            nx = gg[0]; ny = gg[1]; sJ = gg[2];
        } else {
            const Real* gg = geoC + (long long)e * curved_stride(N) + 5 * NQ;
            nx = gg[fg]; ny = gg[NF + fg]; sJ = gg[2 * NF + fg];
        }
        Real Um[4] = {0, 0, 0, 0}, Up[4] = {0, 0, 0, 0};
        const Real* u = sU + e * 4 * NP;
        for (int j = 0; j < NP; ++j) {
            const Real w = sIgT[j * NF + fg];
#pragma unroll
            for (int v = 0; v < 4; ++v) Um[v] += w * u[v * NP + j];
        }
        const Real se = sEps[e];
        Real sep = se;
        if (bc == 0) {
            const int fgn = code_face(cn.w, f) * NG + (NG - 1 - g);
            const Real* un = p.Us + (long long)nb * 4 * NP;
            for (int j = 0; j < NP; ++j) {
                const Real w = sIgT[j * NF + fgn];
#pragma unroll
                for (int v = 0; v < 4; ++v) Up[v] += w * __ldg(un + v * NP + j);
            }
            sep = sqrt(__ldg(p.eps + nb));
        } else {
            ghost_state(Um, bc, nx, ny, p.uinf, Up);
        }
        Real* us = sUS + e * 8 * NF;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const Real st = Real(0.5) * (se * Um[v] + sep * Up[v]) * sJ;
            us[v * NF + fg] = nx * st;
            us[(4 + v) * NF + fg] = ny * st;
        }
    }
    __syncthreads();

    for (int it = threadIdx.x; it < t.ne * 8 * NP; it += blockDim.x) {
        const int e = it / (8 * NP), r = it - e * 8 * NP, m = r / (4 * NP), r2 = r - m * 4 * NP;
        const int v = r2 / NP, i = r2 - v * NP;
        Real acc = 0;
        const Real* us = sUS + (e * 8 + m * 4 + v) * NF;
        for (int fg = 0; fg < NF; ++fg) acc += sXLT[fg * NP + i] * us[fg];
        if (!t.curved) {
            const Real* g = sGeo + e * 16;
            const Real cr = (m == 0) ? g[0] : g[1];  // J r_x or J r_y
            const Real cs = (m == 0) ? g[2] : g[3];  // J s_x or J s_y
            const Real* u = sU + (e * 4 + v) * NP;
            Real dr = 0, ds = 0;
            for (int j = 0; j < NP; ++j) {
                dr += sXrT[j * NP + i] * u[j];
                ds += sXsT[j * NP + i] * u[j];
            }
            const Real val = (acc - sEps[e] * (cr * dr + cs * ds)) * g[4];
            q_out[(t.e0 + e) * 8 * NP + (m * 4 + v) * NP + i] = val;
        } else {
            const Real* gr = sG + e * 16 * NQ + ((2 * m) * 4 + v) * NQ;
            const Real* gs = sG + e * 16 * NQ + ((2 * m + 1) * 4 + v) * NQ;
            for (int qn = 0; qn < NQ; ++qn) acc -= sXrT[qn * NP + i] * gr[qn] + sXsT[qn * NP + i] * gs[qn];
            sR[it] = acc;
        }
    }
    if (t.curved) {
        __syncthreads();
        for (int it = threadIdx.x; it < t.ne * 8 * NP; it += blockDim.x) {
            const int e = it / (8 * NP), r = it - e * 8 * NP, mv = r / NP, i = r - mv * NP;
            const Real* mi = geoC + (long long)e * curved_stride(N) + 5 * NQ + 3 * NF;
            const Real* rr = sR + (e * 8 + mv) * NP;
            Real val = 0;
            for (int j = 0; j < NP; ++j) val += mi[j * NP + i] * rr[j];
            q_out[(t.e0 + e) * 8 * NP + mv * NP + i] = val;
        }
    }
}

template <int N, typename Real>
__global__ void __launch_bounds__(THREADS) grad_kernel(StageArgs<Real> p, Real* q_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileRange t = tile_range(p.K, p.Kaff, Tile<N, Real>::cap(p.tile_e));
    if (t.ne <= 0) return;
    grad_tile<N, Real>(p, q_out, t, smem_raw);
}

template <int N, typename Real>
__device__ __noinline__ void grad_tile_call(const StageArgs<Real>& p, Real* q_out, const TileRange& t,
                                            unsigned char* smem) {
    grad_tile<N, Real>(p, q_out, t, smem);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
inline unsigned tiles_of(long long K, long long Kaff, int E) {
    return (unsigned)((Kaff + E - 1) / E + (K - Kaff + E - 1) / E);
}

// largest shared-memory request of one CTA on this architecture
constexpr size_t SMEM_CTA_MAX = 232448;

// Let a kernel take up to the largest dynamic shared memory it can have next
// to its static shared memory.
inline cudaError_t allow_max_dynamic_smem(const void* kern) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(SMEM_CTA_MAX - fa.sharedSizeBytes));
}

template <int N, typename Real>
int tile_e_default() {
    return Tile<N, Real>::E;
}

template <int N, typename Real>
bool tile_e_fits(int e, int av) {
    using T = Tile<N, Real>;
    return e >= 1 && T::smem_stage(av != 0, e) <= SMEM_CTA_MAX && T::smem_grad(e) <= SMEM_CTA_MAX;
}

template <int N, typename Real>
int launch_stage(const StageArgs<Real>& a, int av, cudaStream_t st) {
    using T = Tile<N, Real>;
    const int E = T::cap(a.tile_e);
    if (!tile_e_fits<N, Real>(E, av)) return (int)cudaErrorInvalidValue;
    const unsigned grid = tiles_of(a.K, a.Kaff, E);
    if (grid == 0) return 0;
    if (av)
        stage_kernel<N, Real, true><<<grid, THREADS, T::smem_stage(true, E), st>>>(a);
    else
        stage_kernel<N, Real, false><<<grid, THREADS, T::smem_stage(false, E), st>>>(a);
    return (int)cudaGetLastError();
}

template <int N, typename Real>
int launch_sensor(const StageArgs<Real>& a, Real* eps_out, cudaStream_t st) {
    const long long Kc = a.K - a.Kaff;
    const int ncb = (int)((Kc + SENSOR_CURVED_PER_BLOCK - 1) / SENSOR_CURVED_PER_BLOCK);
    const unsigned grid = (unsigned)(ncb + (a.Kaff + SENSOR_THREADS - 1) / SENSOR_THREADS);
    if (grid == 0) return 0;
    return (int)launch_pdl(sensor_kernel<N, Real>, grid, SENSOR_THREADS, 0, st, a, eps_out, ncb);
}

template <int N, typename Real>
int launch_grad(const StageArgs<Real>& a, Real* q_out, cudaStream_t st) {
    using T = Tile<N, Real>;
    const int E = T::cap(a.tile_e);
    if (!tile_e_fits<N, Real>(E, 1)) return (int)cudaErrorInvalidValue;
    const unsigned grid = tiles_of(a.K, a.Kaff, E);
    if (grid == 0) return 0;
    grad_kernel<N, Real><<<grid, THREADS, T::smem_grad(E), st>>>(a, q_out);
    return (int)cudaGetLastError();
}

// The limits admit every tile size that tile_e_fits accepts.
template <int N, typename Real>
int prepare_kernels() {
    cudaError_t e1 = allow_max_dynamic_smem((const void*)stage_kernel<N, Real, true>);
    cudaError_t e2 = allow_max_dynamic_smem((const void*)stage_kernel<N, Real, false>);
    cudaError_t e3 = allow_max_dynamic_smem((const void*)grad_kernel<N, Real>);
    return (int)(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3);
}

}  // namespace dgc

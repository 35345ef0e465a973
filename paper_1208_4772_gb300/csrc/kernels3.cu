// Stage kernel of the tetrahedral method (paper Sec. 2 with d = 3) on the
// CUDA cores: L(U) and the Runge-Kutta stage combination for a tile of E
// elements per CTA pass, persistent over tiles.
//
// Per tile (all in shared memory):
//   0  state rows, face codes, affine geometry (cofactors of dx/dr, 1/J);
//      the neighbours' face-node values (gathered through fmask)
//   1  per cubature point: U^cub = I_cub U, the Euler fluxes and the
//      contravariant fluxes sum_d (J dr_a/dx_d) F_d, a = r, s, t
//   2  vol = D_r^T W Fr + D_s^T W Fs + D_t^T W Ft
//   3  per face-frame point: U- and U+ from the face nodes by I2 of the
//      face's orientation (the neighbour's with its own orientation), ghost
//      states on boundary faces, outward normal and area factor, the
//      numerical flux times w_g sJ
//   4  R = vol - sum_f I2_f^T (w sJ F*) scattered to the face nodes
//   5  L = M_k^-1 R (affine: M_ref^-1 / J) and the stage update
#include <algorithm>

#include "kernels3.cuh"

namespace dgc {

namespace {

// Shared-memory layout of a CTA for tiles of E elements (offsets in reals).
template <int N, typename Real>
struct T3 {
    static constexpr int NP = np3_of(N), NFP = nfp3_of(N), NQ = nq3_of(N), NG = ng3_of(N);
    static constexpr int NPP = pad4(NP), NQP = pad4(NQ), NFPP = pad4(NFP), NGP = pad4(NG);
    static constexpr int O_I2 = 0;                           // [6][NG][NFPP]
    static constexpr int O_I2T = O_I2 + 6 * NG * NFPP;       // [6][NFP][NGP]
    static constexpr int O_W = O_I2T + 6 * NFP * NGP;
    static constexpr int O_MI = pad4(O_W + NG);
    static constexpr int O_U = pad4(O_MI + NP * NP);         // [E][5][NPP]
    // flux rows of one (element, direction): 5 rows of NQP plus 4 reals, so
    // that the blocks the lanes of one warp read start in different banks
    static constexpr int FST = 5 * NQP + 4;
    int O_F, O_UF, O_NB, O_FS, O_T, O_R, O_G, O_SE, O_Q, O_QF, O_QN, O_END;
    size_t bytes;
    // mode 0: the Euler stage; 1: with the viscous terms (q rows, their face
    // nodes on both sides, sqrt(eps)); 2: the gradient pass (sqrt(eps))
    __host__ __device__ constexpr explicit T3(int E, int mode = 0)
        : O_F(O_U + E * 5 * NPP),          // [E][3][FST] contravariant fluxes
          O_UF(O_F + E * 3 * FST),         // [E][4][5][NFPP] own face nodes
          O_NB(O_UF + E * 20 * NFPP),      // [E][4][5][NFPP] neighbours' face nodes
          O_FS(O_NB + E * 20 * NFPP),      // [E][4][5][NGP] w sJ F*
          O_T(O_FS + E * 20 * NGP),        // [E][4][5][NFPP] lifted face terms
          O_R(O_T + E * 20 * NFPP),        // [3][E][5][NP] volume parts, then R
          O_G(O_R + 3 * E * 5 * NP),       // [E][16] affine cofactors, 1/J
          O_SE(O_G + E * 16),              // [E][5] sqrt(eps): own, then each face's other side
          O_Q(pad4(O_SE + (mode ? E * 5 : 0))),                  // [E][15][NPP] q rows
          O_QF(O_Q + (mode == 1 ? E * 15 * NPP : 0)),            // [E][4][15][NFPP] own q face nodes
          O_QN(O_QF + (mode == 1 ? E * 60 * NFPP : 0)),          // [E][4][15][NFPP] neighbours'
          O_END(O_QN + (mode == 1 ? E * 60 * NFPP : 0)),
          bytes((size_t)O_END * sizeof(Real) + (size_t)(4 * NFP + 4 * NP + 8 * E) * sizeof(int)) {}
    static constexpr int default_e() { return sizeof(Real) == 4 ? (N <= 2 ? 8 : N == 3 ? 4 : 2) : (N <= 2 ? 4 : N == 3 ? 2 : 1); }
};

// Largest dynamic shared memory of one CTA.
constexpr size_t SMEM3_MAX = 232448;

template <int N, typename Real, int MODE>
__global__ void __launch_bounds__(THREADS) stage3_kernel(const StageArgs3<Real> p) {
    using TT = T3<N, Real>;
    constexpr int NP = TT::NP, NFP = TT::NFP, NQ = TT::NQ, NG = TT::NG, NPP = TT::NPP, NQP = TT::NQP;
    constexpr int NFPP = TT::NFPP, NGP = TT::NGP, NH = (NP + 1) / 2;
    const int E = p.tile_e;
    const TT T(E, MODE);
    constexpr Ops3Layout L = ops3_layout(N);
    constexpr int CS = curved3_stride(N);
    extern __shared__ __align__(16) unsigned char smem3[];
    Real* S = reinterpret_cast<Real*>(smem3);
    Real* sI2 = S + TT::O_I2;
    Real* sI2T = S + TT::O_I2T;
    Real* sW = S + TT::O_W;
    Real* sMiT = S + TT::O_MI;
    Real* sU = S + TT::O_U;
    Real* sF = S + T.O_F;
    Real* sUf = S + T.O_UF;
    Real* sNb = S + T.O_NB;
    Real* sFs = S + T.O_FS;
    Real* sT = S + T.O_T;
    Real* sR = S + T.O_R;
    Real* sG = S + T.O_G;
    Real* sSe = S + T.O_SE;
    Real* sQ = S + T.O_Q;
    Real* sQf = S + T.O_QF;
    Real* sQn = S + T.O_QN;
    int* sFmask = reinterpret_cast<int*>(S + T.O_END);
    int* sFpos = sFmask + 4 * NFP;
    int* sNbr = sFpos + 4 * NP;
    int* sCode = sNbr + 4 * E;
    const int tid = threadIdx.x;
    const Real* __restrict__ IcubB = p.ops + L.icub;

    // the padding of the state, flux, face-node and face-flux rows (and of
    // the q rows and their face nodes) stays zero
    for (int i = tid; i < T.O_T - TT::O_U; i += THREADS) sU[i] = Real(0);
    for (int i = tid; i < T.O_END - T.O_Q; i += THREADS) sQ[i] = Real(0);
    for (int i = tid; i < 6 * NG * NFPP + 6 * NFP * NGP; i += THREADS) sI2[i] = p.ops[L.i2 + i];
    for (int i = tid; i < NG; i += THREADS) sW[i] = p.ops[L.wg + i];
    for (int i = tid; i < NP * NP; i += THREADS) sMiT[i] = p.ops[L.mi + i];
    for (int i = tid; i < 4 * NFP + 4 * NP; i += THREADS) sFmask[i] = p.opsi[i];

    const long long ntiles = (p.K + E - 1) / E;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long e0 = tile * E;
        const int ne = (int)min((long long)E, p.K - e0);
        __syncthreads();
        // ---- phase 0: rows, codes, affine geometry
        const Real* Ug = p.Us + e0 * 5 * NP;
        for (int i = tid; i < ne * 5 * NP; i += THREADS) {
            const int row = i / NP;
            sU[row * NPP + (i - row * NP)] = Ug[i];
        }
        for (int i = tid; i < ne * 4; i += THREADS) {
            const int e = i >> 2, f = i & 3;
            const int4 nb = p.conn[e0 + e];
            const int2 cw = p.code[e0 + e];
            sNbr[i] = f == 0 ? nb.x : f == 1 ? nb.y : f == 2 ? nb.z : nb.w;
            sCode[i] = ((f < 2 ? cw.x : cw.y) >> (16 * (f & 1))) & 0xffff;
            if constexpr (MODE != 0) {   // sqrt(eps) of the face's other side (the element's own on boundaries)
                const long long o = code3_bc(sCode[i]) == 0 ? (long long)sNbr[i] : e0 + e;
                sSe[e * 5 + 1 + f] = sqrt(p.eps[o]);
                if (f == 0) sSe[e * 5] = sqrt(p.eps[e0 + e]);
            }
        }
        if constexpr (MODE == 1) {   // q rows [15][NPP]
            const Real* Qg = p.q + e0 * 15 * NP;
            for (int i = tid; i < ne * 15 * NP; i += THREADS) {
                const int row = i / NP;
                sQ[row * NPP + (i - row * NP)] = Qg[i];
            }
        }
        for (int e = tid; e < ne; e += THREADS) {
            if (e0 + e >= p.Kaff) continue;
            affine_cofactors3(p.geoA + (e0 + e) * 9, sG + e * 16);
        }
        // with artificial viscosity: does eps vanish on the tile's elements
        // and on all their face neighbours?  Then q = 0 on the tile and its
        // viscous terms vanish exactly: the gradient pass writes zeros, the
        // stage runs the inviscid body.
        bool visc = true;
        if constexpr (MODE != 0) {
            int any = 0;
            for (int i = tid; i < ne * 5; i += THREADS) any |= sSe[i] != Real(0);
            visc = __syncthreads_or(any) != 0;
        } else {
            __syncthreads();
        }
        if constexpr (MODE == 2) {
            if (!visc) {
                for (int i = tid; i < ne * 5 * NP; i += THREADS) {
                    const int e = i / (5 * NP), r = i - e * 5 * NP;
                    p.qout[(e0 + e) * 15 * NP + p.grad_m * 5 * NP + r] = Real(0);
                }
                continue;
            }
        }
        // own and neighbours' face-node values, rows of NFPP
        for (int i = tid; i < ne * 20 * NFP; i += THREADS) {
            const int row = i / NFP, n = i - row * NFP;   // row = (e * 4 + f) * 5 + v
            const int e = row / 20, f = (row / 5) & 3, v = row % 5;
            const int code = sCode[e * 4 + f];
            sUf[row * NFPP + n] = sU[(e * 5 + v) * NPP + sFmask[f * NFP + n]];
            if (code3_bc(code) == 0) {
                const long long nb = sNbr[e * 4 + f];
                sNb[row * NFPP + n] = p.Us[nb * 5 * NP + v * NP + sFmask[code3_face(code) * NFP + n]];
            }
        }
        if constexpr (MODE == 1) {   // q face nodes of both sides, rows (e * 4 + f) * 15 + r
            for (int i = tid; i < (visc ? ne * 60 * NFP : 0); i += THREADS) {
                const int row = i / NFP, n = i - row * NFP;
                const int e = row / 60, f = (row / 15) & 3, r = row % 15;
                const int code = sCode[e * 4 + f];
                sQf[row * NFPP + n] = sQ[(e * 15 + r) * NPP + sFmask[f * NFP + n]];
                if (code3_bc(code) == 0) {
                    const long long nb = sNbr[e * 4 + f];
                    sQn[row * NFPP + n] = p.q[nb * 15 * NP + r * NP + sFmask[code3_face(code) * NFP + n]];
                }
            }
        }
        // ---- phase 1: cubature-point fluxes
        for (int i = tid; i < ne * NQ; i += THREADS) {
            const int e = i / NQ, q = i - e * NQ;
            const Real* ue = sU + e * 5 * NPP;
            Real u[5] = {0, 0, 0, 0, 0};
            Real qc[MODE == 1 ? 15 : 1];   // q at the point (viscous stage)
#pragma unroll
            for (int r = 0; r < (MODE == 1 ? 15 : 1); ++r) qc[r] = Real(0);
#pragma unroll 2
            for (int jb = 0; jb < NPP / 4; ++jb) {
                const V4<Real> w = ldg4(IcubB + (jb * NQP + q) * 4);
#pragma unroll
                for (int v = 0; v < 5; ++v) u[v] += dot4(w, lds4(ue + v * NPP + 4 * jb));
                if constexpr (MODE == 1) {
                    if (visc) {
#pragma unroll
                        for (int r = 0; r < 15; ++r) qc[r] += dot4(w, lds4(sQ + (e * 15 + r) * NPP + 4 * jb));
                    }
                }
            }
            Real cof[9];
            const long long eg = e0 + e;
            if (eg < p.Kaff) {
#pragma unroll
                for (int k = 0; k < 9; ++k) cof[k] = sG[e * 16 + k];
            } else {
                const Real* gc = p.geoC + (eg - p.Kaff) * CS;
#pragma unroll
                for (int k = 0; k < 9; ++k) cof[k] = gc[k * NQ + q];
            }
            if constexpr (MODE == 2) {
                // the gradient pass: the flux vector delta_dm sqrt(eps) U,
                // contravariant (J dr_a/dx_m) sqrt(eps) U
                const Real se = sSe[e * 5];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const Real c = cof[3 * p.grad_m + a] * se;
                    Real* out = sF + (e * 3 + a) * TT::FST + q;
#pragma unroll
                    for (int v = 0; v < 5; ++v) out[v * NQP] = c * u[v];
                }
            } else {
                const Real ir = recip(u[0]);
                const Real vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
                const Real pr = (p.gamma - Real(1)) * (u[4] - Real(0.5) * (u[1] * vx + u[2] * vy + u[3] * vz));
                const Real H = u[4] + pr;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    // contravariant velocity and pressure direction for direction a
                    const Real c0 = cof[a], c1 = cof[3 + a], c2 = cof[6 + a];
                    const Real U = c0 * vx + c1 * vy + c2 * vz;
                    Real f[5] = {u[0] * U, u[1] * U + pr * c0, u[2] * U + pr * c1, u[3] * U + pr * c2, H * U};
                    if constexpr (MODE == 1) {   // minus sqrt(eps) q in the physical fluxes
                        if (visc) {
                            const Real se = sSe[e * 5];
#pragma unroll
                            for (int v = 0; v < 5; ++v)
                                f[v] -= se * (c0 * qc[v] + c1 * qc[5 + v] + c2 * qc[10 + v]);
                        }
                    }
                    Real* out = sF + (e * 3 + a) * TT::FST + q;
#pragma unroll
                    for (int v = 0; v < 5; ++v) out[v * NQP] = f[v];
                }
            }
        }
        __syncthreads();
        // ---- phase 2: volume term; one direction a and two nodes per item
        const int n2 = 3 * ne * NH;
        for (int i = tid; i < n2; i += THREADS) {
            const int n = i % NH, rest = i / NH, e = rest % ne, a = rest / ne;
            const int m = n + NH < NP ? n + NH : n;
            const Real* DB = p.ops + (a == 0 ? L.drw : a == 1 ? L.dsw : L.dtw);
            const Real* fa = sF + (e * 3 + a) * TT::FST;
            Real acc0[5] = {0, 0, 0, 0, 0}, acc1[5] = {0, 0, 0, 0, 0};
#pragma unroll 2
            for (int qb = 0; qb < NQP / 4; ++qb) {
                const V4<Real> d0 = ldg4(DB + (qb * NPP + n) * 4);
                const V4<Real> d1 = ldg4(DB + (qb * NPP + m) * 4);
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const V4<Real> f = lds4(fa + v * NQP + 4 * qb);
                    acc0[v] += dot4(d0, f);
                    acc1[v] += dot4(d1, f);
                }
            }
            Real* out = sR + (a * E + e) * 5 * NP;
#pragma unroll
            for (int v = 0; v < 5; ++v) out[v * NP + n] = acc0[v];
            if (n + NH < NP) {
#pragma unroll
                for (int v = 0; v < 5; ++v) out[v * NP + m] = acc1[v];
            }
        }
        // ---- phase 3: face-frame points (first on the threads phase 2 left idle)
        if (MODE == 1 && !visc)
            face_points3<N, Real, 16, 0, 0>(p, e0, ne, (tid + THREADS - n2 % THREADS) % THREADS, sI2, sW, sUf, sNb,
                                             sCode, sG, nullptr, sFs);
        else
            face_points3<N, Real, 16, 0, MODE>(p, e0, ne, (tid + THREADS - n2 % THREADS) % THREADS, sI2, sW, sUf,
                                               sNb, sCode, sG, nullptr, sFs, sSe, sQf, sQn, p.grad_m);
        __syncthreads();
        // ---- phase 4a: lift of each face's flux to its face nodes
        lift3<N, Real>(ne, sI2T, sFs, sCode, sT);
        __syncthreads();
        // ---- phase 4b: R = vol - surf
        combine3<N, Real, 3>(ne, E * 5 * NP, sT, sFpos, sR);
        __syncthreads();
        // ---- phase 5: inverse mass and the stage update (the gradient
        // pass: q_m = -M^-1 R into its rows of q)
        if constexpr (MODE == 2) {
            for (int i = tid; i < ne * 5 * NP; i += THREADS) {
                const int e = i / (5 * NP), r = i - e * 5 * NP, v = r / NP, n = r - v * NP;
                const Real* rr = sR + (e * 5 + v) * NP;
                const long long eg = e0 + e;
                Real Lv = 0;
                if (eg < p.Kaff) {
                    for (int j = 0; j < NP; ++j) Lv += sMiT[j * NP + n] * rr[j];
                    Lv *= sG[e * 16 + 9];
                } else {
                    const Real* mi = p.geoC + (eg - p.Kaff) * CS + 9 * NQ + 16 * NG;
                    for (int j = 0; j < NP; ++j) Lv += mi[j * NP + n] * rr[j];
                }
                p.qout[eg * 15 * NP + (p.grad_m * 5 + v) * NP + n] = -Lv;
            }
        } else {
            update3<N, Real, 16>(p, e0, ne, sR, sMiT, sG, sU);
        }
    }
}

// The element sensor (paper Sec. 2): S_k = the L2 norm of the density's
// highest-degree modes over that of the density, both by the cubature rule
// with J (J = sqrt(det(cofactors)) at the points of a curved element; a
// constant that cancels on an affine one); s_k = log10 S_k and the sine ramp
// of width kappa around s0 up to eps0.  One warp per element; the two sums
// in the real type, the ratio, logarithm and ramp in FP64.
template <int N, typename Real>
__global__ void __launch_bounds__(256) sensor3_kernel(const Real* U, Real* eps, const Real* ops, const Real* av,
                                                       const Real* geoC, long long K, long long Kaff, double kappa,
                                                       double eps0, double s0) {
    constexpr int NP = np3_of(N), NQ = nq3_of(N), NPP = pad4(NP), NQP = pad4(NQ);
    constexpr Ops3Layout L = ops3_layout(N);
    constexpr int CS = curved3_stride(N);
    __shared__ __align__(16) Real sr[8][2][NPP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = NP + lane; j < NPP; j += 32) sr[warp][0][j] = sr[warp][1][j] = Real(0);
    const Real* Fh = av;
    const Real* wq = av + NP * NP;
    for (long long e = (long long)blockIdx.x * 8 + warp; e < K; e += (long long)gridDim.x * 8) {
        for (int j = lane; j < NP; j += 32) sr[warp][0][j] = U[e * 5 * NP + j];
        __syncwarp();
        for (int i = lane; i < NP; i += 32) {
            Real h = 0;
            for (int j = 0; j < NP; ++j) h += Fh[i * NP + j] * sr[warp][0][j];
            sr[warp][1][i] = h;
        }
        __syncwarp();
        Real num = 0, den = 0;
        for (int q = lane; q < NQ; q += 32) {
            Real a = 0, b = 0;
#pragma unroll
            for (int jb = 0; jb < NPP / 4; ++jb) {
                const V4<Real> w = ldg4(ops + L.icub + (jb * NQP + q) * 4);
                a += dot4(w, lds4(&sr[warp][0][4 * jb]));
                b += dot4(w, lds4(&sr[warp][1][4 * jb]));
            }
            Real wj = wq[q];
            if (e >= Kaff) {
                const Real* c = geoC + (e - Kaff) * CS + q;
                const Real c0 = c[0], c1 = c[NQ], c2 = c[2 * NQ], c3 = c[3 * NQ], c4 = c[4 * NQ], c5 = c[5 * NQ];
                const Real c6 = c[6 * NQ], c7 = c[7 * NQ], c8 = c[8 * NQ];
                const Real det = c0 * (c4 * c8 - c5 * c7) - c1 * (c3 * c8 - c5 * c6) + c2 * (c3 * c7 - c4 * c6);
                wj *= sqrt(det);
            }
            num += wj * b * b;
            den += wj * a * a;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (lane == 0) {
            double ev = 0.0;
            const double nm = (double)num, dn = (double)den;
            if (nm > 0.0 && dn > 0.0) {
                const double sk = log10(nm / dn);
                if (sk > s0 + kappa)
                    ev = eps0;
                else if (sk >= s0 - kappa)
                    ev = 0.5 * eps0 * (1.0 + sin(3.141592653589793 * (sk - s0) / (2.0 * kappa)));
            }
            eps[e] = (Real)ev;
        }
        __syncwarp();
    }
}

template <int N, typename Real>
int launch_sensor_t(const Real* U, Real* eps, const Real* ops, const Real* av, const Real* geoC, long long K,
                    long long Kaff, double kappa, double eps0, double s0, cudaStream_t st) {
    if (K <= 0) return 0;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int g = (int)std::min<long long>((K + 7) / 8, (long long)nsm * 8);
    sensor3_kernel<N, Real><<<g, 256, 0, st>>>(U, eps, ops, av, geoC, K, Kaff, kappa, eps0, s0);
    return (int)cudaGetLastError();
}

template <int N, typename Real, int MODE>
int prepare_mode() {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, stage3_kernel<N, Real, MODE>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stage3_kernel<N, Real, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(SMEM3_MAX - fa.sharedSizeBytes));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    return 0;
}

template <int N, typename Real>
int prepare_t(void) {
    int e = prepare_mode<N, Real, 0>();
    if (!e) e = prepare_mode<N, Real, 1>();
    if (!e) e = prepare_mode<N, Real, 2>();
    return e;
}

template <int N, typename Real, int MODE>
int launch_mode(const StageArgs3<Real>& a, cudaStream_t st) {
    int E = a.tile_e > 0 ? a.tile_e : T3<N, Real>::default_e();
    // the viscous layout is larger: the largest tile not above the chosen one that fits
    while (E > 1 && T3<N, Real>(E, MODE).bytes > SMEM3_MAX) --E;
    const size_t bytes = T3<N, Real>(E, MODE).bytes;
    if (bytes > SMEM3_MAX) return (int)cudaErrorInvalidValue;
    if (MODE != 0 && (!a.eps || (MODE == 1 && !a.q) || (MODE == 2 && !a.qout))) return (int)cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int occ = std::max(1, resident_ctas((const void*)stage3_kernel<N, Real, MODE>, THREADS, bytes));
    const long long ntiles = (a.K + E - 1) / E;
    const int g = (int)std::min<long long>(ntiles, (long long)nsm * occ);
    if (g <= 0) return 0;
    StageArgs3<Real> b = a;
    b.tile_e = E;
    stage3_kernel<N, Real, MODE><<<g, THREADS, bytes, st>>>(b);
    return (int)cudaGetLastError();
}

template <int N, typename Real>
int launch_t(const StageArgs3<Real>& a, cudaStream_t st, int mode) {
    return mode == 1 ? launch_mode<N, Real, 1>(a, st) : mode == 2 ? launch_mode<N, Real, 2>(a, st)
                                                                    : launch_mode<N, Real, 0>(a, st);
}

template <int N, typename Real>
bool fits_t(int E) {
    return E >= 1 && T3<N, Real>(E).bytes <= SMEM3_MAX;
}

}  // namespace

bool supported_degree3(int N) { return N >= 2 && N <= 4; }

int tile3_default(int N, int rsize) {
    if (rsize == 8) return N == 2 ? T3<2, double>::default_e() : N == 3 ? T3<3, double>::default_e()
                                                                          : T3<4, double>::default_e();
    return N == 2 ? T3<2, float>::default_e() : N == 3 ? T3<3, float>::default_e() : T3<4, float>::default_e();
}

bool tile3_fits(int N, int rsize, int E) {
    if (rsize == 8) return N == 2 ? fits_t<2, double>(E) : N == 3 ? fits_t<3, double>(E) : fits_t<4, double>(E);
    return N == 2 ? fits_t<2, float>(E) : N == 3 ? fits_t<3, float>(E) : fits_t<4, float>(E);
}

int prepare_stage3(int N, int rsize) {
    if (rsize == 8) return N == 2 ? prepare_t<2, double>() : N == 3 ? prepare_t<3, double>() : prepare_t<4, double>();
    return N == 2 ? prepare_t<2, float>() : N == 3 ? prepare_t<3, float>() : prepare_t<4, float>();
}

int launch_stage3(int N, const StageArgs3<float>& a, cudaStream_t st, int mode) {
    return N == 2 ? launch_t<2, float>(a, st, mode) : N == 3 ? launch_t<3, float>(a, st, mode)
                                                             : launch_t<4, float>(a, st, mode);
}

int launch_stage3(int N, const StageArgs3<double>& a, cudaStream_t st, int mode) {
    return N == 2 ? launch_t<2, double>(a, st, mode) : N == 3 ? launch_t<3, double>(a, st, mode)
                                                              : launch_t<4, double>(a, st, mode);
}

}  // namespace dgc

namespace dgc {

int launch_sensor3(int N, const float* U, float* eps, const float* ops, const float* ops_av, const float* geoC,
                   long long K, long long Kaff, double kappa, double eps0, double s0, cudaStream_t st) {
    return N == 2 ? launch_sensor_t<2, float>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st)
         : N == 3 ? launch_sensor_t<3, float>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st)
                  : launch_sensor_t<4, float>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st);
}

int launch_sensor3(int N, const double* U, double* eps, const double* ops, const double* ops_av,
                   const double* geoC, long long K, long long Kaff, double kappa, double eps0, double s0,
                   cudaStream_t st) {
    return N == 2 ? launch_sensor_t<2, double>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st)
         : N == 3 ? launch_sensor_t<3, double>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st)
                  : launch_sensor_t<4, double>(U, eps, ops, ops_av, geoC, K, Kaff, kappa, eps0, s0, st);
}

}  // namespace dgc

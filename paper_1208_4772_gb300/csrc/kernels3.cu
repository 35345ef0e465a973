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
    int O_F, O_UF, O_NB, O_FS, O_T, O_R, O_G, O_END;
    size_t bytes;
    __host__ __device__ constexpr explicit T3(int E)
        : O_F(O_U + E * 5 * NPP),          // [E][3][FST] contravariant fluxes
          O_UF(O_F + E * 3 * FST),         // [E][4][5][NFPP] own face nodes
          O_NB(O_UF + E * 20 * NFPP),      // [E][4][5][NFPP] neighbours' face nodes
          O_FS(O_NB + E * 20 * NFPP),      // [E][4][5][NGP] w sJ F*
          O_T(O_FS + E * 20 * NGP),        // [E][4][5][NFPP] lifted face terms
          O_R(O_T + E * 20 * NFPP),        // [3][E][5][NP] volume parts, then R
          O_G(O_R + 3 * E * 5 * NP),       // [E][16] affine cofactors, 1/J
          O_END(O_G + E * 16),
          bytes((size_t)O_END * sizeof(Real) + (size_t)(4 * NFP + 4 * NP + 8 * E) * sizeof(int)) {}
    static constexpr int default_e() { return sizeof(Real) == 4 ? (N <= 2 ? 8 : N == 3 ? 4 : 2) : (N <= 2 ? 4 : N == 3 ? 2 : 1); }
};

// Largest dynamic shared memory of one CTA.
constexpr size_t SMEM3_MAX = 232448;

template <int N, typename Real>
__global__ void __launch_bounds__(THREADS) stage3_kernel(const StageArgs3<Real> p) {
    using TT = T3<N, Real>;
    constexpr int NP = TT::NP, NFP = TT::NFP, NQ = TT::NQ, NG = TT::NG, NPP = TT::NPP, NQP = TT::NQP;
    constexpr int NFPP = TT::NFPP, NGP = TT::NGP, NH = (NP + 1) / 2;
    const int E = p.tile_e;
    const TT T(E);
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
    int* sFmask = reinterpret_cast<int*>(S + T.O_END);
    int* sFpos = sFmask + 4 * NFP;
    int* sNbr = sFpos + 4 * NP;
    int* sCode = sNbr + 4 * E;
    const int tid = threadIdx.x;
    const Real* __restrict__ IcubB = p.ops + L.icub;

    // the padding of the state, flux, face-node and face-flux rows stays zero
    for (int i = tid; i < T.O_T - TT::O_U; i += THREADS) sU[i] = Real(0);
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
        }
        for (int e = tid; e < ne; e += THREADS) {
            if (e0 + e >= p.Kaff) continue;
            affine_cofactors3(p.geoA + (e0 + e) * 9, sG + e * 16);
        }
        __syncthreads();
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
        // ---- phase 1: cubature-point fluxes
        for (int i = tid; i < ne * NQ; i += THREADS) {
            const int e = i / NQ, q = i - e * NQ;
            const Real* ue = sU + e * 5 * NPP;
            Real u[5] = {0, 0, 0, 0, 0};
#pragma unroll 2
            for (int jb = 0; jb < NPP / 4; ++jb) {
                const V4<Real> w = ldg4(IcubB + (jb * NQP + q) * 4);
#pragma unroll
                for (int v = 0; v < 5; ++v) u[v] += dot4(w, lds4(ue + v * NPP + 4 * jb));
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
            const Real ir = recip(u[0]);
            const Real vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
            const Real pr = (p.gamma - Real(1)) * (u[4] - Real(0.5) * (u[1] * vx + u[2] * vy + u[3] * vz));
            const Real H = u[4] + pr;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // contravariant velocity and pressure direction for direction a
                const Real c0 = cof[a], c1 = cof[3 + a], c2 = cof[6 + a];
                const Real U = c0 * vx + c1 * vy + c2 * vz;
                Real* out = sF + (e * 3 + a) * TT::FST + q;
                out[0] = u[0] * U;
                out[NQP] = u[1] * U + pr * c0;
                out[2 * NQP] = u[2] * U + pr * c1;
                out[3 * NQP] = u[3] * U + pr * c2;
                out[4 * NQP] = H * U;
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
        face_points3<N, Real, 16, 0>(p, e0, ne, (tid + THREADS - n2 % THREADS) % THREADS, sI2, sW, sUf, sNb, sCode,
                                  sG, nullptr, sFs);
        __syncthreads();
        // ---- phase 4a: lift of each face's flux to its face nodes
        lift3<N, Real>(ne, sI2T, sFs, sCode, sT);
        __syncthreads();
        // ---- phase 4b: R = vol - surf
        combine3<N, Real, 3>(ne, E * 5 * NP, sT, sFpos, sR);
        __syncthreads();
        // ---- phase 5: inverse mass and the stage update
        update3<N, Real, 16>(p, e0, ne, sR, sMiT, sG, sU);
    }
}

template <int N, typename Real>
int prepare_t(void) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, stage3_kernel<N, Real>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stage3_kernel<N, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(SMEM3_MAX - fa.sharedSizeBytes));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    return 0;
}

template <int N, typename Real>
int launch_t(const StageArgs3<Real>& a, cudaStream_t st) {
    const int E = a.tile_e > 0 ? a.tile_e : T3<N, Real>::default_e();
    const size_t bytes = T3<N, Real>(E).bytes;
    if (bytes > SMEM3_MAX) return (int)cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int occ = std::max(1, resident_ctas((const void*)stage3_kernel<N, Real>, THREADS, bytes));
    const long long ntiles = (a.K + E - 1) / E;
    const int g = (int)std::min<long long>(ntiles, (long long)nsm * occ);
    if (g <= 0) return 0;
    StageArgs3<Real> b = a;
    b.tile_e = E;
    stage3_kernel<N, Real><<<g, THREADS, bytes, st>>>(b);
    return (int)cudaGetLastError();
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

int launch_stage3(int N, const StageArgs3<float>& a, cudaStream_t st) {
    return N == 2 ? launch_t<2, float>(a, st) : N == 3 ? launch_t<3, float>(a, st) : launch_t<4, float>(a, st);
}

int launch_stage3(int N, const StageArgs3<double>& a, cudaStream_t st) {
    return N == 2 ? launch_t<2, double>(a, st) : N == 3 ? launch_t<3, double>(a, st) : launch_t<4, double>(a, st);
}

}  // namespace dgc

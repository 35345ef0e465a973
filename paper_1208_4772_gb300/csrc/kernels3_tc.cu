// Stage kernel of the tetrahedral method (paper Sec. 2 with d = 3) with the
// two volume products on the tensor cores (tcgen05, kind::tf32, FP32
// accumulate in TMEM); the face terms, the inverse mass and the stage
// update run on the CUDA cores as in the FP32 kernel.
//
// A tile holds E elements; the rows of both products are the tile's
// (element, variable) pairs, r = 5 e + v (5 E <= 128 = M; the rows past 5 E
// are not held in shared memory and their results are never read).
//   G1  D1 = A1 B1^T: A1 = the state minus its element mean (exact: the rows
//       of I_cub sum to one), B1 = I_cub -> the state at all cubature points.
//   per chunk of QC cubature points (one point of one element per thread):
//       the contravariant flux deviations sum_d (J dr_a/dx_d)(F_d(U) -
//       F_d(Ubar)), Ubar the element mean, written as A2 (K = 3 QC);
//   G2  D2 += A2 B2^T, B2 = [D_r^T W, D_s^T W, D_t^T W] of the chunk.
// The face terms subtract the normal flux of the same mean state, so that
// the subtracted constant flux cancels between the volume and face terms
// (the discrete divergence of a constant flux vanishes, for affine and
// curved elements alike: both integrands are polynomials the rules
// integrate exactly) and the TF32 products act on small deviations only.
//
// Shared-memory operand layout: K-major, no swizzle, 8-row x 16-byte core
// matrices.  I_cub keeps the usual order (core matrices adjacent along K);
// the tile operands and B2 are stored with their 8-row groups adjacent and
// the K columns of core matrices G x 128 bytes apart, so that the row
// groups past the ones held read neighbouring data instead of memory past
// the buffer.  Each CTA is persistent over a static tile schedule; every
// mbarrier wait is bounded and a wait that runs out sets bit 16 of the
// mesh's error word and ends the CTA's work.
#include <algorithm>

#include "kernels3.cuh"
#include "tc_ptx.cuh"

namespace dgc {

namespace {

template <int N>
struct TC3 {
    static constexpr int NP = np3_of(N), NQ = nq3_of(N), NG = ng3_of(N), NFP = nfp3_of(N);
    static constexpr int NPP = pad4(NP), NQP = pad4(NQ), NFPP = pad4(NFP), NGP = pad4(NG);
    static constexpr int E = N == 2 ? 16 : 8;           // elements per tile
    static constexpr int QC = THREADS / E;              // cubature points per chunk: one flux per thread
    static constexpr int NQT = (NQ + QC - 1) / QC * QC; // cubature points padded to whole chunks
    static constexpr int NCH = NQT / QC;
    static constexpr int ROWS = 5 * E;                  // (element, variable) rows
    static constexpr int RG = ROWS / 8;                 // 8-row groups of the tile operands held
    static constexpr int QU = (ROWS + 31) / 32;         // TMEM lane quarters holding rows
    static constexpr int NPK = (NP + 7) / 8 * 8;        // G1 summation length
    static constexpr int NPN = (NP + 15) / 16 * 16;     // G2 result columns (the MMA's N)
    static constexpr int BG = (NP + 7) / 8;             // 8-row groups of B2 held
    static constexpr int KC = 3 * QC;                   // G2 summation length per chunk
    static constexpr int TMEM_COLS = NQT + NPN <= 128 ? 128 : 256;
    static constexpr int GST = 17;                      // reals per element: cofactors, 1/J
    static constexpr int BST = 11;                      // reals per element: mean state data
    static constexpr int LBO_A = RG * 128, LBO_B2 = BG * 128;
    static constexpr int al(int x) { return (x + 127) / 128 * 128; }
    static constexpr int mx(int a, int b) { return a > b ? a : b; }
    // byte offsets in dynamic shared memory; constant region first
    static constexpr int O_B1 = 0;                                        // [NQT][NPK], LBO 128
    static constexpr int O_B2 = al(O_B1 + NQT * NPK * 4);                 // 3 NQT / 4 columns x BG groups
    static constexpr int O_I2 = al(O_B2 + 3 * NQT / 4 * LBO_B2);          // [6][NG][NFPP]
    static constexpr int O_I2T = O_I2 + 6 * NG * NFPP * 4;                // [6][NFP][NGP]
    static constexpr int O_W = O_I2T + 6 * NFP * NGP * 4;                 // [NGP]
    static constexpr int O_MI = O_W + NGP * 4;                            // [NP][NP]
    static constexpr int O_FM = al(O_MI + NP * NP * 4);                   // fmask [4][NFP], fpos [4][NP]
    // per-tile region
    static constexpr int O_U = al(O_FM + (4 * NFP + 4 * NP) * 4);         // [E][5][NPP]
    static constexpr int O_NB = al(O_U + E * 5 * NPP * 4);                // [E][4][5][NFPP]
    static constexpr int O_R = al(O_NB + E * 20 * NFPP * 4);              // [E][5][NP]
    static constexpr int O_G = al(O_R + E * 5 * NP * 4);                  // [E][GST]
    static constexpr int O_BAR = O_G + E * GST * 4;                       // [E][BST]
    static constexpr int O_NBR = O_BAR + E * BST * 4;                     // int [E][4]
    static constexpr int O_CODE = O_NBR + E * 4 * 4;                      // int [E][4]
    // the next tile's inputs, copied asynchronously during this tile
    static constexpr int O_SC = al(O_CODE + E * 4 * 4);                   // int4 [E] neighbours
    static constexpr int O_SK = O_SC + E * 16;                            // int2 [E] face codes
    static constexpr int O_SG = O_SK + E * 8;                             // [E][9] dx/dr (affine)
    static constexpr int O_SU = al(O_SG + E * 9 * 4);                     // [E][5][NP] state rows
    // the volume operands, then (same storage) the face arrays
    static constexpr int O_A1 = al(O_SU + E * 5 * NP * 4);                // NPK / 4 columns x RG groups
    static constexpr int O_A2 = al(O_A1 + NPK / 4 * LBO_A);               // KC / 4 columns x RG groups
    static constexpr int O_UQ = al(O_A2 + KC / 4 * LBO_A);                // [2][QC][ROWS]
    static constexpr int VOL_END = O_UQ + 2 * QC * ROWS * 4;
    static constexpr int O_UF = O_A1;                                     // [E][4][5][NFPP], then the lifted terms
    static constexpr int O_FS = al(O_UF + E * 20 * NFPP * 4);             // [E][4][5][NGP]
    static constexpr int FACE_END = O_FS + E * 20 * NGP * 4;
    static constexpr int TOTAL = al(mx(VOL_END, FACE_END));
    static_assert(ROWS % 8 == 0 && ROWS <= 128 && E * QC == THREADS, "tile shape");
    static_assert(NQT <= 256 && NQT % 16 == 0 && NPN <= 256, "MMA shapes");
    static_assert(NQT + NPN <= TMEM_COLS, "TMEM columns");
    // the row groups past RG (A operands) and past BG (B2) read the bytes
    // that follow the buffer's last column: keep them inside the allocation
    static_assert(O_A1 + NPK / 4 * LBO_A + (16 - RG) * 128 <= TOTAL &&
                  O_A2 + KC / 4 * LBO_A + (16 - RG) * 128 <= TOTAL, "operand tails");
    static_assert(O_I2 - O_B2 - 3 * NQT / 4 * LBO_B2 + 6 * NG * NFPP * 4 >= (NPN / 8 - BG) * 128, "B2 tail");
};

constexpr size_t SMEM3TC_MAX = 232448 - 1024;

// Byte offset of (row, k) of a 4-byte operand whose 8-row groups are
// adjacent (128 B apart) and whose columns of core matrices along K are lbo
// bytes apart.
__device__ __forceinline__ uint32_t il_offset(int row, int k, int lbo) {
    return (uint32_t)((k >> 2) * lbo + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

template <int N>
__global__ void __launch_bounds__(THREADS, 2) stage3_tc_kernel(const StageArgs3<float> p) {
    using C = TC3<N>;
    constexpr int NP = C::NP, NQ = C::NQ, NG = C::NG, NFP = C::NFP, NPP = C::NPP, NQP = C::NQP;
    constexpr int NFPP = C::NFPP, NGP = C::NGP, E = C::E, QC = C::QC, ROWS = C::ROWS;
    constexpr int GST = C::GST, BST = C::BST;
    constexpr Ops3Layout L = ops3_layout(N);
    constexpr int CS = curved3_stride(N);
    extern __shared__ __align__(128) unsigned char sm3[];
    __shared__ uint64_t bars[3];   // G1 complete, G2 chunk complete, final drain
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    float* sI2 = reinterpret_cast<float*>(sm3 + C::O_I2);
    float* sI2T = reinterpret_cast<float*>(sm3 + C::O_I2T);
    float* sW = reinterpret_cast<float*>(sm3 + C::O_W);
    float* sMiT = reinterpret_cast<float*>(sm3 + C::O_MI);
    int* sFmask = reinterpret_cast<int*>(sm3 + C::O_FM);
    int* sFpos = sFmask + 4 * NFP;
    float* sU = reinterpret_cast<float*>(sm3 + C::O_U);
    float* sNb = reinterpret_cast<float*>(sm3 + C::O_NB);
    float* sR = reinterpret_cast<float*>(sm3 + C::O_R);
    float* sG = reinterpret_cast<float*>(sm3 + C::O_G);
    float* sBar = reinterpret_cast<float*>(sm3 + C::O_BAR);
    int* sNbr = reinterpret_cast<int*>(sm3 + C::O_NBR);
    int* sCode = reinterpret_cast<int*>(sm3 + C::O_CODE);
    float* sUq = reinterpret_cast<float*>(sm3 + C::O_UQ);
    float* sUf = reinterpret_cast<float*>(sm3 + C::O_UF);   // then the lifted face terms
    float* sFs = reinterpret_cast<float*>(sm3 + C::O_FS);
    int4* sSC = reinterpret_cast<int4*>(sm3 + C::O_SC);
    int2* sSK = reinterpret_cast<int2*>(sm3 + C::O_SK);
    float* sSG = reinterpret_cast<float*>(sm3 + C::O_SG);
    float* sSU = reinterpret_cast<float*>(sm3 + C::O_SU);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = (p.K + E - 1) / E;
    // a tile's rows, neighbours, codes and affine dx/dr into the staging
    // buffers by asynchronous copies (waited for at the top of that tile)
    auto prefetch = [&](long long t) {
        if (t >= ntiles) return;
        const long long f0 = t * E;
        const int nf = (int)min((long long)E, p.K - f0);
        const float* su = p.Us + f0 * 5 * NP;
        for (int i = tid; i < nf * 5 * NP; i += THREADS) tc::cp_async4(sSU + i, su + i);
        for (int i = tid; i < nf; i += THREADS) {
            tc::cp_async16(sSC + i, p.conn + f0 + i);
            tc::cp_async4(reinterpret_cast<int*>(sSK + i), reinterpret_cast<const int*>(p.code + f0 + i));
            tc::cp_async4(reinterpret_cast<int*>(sSK + i) + 1, reinterpret_cast<const int*>(p.code + f0 + i) + 1);
        }
        const int naff = (int)max(0LL, min((long long)nf, p.Kaff - f0));
        for (int i = tid; i < naff * 9; i += THREADS) tc::cp_async4(sSG + i, p.geoA + f0 * 9 + i);
    };

    prefetch(blockIdx.x);
    // operators: B1 = I_cub (rows q, K = j), B2 = the three D_a^T W (rows n,
    // K = (chunk, direction, point)), rounded to TF32, zero padding
    for (int i = tid; i < C::NQT * C::NPK; i += THREADS) {
        const int q = i / C::NPK, j = i - q * C::NPK;
        const float v = (q < NQ && j < NP) ? p.ops[L.icub + ((j >> 2) * NQP + q) * 4 + (j & 3)] : 0.f;
        *reinterpret_cast<float*>(sm3 + C::O_B1 + tc::cm_offset(q, j * 4, C::NPK * 4)) = tc::to_tf32(v);
    }
    for (int i = tid; i < C::BG * 8 * 3 * C::NQT; i += THREADS) {
        const int n = i / (3 * C::NQT), kk = i - n * 3 * C::NQT;
        const int c = kk / C::KC, rem = kk - c * C::KC, a = rem / QC, q = c * QC + rem - a * QC;
        const float* D = p.ops + (a == 0 ? L.drw : a == 1 ? L.dsw : L.dtw);
        const float v = (n < NP && q < NQ) ? D[((q >> 2) * NPP + n) * 4 + (q & 3)] : 0.f;
        *reinterpret_cast<float*>(sm3 + C::O_B2 + il_offset(n, kk, C::LBO_B2)) = tc::to_tf32(v);
    }
    for (int i = tid; i < 6 * NG * NFPP + 6 * NFP * NGP; i += THREADS) sI2[i] = p.ops[L.i2 + i];
    for (int i = tid; i < NGP; i += THREADS) sW[i] = i < NG ? p.ops[L.wg + i] : 0.f;
    for (int i = tid; i < NP * NP; i += THREADS) sMiT[i] = p.ops[L.mi + i];
    for (int i = tid; i < 4 * NFP + 4 * NP; i += THREADS) sFmask[i] = p.opsi[i];
    for (int i = tid; i < E * 20 * NFPP; i += THREADS) sNb[i] = 0.f;
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_init(&bars[2], 1);
        tc::mbar_fence_init();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, C::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem, tD1 = tmem, tD2 = tmem + C::NQT;
    const int quad = warp & 3, half = warp >> 2, row = 32 * quad + lane;
    const uint32_t lanes = (uint32_t)(32 * quad) << 16;
    const uint32_t idesc1 = tc::instr_desc(2, 128, C::NQT), idesc2 = tc::instr_desc(2, 128, C::NPN);
    const uint32_t aA1 = tc::smem_addr(sm3 + C::O_A1), aA2 = tc::smem_addr(sm3 + C::O_A2);
    const uint32_t aB1 = tc::smem_addr(sm3 + C::O_B1), aB2 = tc::smem_addr(sm3 + C::O_B2);
    uint32_t ph1 = 0, ph2 = 0;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long e0 = tile * E;
        const int ne = (int)min((long long)E, p.K - e0);
        tc::cp_async_wait_all();
        __syncthreads();
        if (s_abort) break;
        // ---- rows, codes, affine cofactors from the staging buffers
        for (int i = tid; i < ne * 5 * NP; i += THREADS) {
            const int r = i / NP;
            sU[r * NPP + (i - r * NP)] = sSU[i];
        }
        for (int i = tid; i < ne * 4; i += THREADS) {
            const int e = i >> 2, f = i & 3;
            const int4 nb = sSC[e];
            const int2 cw = sSK[e];
            sNbr[i] = f == 0 ? nb.x : f == 1 ? nb.y : f == 2 ? nb.z : nb.w;
            sCode[i] = ((f < 2 ? cw.x : cw.y) >> (16 * (f & 1))) & 0xffff;
        }
        for (int e = tid; e < ne; e += THREADS)
            if (e0 + e < p.Kaff) affine_cofactors3(sSG + e * 9, sG + e * GST);
        __syncthreads();
        // ---- the next tile's inputs and this tile's neighbour face-node
        // values (waited for before the face terms) by asynchronous copies;
        // element means (rows past the tile: a unit state)
        prefetch(tile + gridDim.x);
        for (int i = tid; i < ne * 20 * NFP; i += THREADS) {
            const int rw = i / NFP, n = i - rw * NFP;   // rw = (e * 4 + f) * 5 + v
            const int e = rw / 20, f = (rw / 5) & 3, v = rw % 5;
            const int code = sCode[e * 4 + f];
            if (code3_bc(code) == 0) {
                const long long nb = sNbr[e * 4 + f];
                tc::cp_async4(sNb + rw * NFPP + n, p.Us + nb * 5 * NP + v * NP + sFmask[code3_face(code) * NFP + n]);
            }
        }
        if (tid < ROWS) {
            const int e = tid / 5, v = tid - 5 * e;
            float m = (v == 0 || v == 4) ? 1.f : 0.f;
            if (e < ne) {
                m = 0.f;
#pragma unroll
                for (int j = 0; j < NP; ++j) m += sU[tid * NPP + j];
                m *= 1.f / NP;
            }
            sBar[e * BST + v] = m;
        }
        __syncthreads();
        // ---- A1 = TF32(U - Ubar); the mean state's velocity, pressure, enthalpy
        for (int i = tid; i < ROWS * C::NPK; i += THREADS) {
            const int r = i / C::NPK, j = i - r * C::NPK, e = r / 5;
            const float v = (e < ne && j < NP) ? sU[r * NPP + j] - sBar[e * BST + r - 5 * e] : 0.f;
            *reinterpret_cast<float*>(sm3 + C::O_A1 + il_offset(r, j, C::LBO_A)) = tc::to_tf32(v);
        }
        if (tid < E) {
            float* b = sBar + tid * BST;
            const float ir = 1.f / b[0];
            b[5] = b[1] * ir;
            b[6] = b[2] * ir;
            b[7] = b[3] * ir;
            b[8] = (p.gamma - 1.f) * (b[4] - 0.5f * (b[1] * b[5] + b[2] * b[6] + b[3] * b[7]));
            b[9] = b[4] + b[8];
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {   // G1: the state at every cubature point
            tc::fence_after_sync();
            for (int ks = 0; ks < C::NPK / 8; ++ks)
                tc::mma_tf32(tD1, tc::smem_desc(aA1 + ks * 2 * C::LBO_A, (uint32_t)C::LBO_A, 128u),
                             tc::smem_desc(aB1 + ks * 256, (uint32_t)(C::NPK * 4)), idesc1, ks > 0 ? 1u : 0u);
            tc::mma_commit(&bars[0]);
        }
        bool ok = tc::mbar_wait(&bars[0], ph1 & 1);
        ph1++;
        tc::fence_after_sync();
        // ---- a chunk's states at its cubature points (plus the mean) to
        // sUq[b] [QC][ROWS], by the warps whose TMEM lanes hold rows; the two
        // halves of the CTA take half the columns each
        auto readout = [&](int c, float* dst) {
            if (quad < C::QU) {
                constexpr int HC = QC / 2;
                float x[HC];
#pragma unroll
                for (int k = 0; k < HC / 8; ++k) tc::tmem_ld8(tD1 + lanes + c * QC + half * HC + 8 * k, x + 8 * k);
                tc::tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < HC / 8; ++k) tc::reg_fence8(x + 8 * k);
                if (row < ROWS) {
                    const float m = sBar[(row / 5) * BST + row % 5];
#pragma unroll
                    for (int k = 0; k < HC; ++k) dst[(half * HC + k) * ROWS + row] = x[k] + m;
                }
            }
        };
        readout(0, sUq);
        tc::fence_before_sync();
        __syncthreads();
        for (int c = 0; c < C::NCH; ++c) {
            // the next chunk's readout overlaps the previous chunk's G2
            if (c + 1 < C::NCH) readout(c + 1, sUq + ((c + 1) & 1) * QC * ROWS);
            if (c > 0) {   // the previous chunk's G2 has read A2
                ok &= tc::mbar_wait(&bars[1], ph2 & 1);
                ph2++;
            }
            // ---- one point of one element per thread: the contravariant flux
            // deviations, rounded to TF32, as A2 (row 5 e + v, K = a QC + point)
            {
                const int e = tid % E, qq = tid / E, q = c * QC + qq;
                float g[3][5];
                if (e < ne && q < NQ) {
                    const float* uq = sUq + (c & 1) * QC * ROWS + qq * ROWS + 5 * e;
                    float u[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) u[v] = uq[v];
                    float cof[9];
                    const long long eg = e0 + e;
                    if (eg < p.Kaff) {
#pragma unroll
                        for (int k = 0; k < 9; ++k) cof[k] = sG[e * GST + k];
                    } else {
                        const float* gc = p.geoC + (eg - p.Kaff) * CS;
#pragma unroll
                        for (int k = 0; k < 9; ++k) cof[k] = gc[k * NQ + q];
                    }
                    const float* b = sBar + e * BST;
                    const float ir = recip(u[0]);
                    const float vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
                    const float pr = (p.gamma - 1.f) * (u[4] - 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz));
                    const float dp = pr - b[8], H = u[4] + pr;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float c0 = cof[a], c1 = cof[3 + a], c2 = cof[6 + a];
                        const float Ua = c0 * vx + c1 * vy + c2 * vz, Ub = c0 * b[5] + c1 * b[6] + c2 * b[7];
                        g[a][0] = u[0] * Ua - b[0] * Ub;
                        g[a][1] = u[1] * Ua - b[1] * Ub + dp * c0;
                        g[a][2] = u[2] * Ua - b[2] * Ub + dp * c1;
                        g[a][3] = u[3] * Ua - b[3] * Ub + dp * c2;
                        g[a][4] = H * Ua - b[9] * Ub;
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int v = 0; v < 5; ++v) g[a][v] = 0.f;
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int v = 0; v < 5; ++v)
                        *reinterpret_cast<float*>(sm3 + C::O_A2 + il_offset(5 * e + v, a * QC + qq, C::LBO_A)) =
                            tc::to_tf32(g[a][v]);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {   // G2: this chunk's share of the volume term
                tc::fence_after_sync();
                const uint32_t b0 = aB2 + c * (C::KC / 4) * C::LBO_B2;
                for (int ks = 0; ks < C::KC / 8; ++ks)
                    tc::mma_tf32(tD2, tc::smem_desc(aA2 + ks * 2 * C::LBO_A, (uint32_t)C::LBO_A, 128u),
                                 tc::smem_desc(b0 + ks * 2 * C::LBO_B2, (uint32_t)C::LBO_B2, 128u), idesc2,
                                 (c > 0 || ks > 0) ? 1u : 0u);
                tc::mma_commit(&bars[1]);
            }
        }
        ok &= tc::mbar_wait(&bars[1], ph2 & 1);
        ph2++;
        tc::fence_after_sync();
        // ---- the volume term (deviation form) to sR [E][5][NP]
        if (quad < C::QU) {
            constexpr int NL = (NP + 7) / 8;
            for (int k = half; k < NL; k += 2) {
                float x[8];
                tc::tmem_ld8(tD2 + lanes + 8 * k, x);
                tc::tmem_ld_wait(x);
                if (row < ROWS) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (8 * k + i < NP) sR[row * NP + 8 * k + i] = x[i];
                }
            }
        }
        if (!ok) {
            atomicOr(p.err, 16);
            s_abort = 1;
        }
        // the second operand of the stage combination (U^n, or the
        // low-storage register) for this thread's outputs, loaded now so that
        // its latency overlaps the face terms
        constexpr int NIT = (E * 5 * NP + THREADS - 1) / THREADS;
        float aux[NIT];
        {
            const bool need = !p.rhs_only && p.a != 0.f;
#pragma unroll
            for (int k = 0; k < NIT; ++k) {
                const int i = tid + k * THREADS;
                const long long at = e0 * 5 * NP + i;
                aux[k] = (need && i < ne * 5 * NP) ? (p.dU ? p.dU[at] : p.Un[at]) : 0.f;
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // ---- face terms on the CUDA cores (the volume operands' storage is free)
        for (int i = tid; i < ne * 20 * NFPP; i += THREADS) {
            const int rw = i / NFPP, n = i - rw * NFPP;   // rw = (e * 4 + f) * 5 + v
            const int e = rw / 20, f = (rw / 5) & 3, v = rw % 5;
            sUf[i] = n < NFP ? sU[(e * 5 + v) * NPP + sFmask[f * NFP + n]] : 0.f;
        }
        if constexpr (NGP > NG) {
            constexpr int PG = NGP - NG;
            for (int i = tid; i < ne * 20 * PG; i += THREADS) {
                const int rw = i / PG;
                sFs[rw * NGP + NG + (i - rw * PG)] = 0.f;
            }
        }
        tc::cp_async_wait_all();   // the neighbours' face-node values (and the next tile's inputs)
        __syncthreads();
        face_points3<N, float, GST, BST>(p, e0, ne, tid, sI2, sW, sUf, sNb, sCode, sG, sBar, sFs);
        __syncthreads();
        lift3<N, float>(ne, sI2T, sFs, sCode, sUf);
        __syncthreads();
        combine3<N, float, 1>(ne, 0, sUf, sFpos, sR);
        __syncthreads();
        // L = M_k^-1 R and the stage combination
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int i = tid + k * THREADS;
            if (i >= ne * 5 * NP) break;
            const int e = i / (5 * NP), r = i - e * 5 * NP, v = r / NP, n = r - v * NP;
            const float* rr = sR + (e * 5 + v) * NP;
            const long long eg = e0 + e;
            float Lv = 0.f;
            if (eg < p.Kaff) {
#pragma unroll
                for (int j = 0; j < NP; ++j) Lv += sMiT[j * NP + n] * rr[j];
                Lv *= sG[e * GST + 9];
            } else {
                const float* mi = p.geoC + (eg - p.Kaff) * CS + 9 * NQ + 16 * NG;
#pragma unroll
                for (int j = 0; j < NP; ++j) Lv += mi[j * NP + n] * rr[j];
            }
            const long long at = e0 * 5 * NP + i;
            const float us = sU[(e * 5 + v) * NPP + n];
            float out;
            if (p.rhs_only) {
                out = Lv;
            } else if (p.dU) {
                const float d = p.a * aux[k] + p.dt * Lv;
                p.dU[at] = d;
                out = us + p.b * d;
            } else {
                out = p.a * aux[k] + p.b * (us + p.dt * Lv);
            }
            p.Uout[at] = out;
        }
    }
    // every copy and MMA of this CTA complete before it exits
    tc::cp_async_wait_all();
    __syncthreads();
    if (tid == 0) {
        tc::mma_commit(&bars[2]);
        if (!tc::mbar_wait(&bars[2], 0)) atomicOr(p.err, 16);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tmem, C::TMEM_COLS);
}

template <int N>
int prepare_tc_t() {
    static_assert(TC3<N>::TOTAL <= (int)SMEM3TC_MAX, "tensor-core tetrahedral tile exceeds shared memory");
    const cudaError_t e =
        cudaFuncSetAttribute(stage3_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC3<N>::TOTAL);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    return 0;
}

template <int N>
int launch_tc_t(const StageArgs3<float>& a, cudaStream_t st) {
    using C = TC3<N>;
    if (!a.err) return (int)cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int occ = std::max(1, resident_ctas((const void*)stage3_tc_kernel<N>, THREADS, C::TOTAL));
    const long long ntiles = (a.K + C::E - 1) / C::E;
    const int g = (int)std::min<long long>(ntiles, (long long)nsm * occ);
    if (g <= 0) return 0;
    StageArgs3<float> b = a;
    b.tile_e = C::E;
    stage3_tc_kernel<N><<<g, THREADS, C::TOTAL, st>>>(b);
    return (int)cudaGetLastError();
}

}  // namespace

bool supported_degree3_tc(int N) { return N == 2 || N == 3; }

int tile3_tc(int N) { return N == 2 ? TC3<2>::E : TC3<3>::E; }

int prepare_stage3_tc(int N) { return N == 2 ? prepare_tc_t<2>() : prepare_tc_t<3>(); }

int launch_stage3_tc(int N, const StageArgs3<float>& a, cudaStream_t st) {
    return N == 2 ? launch_tc_t<2>(a, st) : launch_tc_t<3>(a, st);
}

}  // namespace dgc

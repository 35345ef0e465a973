// Tensor-core gradient kernel of the artificial viscosity: q = sqrt(eps)
// grad U by the DG weak form with central fluxes (the BR1 q equation), for
// tiles of 32 affine elements, products on tcgen05 with FP32 accumulate:
//   G1: D1 = dU I_g^T (own traces), DQ = dU [Q_r; Q_s]^T with
//       Q_r = Mref^-1 D_r^T W I_cub (node to node);
//   GL: D_f = US (-Mref^-1 Lift_f)^T for the three faces f in one product
//       (the lift table split by face), US = sJ ((sqrt(eps) U)* - sqrt(eps)
//       Ubar) at the face points, and DL_m = sum_f n_m(f) D_f;
//   q_m = (1/J) (-sqrt(eps) (J r_m Q_r dU + J s_m Q_s dU) - DL_m).
// dU is the state minus its element mean; the mean drops out exactly
// because the discrete gradient of a constant vanishes.  Curved tiles run
// the CUDA-core body in a second launch.
#pragma once
#include <cstdio>
#include <cstdlib>
#include "tc_kernels.cuh"

namespace dgc {

template <int N>
struct TgSmem {
    using D = TcDims<N>;
    using L = TcLayout<N>;
    static constexpr int al(int x) { return (x + 127) / 128 * 128; }
    static constexpr int mx(int a, int b) { return a > b ? a : b; }
    static constexpr int sB1Q = 0;                                 // I_g rows
    static constexpr int sBQ = sB1Q + L::B1Q_BYTES;                // Q_r; Q_s rows
    static constexpr int sB2F = sBQ + L::BQ_BYTES;                 // -Mref^-1 Lift split by face
    static constexpr int sIGF = sB2F + L::B2F3_BYTES;
    static constexpr int A1_BYTES = 128 * D::NPK * 4;
    static constexpr int NBV_C = 5;                                // U+ (4) and sqrt(eps+)
    static constexpr int sA1 = al(sIGF + D::NF * D::NP * 4);       // G1 operand, then neighbour traces
    static constexpr int A1_REGION = al(mx(A1_BYTES, 32 * D::NF * NBV_C * 4));
    static constexpr int A2_BYTES = 128 * 32 * 4;
    static constexpr int sA2 = sA1 + A1_REGION;                    // face-term operand
    static constexpr int sTR = sA2 + A2_BYTES;                     // U tile, neighbour records, traces, face terms
    static constexpr int REC = 4 * D::NP + 4;                      // one element's U record and eps
    static constexpr int TR_BYTES = al(mx(mx(128 * D::NFS * 4, 32 * REC * 4), TileStage<N, false>::FLOATS * 4));
    static constexpr int NBB = TR_BYTES / (REC * 4);               // neighbour records per batch
    static constexpr int sIO = sTR + TR_BYTES;                     // q tile
    static constexpr int IO_REGION = al(32 * 8 * D::NP * 4);
    static constexpr int sMEAN = al(mx(sIO + IO_REGION, (int)Tile<N, float>::smem_grad()));  // curved tiles use all below
    static constexpr int sGEO = sMEAN + 128 * 4;
    static constexpr int sSE = sGEO + 32 * 16 * 4;
    static constexpr int sNB = sSE + 32 * 4;
    static constexpr int sBAR = sNB + 32 * 16;
    static constexpr int sTMEM = sBAR + 4 * 8;
    static constexpr int sLIST = sTMEM + 16;                       // out-of-tile faces: n, then (e,f)
    static constexpr int sFL = sLIST + 100 * 4;                    // faces owned by the tile: n, then (e,f)
    static constexpr int TOTAL = sFL + 100 * 4;
    static constexpr int TMEM_COLS = (D::NFP + 5 * D::N2) <= 128 ? 128 : 256;
    static_assert(TOTAL <= 232448, "gradient tile exceeds the shared-memory limit");
    static_assert(NBB >= 32 && (REC * 4) % 16 == 0, "bulk-copy staging layout");
    static_assert(Tile<N, float>::smem_grad() <= (size_t)sMEAN, "curved tile would clobber the tile state");
};

template <int N, int PREC>
__device__ __forceinline__ bool grad_tile_tc(const StageArgs<float>& p, float* q_out, long long e0, int ne,
                                             unsigned char* smem, uint32_t tmem, uint32_t& nwait, uint32_t& nld, int* err,
                                             bool rows_ready, int claim, int* next_tile, long long nCur,
                                             long long nAff) {
    using D = TcDims<N>;
    using S = TgSmem<N>;
    constexpr int NP = D::NP, NG = D::NG, NF = D::NF, NPK = D::NPK, NFP = D::NFP, N2 = D::N2, NFS = D::NFS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = (warp & 3) * 32 + lane;
    const int half = warp >> 2;
    const int e = row >> 2, v = row & 3;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t tD1 = tmem, tDQ = tmem + NFP, tDL = tDQ + 2 * N2;   // DL: 3 faces x N2

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::sBAR);
    float* sMean = reinterpret_cast<float*>(smem + S::sMEAN);
    float* sGeo = reinterpret_cast<float*>(smem + S::sGEO);
    float* sSe = reinterpret_cast<float*>(smem + S::sSE);
    int4* sNb = reinterpret_cast<int4*>(smem + S::sNB);
    float* sTr = reinterpret_cast<float*>(smem + S::sTR);
    const float* sIgF = reinterpret_cast<const float*>(smem + S::sIGF);
    unsigned char* A1 = smem + S::sA1;

    int* sList = reinterpret_cast<int*>(smem + S::sLIST);
    int* sFL = reinterpret_cast<int*>(smem + S::sFL);
    // the tile's U rows by a TMA bulk copy into the trace region
    using TS = TileStage<N, false>;
    if (tid == 32 && !rows_ready) issue_tile_rows<N, false, true>(p, e0, ne, sTr, &bars[1]);
    if (!tc::mbar_wait(&bars[1], nld & 1)) atomicOr(err, 8);
    ++nld;
    if (tid < 32)
        tile_info(threadIdx.x, e0, ne, true, sTr + TS::G, reinterpret_cast<const int4*>(sTr + TS::C), sTr + TS::E, sGeo, sNb, sSe,
                  sList, sFL);
    const bool live = e < ne;
    {   // both halves: the row's mean, then half h writes K values [h NPK/2, (h+1) NPK/2)
        float u[NP];
        float mean = 0.f;
        if (live) {
            const float* src = sTr + TS::U + row * NP;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                u[j] = src[j];
                mean += u[j];
            }
            mean *= (1.0f / NP);
        } else {
            mean = (v == 0) ? 1.f : (v == 3) ? 2.5f : 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j) u[j] = mean;
        }
        if (half == 0) sMean[row] = mean;
#pragma unroll
        for (int j0 = 0; j0 < NPK / 2; j0 += 8) {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {   // compile-time indices for either half
                constexpr int H = NPK / 2;
                const int jl = j0 + i, jh = H + j0 + i;
                const float lo = (jl < NP) ? u[jl < NP ? jl : 0] - mean : 0.f;
                const float hi = (jh < NP) ? u[jh < NP ? jh : 0] - mean : 0.f;
                x[i] = half ? hi : lo;
            }
            store8<PREC>(A1, row, half * (NPK / 2) + j0, NPK, x);
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
        issue_mma<PREC>(tD1, A1, smem + S::sB1Q, NFP, NPK, false);
        issue_mma<PREC>(tDQ, A1, smem + S::sBQ, 2 * N2, NPK, false);
        tc::mma_commit(&bars[0]);
    }
    // out-of-tile neighbours: their U records by 16-byte asynchronous copies
    // into the trace region, in batches of NBB faces (the first batch
    // overlaps G1), then the trace at the reversed point and sqrt(eps) into
    // the G1 operand region, one item per (face, variable, half of the face
    // points)
    float* sNbv = reinterpret_cast<float*>(smem + S::sA1);
    const int nlist = sList[0];
    auto issue_batch = [&](int b0) {
        constexpr int CH = NP + 1;   // 16-byte pieces of the U rows, then the eps word
        const int nc = min(S::NBB, nlist - b0) * CH;
        for (int c = tid; c < nc; c += blockDim.x) {
            const int i = c / CH, j = c - i * CH;
            const int entry = sList[1 + b0 + i];
            const int ee = entry / 3, f = entry - ee * 3;
            const int4 nbw = sNb[ee];
            const long long nb = (f == 0) ? nbw.x : (f == 1) ? nbw.y : nbw.z;
            if (j == NP)
                tc::cp_async4(sTr + i * S::REC + 4 * NP, p.eps + nb);
            else
                tc::cp_async16(sTr + i * S::REC + j * 4, p.Us + nb * 4 * NP + j * 4);
        }
    };
    if (nlist > 0) issue_batch(0);
    if (!tc::mbar_wait(&bars[0], nwait & 1)) atomicOr(err, 8);
    ++nwait;
    tc::fence_after_sync();
    {
        constexpr int GH = (NG + 1) / 2;
        for (int b0 = 0; b0 < nlist; b0 += S::NBB) {
            if (b0 > 0) {
                __syncthreads();   // the previous batch is consumed
                issue_batch(b0);
            }
            tc::cp_async_wait_all();
            __syncthreads();
            const int nitems = min(S::NBB, nlist - b0) * 8;
            for (int it = tid; it < nitems; it += blockDim.x) {
                const int fi = it >> 3, w = it & 3, hp = (it >> 2) & 1;
                const int entry = sList[1 + b0 + fi];
                const int ee = entry / 3, f = entry - ee * 3;
                const int4 nbw = sNb[ee];
                const int fn = code_face(nbw.w, f);
                const float* rec = sTr + fi * S::REC;
                // the neighbour's values at the nodes of its face fn
                constexpr int NE = TcDims<N>::NE;
                const int* fmask = reinterpret_cast<const int*>(sIgF + 3 * NG * NE) + fn * NE;
                float un[NE];
#pragma unroll
                for (int k = 0; k < NE; ++k) un[k] = rec[w * NP + fmask[k]];
                const float sen = sqrtf(rec[4 * NP]);
                const int g1 = hp ? NG : GH;
#pragma unroll 1
                for (int gg = hp * GH; gg < g1; ++gg) {
                    const float* eg = sIgF + (fn * NG + (NG - 1 - gg)) * NE;
                    float* dst = sNbv + (ee * NF + f * NG + gg) * S::NBV_C;
                    float a = 0.f;
#pragma unroll
                    for (int k = 0; k < NE; ++k) a += eg[k] * un[k];
                    dst[w] = a;
                    if (w == 0) dst[4] = sen;
                }
            }
        }
    }
    __syncthreads();   // the trace region is free again
    const float mean_v = sMean[row];
    if (half == 0) {
#pragma unroll
        for (int c0 = 0; c0 < NF; c0 += 8) {
            float x[8];
            tc::tmem_ld8(tD1 + lane_base + c0, x);
            tc::tmem_ld_wait(x);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (c0 + i < NF) sTr[row * NFS + c0 + i] = x[i] + mean_v;
        }
    }
    __syncthreads();

    // face points, once per point, in place: sJ ((sqrt(eps) U)* - sqrt(eps) Ubar)
    // for the 4 variables replaces the trace of each side; (sqrt(eps) U)* is
    // the central value, the same from both sides
    {
        const int nitems = sFL[0] * NG;
        for (int it = tid; it < nitems; it += blockDim.x) {
            const int entry = sFL[1 + it / NG], gg = it % NG;
            const int ee = entry / 3, f = entry - ee * 3, fg = f * NG + gg;
            const int4 nbw = sNb[ee];
            const int bc = code_bc(nbw.w, f);
            const int nb = (f == 0) ? nbw.x : (f == 1) ? nbw.y : nbw.z;
            const int fn = code_face(nbw.w, f), fgn = fn * NG + (NG - 1 - gg);
            const float* ge = sGeo + ee * 16;
            const float nx = ge[5 + 3 * f], ny = ge[6 + 3 * f], sJ = ge[7 + 3 * f];
            const float se = sSe[ee];
            const long long nbll = (long long)nb - e0;
            const bool in_tile = (bc == 0) && nbll >= 0 && nbll < ne;
            const int nbl = in_tile ? (int)nbll : 0;
            float Um[4], Up[4], sep;
#pragma unroll
            for (int w = 0; w < 4; ++w) Um[w] = sTr[(ee * 4 + w) * NFS + fg];
            if (bc != 0) {
                ghost_state(Um, bc, nx, ny, p.uinf, Up);
                sep = se;
            } else if (in_tile) {
#pragma unroll
                for (int w = 0; w < 4; ++w) Up[w] = sTr[(nbl * 4 + w) * NFS + fgn];
                sep = sSe[nbl];
            } else {
                const float* src = sNbv + (ee * NF + fg) * S::NBV_C;
#pragma unroll
                for (int w = 0; w < 4; ++w) Up[w] = src[w];
                sep = src[4];
            }
            float c[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                c[w] = 0.5f * (se * Um[w] + sep * Up[w]);
                sTr[(ee * 4 + w) * NFS + fg] = (c[w] - se * sMean[ee * 4 + w]) * sJ;
            }
            if (in_tile) {
                const float sJn = sGeo[nbl * 16 + 7 + 3 * fn];
#pragma unroll
                for (int w = 0; w < 4; ++w) sTr[(nbl * 4 + w) * NFS + fgn] = (c[w] - sep * sMean[nbl * 4 + w]) * sJn;
            }
        }
    }
    if (tid == THREADS - 1) *next_tile = claim;   // the claim made at the start of this tile
    __syncthreads();
    {   // the face terms of the row, 16 slots per half; the normals enter per
        // face in the epilogue (the lift table is split by face)
        unsigned char* dst = smem + S::sA2;
#pragma unroll
        for (int s0 = 0; s0 < 16; s0 += 8) {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = half * 16 + s0 + i;
                x[i] = (c < NF) ? sTr[row * NFS + c] : 0.f;
            }
            store8<PREC>(dst, row, half * 16 + s0, 32, x);
        }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        issue_mma<PREC>(tDL, smem + S::sA2, smem + S::sB2F, 3 * N2, 32, false);
        tc::mma_commit(&bars[0]);
    }
    // the next tile's rows into the (now free) trace region
    bool pre = false;
    {
        const long long tn = *next_tile;
        if (tn >= nCur && tn < nCur + nAff) {
            pre = true;
            if (tid == 32) {
                const long long en = (tn - nCur) * D::E;
                issue_tile_rows<N, false, true>(p, en, (int)min((long long)D::E, p.Kaff - en), sTr, &bars[1]);
            }
        }
    }
    if (!tc::mbar_wait(&bars[0], nwait & 1)) atomicOr(err, 16);
    ++nwait;
    tc::fence_after_sync();

    // epilogue: q_m for (element, variable) rows, then a coalesced store
    {
        float* sOut = reinterpret_cast<float*>(smem + S::sIO);   // [e][2][4][NP]
        const float* ge = sGeo + e * 16;
        const float jrx = ge[0], jry = ge[1], jsx = ge[2], jsy = ge[3], invJ = ge[4];
        const float nx0 = ge[5], ny0 = ge[6], nx1 = ge[8], ny1 = ge[9], nx2 = ge[11], ny2 = ge[12];
        const float se = sSe[e];
        constexpr int per_half = N2 / 2;
#pragma unroll
        for (int c0 = 0; c0 < per_half; c0 += 8) {
            const int i0 = half * per_half + c0;
            float qr[8], qs[8], d0[8], d1[8], d2[8];
            tc::tmem_ld8(tDQ + lane_base + i0, qr);
            tc::tmem_ld8(tDQ + N2 + lane_base + i0, qs);
            tc::tmem_ld8(tDL + lane_base + i0, d0);
            tc::tmem_ld8(tDL + N2 + lane_base + i0, d1);
            tc::tmem_ld_wait(qr, qs, d0, d1);
            tc::tmem_ld8(tDL + 2 * N2 + lane_base + i0, d2);
            tc::tmem_ld_wait(d2);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i0 + i < NP) {
                    const float lx = nx0 * d0[i] + nx1 * d1[i] + nx2 * d2[i];
                    const float ly = ny0 * d0[i] + ny1 * d1[i] + ny2 * d2[i];
                    sOut[(e * 8 + v) * NP + i0 + i] = invJ * (-se * (jrx * qr[i] + jsx * qs[i]) - lx);
                    sOut[(e * 8 + 4 + v) * NP + i0 + i] = invJ * (-se * (jry * qr[i] + jsy * qs[i]) - ly);
                }
        }
        tc::fence_before_sync();
        __syncthreads();
        const int n4 = ne * 2 * NP;   // float4 groups: ne * 8 * NP / 4
        float4* qo = reinterpret_cast<float4*>(q_out + e0 * 8 * NP);
        const float4* so = reinterpret_cast<const float4*>(sOut);
        for (int i = tid; i < n4; i += blockDim.x) qo[i] = so[i];
        __syncthreads();
    }
    return pre;
}

template <int N>
__device__ __forceinline__ void load_grad_operators(const unsigned char* ops_tc, unsigned char* smem) {
    using S = TgSmem<N>;
    using L = TcLayout<N>;
    constexpr int NF = TcDims<N>::NF, NP = TcDims<N>::NP;
    const int tid = threadIdx.x;
    const int4* src = reinterpret_cast<const int4*>(ops_tc);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = tid; i < L::B1Q_BYTES / 16; i += blockDim.x) dst[S::sB1Q / 16 + i] = src[L::B1Q / 16 + i];
    for (int i = tid; i < L::BQ_BYTES / 16; i += blockDim.x) dst[S::sBQ / 16 + i] = src[L::BQ / 16 + i];
    for (int i = tid; i < L::B2F3_BYTES / 16; i += blockDim.x) dst[S::sB2F / 16 + i] = src[L::B2F3 / 16 + i];
    const float* igs = reinterpret_cast<const float*>(ops_tc + L::IGF);
    float* igd = reinterpret_cast<float*>(smem + S::sIGF);
    for (int i = tid; i < NF * NP; i += blockDim.x) igd[i] = igs[i];
}

// Persistent grid claiming tiles from an atomic counter: curved tiles first
// (CUDA-core body), then affine tiles on the tensor cores.
template <int N, int PREC>
__global__ void __launch_bounds__(THREADS, 2) grad_kernel_tc(StageArgs<float> p, float* q_out,
                                                             const unsigned char* ops_tc, int* err, int* counter,
                                                             int* done) {
    extern __shared__ __align__(128) unsigned char smem_g[];
    using S = TgSmem<N>;
    constexpr int ET = TcDims<N>::E, EC = Tile<N, float>::E;
    const int tid = threadIdx.x;
    const long long nAff = (p.Kaff + ET - 1) / ET;
    const long long nCur = (p.K - p.Kaff + EC - 1) / EC;
    __shared__ int s_tile;
    __shared__ bool s_visc;
    // prologue (barriers, TMEM, operators) overlaps the previous kernel
    tc::pdl_trigger();
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_g + S::sBAR);
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) tc::mbar_init(&bars[b], 1);
        tc::mbar_fence_init();
    }
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem_g + S::sTMEM);
    if ((tid >> 5) == 0) tc::tmem_alloc(slot, S::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    uint32_t nwait = 0, nld = 0;
    bool ops_loaded = false, rows_ready = false;   // operators loaded with the first tile that needs them
    tc::pdl_wait();
    // no element anywhere with eps > 0 (the count comes with eps from the
    // kernel that wrote it; the stage kernel that follows resets it): q is
    // not needed at all
    if (p.visc != nullptr && *reinterpret_cast<volatile int*>(p.visc) == 0) {
        tc::fence_before_sync();
        __syncthreads();
        if ((tid >> 5) == 0) tc::tmem_free(tmem, S::TMEM_COLS);
        return;
    }
    if (tid == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    long long t = s_tile;
    while (t < nCur + nAff) {
        __syncthreads();   // every thread has read s_tile
        // claim the following tile now; the result is stored late in the tile
        const int claim = (tid == THREADS - 1) ? atomicAdd(counter, 1) : 0;
        if (t < nCur) {
            TileRange tr;
            tr.curved = true;
            tr.e0 = p.Kaff + t * EC;
            tr.ne = (int)min((long long)EC, p.K - tr.e0);
            grad_tile_call<N, float>(p, q_out, tr, smem_g);
            ops_loaded = false;
            rows_ready = false;
            if (tid == THREADS - 1) s_tile = claim;
            __syncthreads();
        } else {
            const long long e0 = (t - nCur) * ET;
            const int ne = (int)min((long long)ET, p.Kaff - e0);
            // q enters the stage only as sqrt(eps) q of its own element, so a
            // tile whose 32 elements all have eps = 0 needs none: its q is
            // neither computed nor written (the eps array is padded to whole
            // tiles with zeros)
            if (tid < 32) {
                const bool any = __any_sync(0xffffffffu, tid < ne && p.eps[e0 + tid] > 0.f);
                if (tid == 0) s_visc = any;
            }
            __syncthreads();
            if (!s_visc) {
                if (rows_ready) {   // this tile's rows were prefetched: complete that copy
                    if (!tc::mbar_wait(&bars[1], nld & 1)) atomicOr(err, 8);
                    ++nld;
                    rows_ready = false;
                }
                if (tid == THREADS - 1) s_tile = claim;
                __syncthreads();
            } else {
                if (!ops_loaded) {
                    load_grad_operators<N>(ops_tc, smem_g);
                    __syncthreads();
                    ops_loaded = true;
                }
                rows_ready = grad_tile_tc<N, PREC>(p, q_out, e0, ne, smem_g, tmem, nwait, nld, err, rows_ready, claim,
                                                   &s_tile, nCur, nAff);
            }
        }
        t = s_tile;
    }
    // the last CTA to leave resets the counters for the next launch
    __threadfence();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && atomicAdd(done, 1) == (int)gridDim.x - 1) {
        __threadfence();
        *counter = 0;
        *done = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_free(tmem, S::TMEM_COLS);
}

template <int N, int PREC>
struct TgGrid {
    static inline int ctas = 0;
};

template <int N, int PREC>
int prepare_grad_tc_t() {
    auto kern = grad_kernel_tc<N, PREC>;
    const int sm = TgSmem<N>::TOTAL;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return (int)e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
        return (int)e;
    int occ = resident_ctas((const void*)kern, THREADS, sm), dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
    const int by_tmem = 512 / TgSmem<N>::TMEM_COLS;
    occ = occ < by_tmem ? occ : by_tmem;
    if (occ < 1) return (int)cudaErrorInvalidConfiguration;
    if (getenv("DGC_VERBOSE")) fprintf(stderr, "dgcurved: %s N=%d: %d CTAs per SM\n", __func__, N, occ);
    TgGrid<N, PREC>::ctas = nsm * occ;
    return 0;
}

template <int N>
int prepare_grad_tc() {
    int e = prepare_grad_tc_t<N, PREC_TF32>();
    if (!e) e = prepare_grad_tc_t<N, PREC_BF16X3>();
    return e;
}

// err[2]: tile counter, err[4]: CTAs done (zero between launches: the last
// CTA resets them).
template <int N>
int launch_grad_tc(const StageArgs<float>& a, float* q_out, int prec, const unsigned char* ops_tc, int* err,
                   cudaStream_t st) {
    constexpr int ET = TcDims<N>::E, EC = Tile<N, float>::E;
    const long long tiles = (a.Kaff + ET - 1) / ET + (a.K - a.Kaff + EC - 1) / EC;
    if (tiles == 0) return 0;
    const int ctas = prec == PREC_TF32 ? TgGrid<N, PREC_TF32>::ctas : TgGrid<N, PREC_BF16X3>::ctas;
    if (ctas <= 0) return (int)cudaErrorNotReady;
    // the tile and neighbour records travel by TMA bulk copies: 16-byte aligned
    if (((uintptr_t)a.Us | (uintptr_t)q_out | (uintptr_t)ops_tc) & 15) return (int)cudaErrorMisalignedAddress;
    const unsigned grid = (unsigned)(tiles < ctas ? tiles : ctas);
    if (prec == PREC_TF32)
        return (int)launch_pdl(grad_kernel_tc<N, PREC_TF32>, grid, THREADS, TgSmem<N>::TOTAL, st, a, q_out, ops_tc,
                               err, err + 2, err + 4);
    return (int)launch_pdl(grad_kernel_tc<N, PREC_BF16X3>, grid, THREADS, TgSmem<N>::TOTAL, st, a, q_out, ops_tc, err,
                           err + 2, err + 4);
}

}  // namespace dgc

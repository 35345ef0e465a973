// Tensor-core (tcgen05) stage kernel: the right-hand side and SSP-RK stage
// of one tile of 32 affine elements, with the element-local operator
// products on the fifth-generation tensor cores (TF32, or BF16 split into a
// high and a low part with three products), FP32 accumulate in TMEM.
//
// Rows of both products are the 128 (element, variable) pairs of the tile:
//   G1: D1[(e,v), p] = sum_j dU[(e,v), j] B1[p, j]
//       B1 rows: I_cub (cubature points p < NQ), I_g (face points at FOFF+fg);
//       dU = U - mean_e(U): the element mean is added back exactly
//       (rows of I_cub and I_g sum to 1), so the low-precision products only
//       see the deviation.
//   G2: D2[(e,v), i] = sum_k A2[(e,v), k] B2[i, k], K in chunks of 32:
//       face chunks    A2 = (F*.n - F(Ubar).n) sJ          B2 = -Mref^-1 Lift
//       cubature chunks A2 = J(r_x dF + r_y dG), J(s_x dF + s_y dG), dF = F - F(Ubar)
//                                                         B2 = Mref^-1 D_r^T W, Mref^-1 D_s^T W
//       viscous chunks A2 = sqrt(eps) (J r_x q_x + J r_y q_y), ... at nodes
//                                                         B2 = -Mref^-1 D^T W I_cub
//   Subtracting the element-constant flux F(Ubar) changes nothing in exact
//   arithmetic (free-stream preservation: the volume and face terms of a
//   constant flux cancel on an affine element) and removes the cancellation
//   that would otherwise amplify the products' rounding.
//   L = D2 / J; U_out = a U^n + b (U_s + dt L).
// Each A2 chunk is written by the 256 threads from registers while the
// tensor core works on the previous chunk (two smem buffers, one mbarrier
// each).  Curved tiles run the CUDA-core tile body in the same launch.
#pragma once
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "refops.h"
#include "tc_ptx.cuh"

namespace dgc {

constexpr int PREC_TF32 = 1, PREC_BF16X3 = 2;

template <int N>
struct TcDims {
    static constexpr int NP = np_of(N), NQ = nq_of(N), NG = ng_of(N), NF = nf_of(N);
    static constexpr int NE = N + 1;                       // nodes on a face
    static_assert(3 * NG * NE + 3 * NE <= NF * NP, "the compact face tables fit the trace table's slot");
    static constexpr int NPK = (NP + 15) / 16 * 16;        // K of G1
    static constexpr int FOFF = (NQ + 15) / 16 * 16;       // first face column of D1
    static constexpr int N1 = (FOFF + NF + 15) / 16 * 16;  // columns of D1
    static constexpr int NFP = (NF + 15) / 16 * 16;        // columns of each q-trace block
    static constexpr int N2 = (NP + 15) / 16 * 16;         // columns of D2
    static constexpr int CF = (NF + 31) / 32;              // face chunks
    // the points of a partial last cubature chunk ride in the face chunk's
    // spare K slots when they fit (2 slots each: r and s parts; N = 4: the
    // 49th point), saving a chunk
    static constexpr int NQR = NQ % 16;
    static constexpr int NQF = (NQR != 0 && 2 * NQR <= 32 * CF - NF) ? NQR : 0;   // folded points
    static constexpr int CQ = NQF ? NQ / 16 : (NQ + 15) / 16;                     // cubature chunks
    static constexpr int CA = (NP + 15) / 16;              // viscous chunks
    static constexpr int NCH = CF + CQ + CA;               // chunks in the operator table
    static constexpr int E = 32;
    static constexpr int NFS = (NF + 2 * NQF) | 1;         // odd row stride of the trace exchange
    static constexpr int TMEM_COLS = (N1 + 2 * NFP + N2) <= 128 ? 128 : 256;
};

// Staging of one tile's inputs (float offsets): the U rows, the q rows
// (when Q), then x_r, x_s, y_r, y_s, the connectivity words and eps of the
// 32 elements.  Every piece starts on a 16-byte boundary.
template <int N, bool Q>
struct TileStage {
    static constexpr int NP = TcDims<N>::NP;
    static constexpr int U = 0;
    static constexpr int QR = 32 * 4 * NP;
    static constexpr int G = QR + (Q ? 32 * 8 * NP : 0);
    static constexpr int C = G + 32 * 4;
    static constexpr int E = C + 32 * 4;
    static constexpr int FLOATS = E + 32;
};

// Operator table of the tensor-core path (bytes; built by the host).
template <int N>
struct TcLayout {
    using D = TcDims<N>;
    static constexpr int B1 = 0;                                   // [N1 rows][NPK]
    static constexpr int B1_BYTES = D::N1 * D::NPK * 4;
    static constexpr int B1Q = B1 + B1_BYTES;                      // [NFP rows][NPK]  I_g
    static constexpr int B1Q_BYTES = D::NFP * D::NPK * 4;
    static constexpr int B2 = B1Q + B1Q_BYTES;                     // NCH x [N2 rows][32]
    static constexpr int B2_CHUNK = D::N2 * 32 * 4;
    // face traces from the face nodes, fp32 [3][NG][NE], then the face nodes int [3][NE]
    // (in a slot of NF x NP floats)
    static constexpr int IGF = B2 + D::NCH * B2_CHUNK;
    static constexpr int BQ = (IGF + D::NF * D::NP * 4 + 15) / 16 * 16;  // [2 N2 rows][NPK]: Q_r; Q_s
    static constexpr int BQ_BYTES = 2 * D::N2 * D::NPK * 4;
    static constexpr int VINV = BQ + BQ_BYTES;                      // V^-1 transposed, fp32 [NP][NP] (sensor)
    // gradient face terms: -Mref^-1 Lift split by face, [3 N2 rows][32]
    // (row f N2 + i keeps the columns of face f)
    static constexpr int B2F3 = (VINV + D::NP * D::NP * 4 + 15) / 16 * 16;
    static constexpr int B2F3_BYTES = 3 * B2_CHUNK;
    static constexpr int TOTAL = B2F3 + B2F3_BYTES;
};

// Shared-memory carve-up of the tensor-core kernel.  Regions whose
// lifetimes do not overlap share storage: the out-of-tile neighbour traces
// reuse the G1 operand region once G1 has completed; the trace region holds
// the own traces, then the face fluxes (in place), then the warp-private
// transposes of the cubature chunks, then the epilogue rows.  Two A2
// buffers, so that the tensor core works on one chunk while the next is
// written; the lean layout (inviscid only) has one, so that three tile
// pipelines fit an SM at the high degrees, and borrows the G1 operand
// region as the second: free from the face phase to the epilogue, when the
// chunks after the first (which uses the first buffer) are written.
template <int N, bool AV, bool SENSE = AV, bool LEAN = false>   // SENSE: the epilogue computes the next stage's eps
struct TcSmem {
    using D = TcDims<N>;
    using L = TcLayout<N>;
    static constexpr int NCHU = D::CF + D::CQ + (AV ? D::CA : 0);  // chunks used
    static constexpr int al(int x) { return (x + 127) / 128 * 128; }
    static constexpr int al1k(int x) { return (x + 1023) / 1024 * 1024; }
    static constexpr int mx(int a, int b) { return a > b ? a : b; }
    // constant region: operators, loaded once per CTA.  The viscous layout
    // extends the inviscid one with the sensor (SENSE) at its end: the
    // viscous chunks follow the face and cubature chunks, then I_g for q, so
    // a launch can load the common part before it knows which it is.
    static constexpr int sB1 = 0;
    static constexpr int sIGF = sB1 + L::B1_BYTES;
    static constexpr int sVI = sIGF + D::NF * D::NP * 4;                     // V^-1 transposed (the sensor)
    static constexpr int sB2 = al(sVI + (SENSE ? D::NP * D::NP * 4 : 0));
    static constexpr int sB1Q = sB2 + NCHU * L::B2_CHUNK;
    static constexpr int OPS_END = sB1Q + (AV ? L::B1Q_BYTES : 0);
    // per-tile region
    static constexpr int A1_BYTES = 128 * D::NPK * 4;
    static constexpr int NBV_C = AV ? 8 : 4;                                  // values per face point
    static constexpr int NBV_BYTES = 32 * D::NF * NBV_C * 4;
    // the A2 buffers (128-byte-swizzled operands) start on 1024-byte
    // boundaries: the per-tile region and the G1 operand region are
    // multiples of 1024 bytes
    static constexpr int sA1 = al1k(OPS_END);                                // G1 operands, then neighbour traces
    static constexpr int A1_REGION = al1k(mx(A1_BYTES * (AV ? 3 : 1), NBV_BYTES));
    static constexpr int A2_BYTES = 128 * 128;                               // 128 rows of 128 bytes
    static constexpr int NBUF = LEAN ? 1 : 2;
    static_assert(!(LEAN && AV), "the lean layout is inviscid");
    static constexpr int TR_FLOATS = 128 * D::NFS;
    static constexpr int REC = (AV ? 12 : 4) * D::NP + (AV ? 4 : 0);        // one element's U (and q, eps) record
    static constexpr int TR_REGION =
        al(mx(TR_FLOATS * 4 * (AV ? 2 : 1), mx(TileStage<N, AV>::FLOATS * 4, 32 * REC * 4)));
    static constexpr int NBB = TR_REGION / (REC * 4);                        // neighbour records per batch
    static constexpr int sA2 = sA1 + A1_REGION;
    static constexpr int sBUF1 = LEAN ? sA1 : sA2 + A2_BYTES;                // the second A2 buffer
    static constexpr bool LEAN_OK = A1_REGION >= A2_BYTES;                   // (the lean layout needs it)
    static constexpr int sTR = sA2 + NBUF * A2_BYTES;
    static constexpr int sMEAN = sTR + TR_REGION;                            // [128]
    static constexpr int sGEO = sMEAN + 128 * 4;                             // [32][16]
    static constexpr int sSE = sGEO + 32 * 16 * 4;                           // [32] sqrt(eps)
    static constexpr int sNB = sSE + 32 * 4;                                 // [32] int4
    static constexpr int sLIST = sNB + 32 * 16;                              // out-of-tile faces: n, then (e,f)
    static constexpr int sFL = sLIST + 100 * 4;                              // faces owned by the tile: n, then (e,f)
    static constexpr int sND = sFL + 100 * 4;                                // [32][2] sensor sums of the new state
    static constexpr int sFC = sND + 64 * 4;                                 // [32][8] contravariant mean flux
    static constexpr int sFBN = sFC + 32 * 8 * 4;                            // [32][3][4] (F(Ubar).n) sJ per face
    // [96] face records, 3 int4 each: in the last A2 buffer, free from the
    // previous tile's end to the face chunk unless viscous chunks occupy both
    // buffers at tile start (then a region of their own)
    static constexpr bool REC_OWN = AV && D::CA >= 2;
    static constexpr int REC_BYTES = 96 * 48;
    static constexpr int sREC = REC_OWN ? sFBN + 32 * 3 * 4 * 4 : sA2 + (NBUF - 1) * A2_BYTES;
    static constexpr int TOTAL = sFBN + 32 * 3 * 4 * 4 + (REC_OWN ? REC_BYTES : 0);
    static_assert(REC_BYTES <= A2_BYTES, "face records fit an A2 buffer");
    static_assert(TOTAL + 256 <= 232448, "tensor-core tile exceeds the shared-memory limit");
    static_assert(!AV || D::CA <= NBUF, "viscous chunks are written at tile start, one per A2 buffer");
    static_assert(NBB >= 32 && (REC * 4) % 16 == 0 && (32 * 4 * D::NP * 4) % 16 == 0, "bulk-copy staging layout");
    // epilogue rows: element e at floats [ES e, ES e + 4 NP); with rows on
    // 16-byte boundaries a padding of 4 floats per element spreads the
    // 16-byte stores of one quarter-warp over all banks
    static constexpr int ES = (D::NP % 4 == 0) ? 4 * D::NP + 4 : 4 * D::NP;
    static_assert(A1_REGION >= 32 * ES * 4, "epilogue rows live in the G1 operand region");
    // a curved tile (CUDA-core body, with viscosity in either kind of
    // launch) overwrites the dynamic region; the mbarriers and the TMEM slot
    // live in static shared memory and the operators are reloaded after it
    // (the lean layout: a curved tile of fewer elements, set by the launch)
    static_assert(LEAN || Tile<N, float>::smem_stage(AV) <= (size_t)TOTAL, "curved tile exceeds the tile's region");
};

template <int N, bool AV>
constexpr size_t tc_smem_bytes() {
    return TcSmem<N, AV>::TOTAL;
}

// The contravariant Euler flux of one point, less that of the element-mean
// state: with the element's metric g = (J r_x, J r_y, J s_x, J s_y),
//   Fr = g0 F + g1 G - fr,   Fs = g2 F + g3 G - fs,
// formed from the contravariant momenta m_r = g0 m_x + g1 m_y (and m_s):
//   g0 F + g1 G = (m_r, m_x u_r + g0 p, m_y u_r + g1 p, (E + p) u_r),
// u_r = m_r / rho; fr, fs are the same quantities of the mean state.
__device__ __forceinline__ void contra_flux_dev(const float U[4], float gamma, const float g[4], const float fr[4],
                                                const float fs[4], float Fr[4], float Fs[4]) {
    const float ir = recip(U[0]);
    const float mr = g[0] * U[1] + g[1] * U[2], ms = g[2] * U[1] + g[3] * U[2];
    const float ur = mr * ir, us = ms * ir;
    const float p = (gamma - 1.f) * (U[3] - 0.5f * (U[1] * U[1] + U[2] * U[2]) * ir);
    const float H = U[3] + p;
    Fr[0] = mr - fr[0];
    Fr[1] = fmaf(U[1], ur, fmaf(g[0], p, -fr[1]));
    Fr[2] = fmaf(U[2], ur, fmaf(g[1], p, -fr[2]));
    Fr[3] = fmaf(H, ur, -fr[3]);
    Fs[0] = ms - fs[0];
    Fs[1] = fmaf(U[1], us, fmaf(g[2], p, -fs[1]));
    Fs[2] = fmaf(U[2], us, fmaf(g[3], p, -fs[2]));
    Fs[3] = fmaf(H, us, -fs[3]);
}

// contra_flux_dev for two points at once on packed FP32 pairs (one FMA2,
// FADD2 or FMUL2 instruction for both points): U[w] holds variable w at the
// two points; g, nfr, nfs are the element's metric and the negated mean
// contravariant fluxes -fr, -fs, each value in both halves of its pair;
// gm1 = (gamma - 1) in both halves.  Each component is rounded as the
// scalar form's, up to the order of the two products in m_r and m_s.
__device__ __forceinline__ void contra_flux2_dev(const float2 U[4], float2 gm1, const float2 g[4],
                                                 const float2 nfr[4], const float2 nfs[4], float2 Fr[4],
                                                 float2 Fs[4]) {
    const float2 ir = make_float2(recip(U[0].x), recip(U[0].y));
    const float2 mr = __ffma2_rn(g[1], U[2], __fmul2_rn(g[0], U[1]));
    const float2 ms = __ffma2_rn(g[3], U[2], __fmul2_rn(g[2], U[1]));
    const float2 ur = __fmul2_rn(mr, ir), us = __fmul2_rn(ms, ir);
    // p = (gamma - 1) (E - |m|^2 / (2 rho))
    const float2 m2 = __ffma2_rn(U[2], U[2], __fmul2_rn(U[1], U[1]));
    const float2 p = __fmul2_rn(gm1, __ffma2_rn(__fmul2_rn(m2, ir), make_float2(-0.5f, -0.5f), U[3]));
    const float2 H = __fadd2_rn(U[3], p);
    Fr[0] = __fadd2_rn(mr, nfr[0]);
    Fr[1] = __ffma2_rn(U[1], ur, __ffma2_rn(g[0], p, nfr[1]));
    Fr[2] = __ffma2_rn(U[2], ur, __ffma2_rn(g[1], p, nfr[2]));
    Fr[3] = __ffma2_rn(H, ur, nfr[3]);
    Fs[0] = __fadd2_rn(ms, nfs[0]);
    Fs[1] = __ffma2_rn(U[1], us, __ffma2_rn(g[2], p, nfs[1]));
    Fs[2] = __ffma2_rn(U[2], us, __ffma2_rn(g[3], p, nfs[2]));
    Fs[3] = __ffma2_rn(H, us, nfs[3]);
}

// Writes 8 consecutive K values (k0 multiple of 8) of one row of an A
// operand with row_k K values.  TF32: rounded fp32; BF16X3: high part in the
// first half of the buffer, low part (x - high) in the second half.
template <int PREC>
__device__ __forceinline__ void store8(unsigned char* A, int row, int k0, int row_k, const float x[8]) {
    if constexpr (PREC == PREC_TF32) {
        const uint32_t rb = row_k * 4;
        float y[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            y[i] = x[i];
            y[i + 1] = x[i + 1];
            tc::to_tf32x2(y[i], y[i + 1]);
        }
        *reinterpret_cast<float4*>(A + tc::cm_offset(row, k0 * 4, rb)) = make_float4(y[0], y[1], y[2], y[3]);
        *reinterpret_cast<float4*>(A + tc::cm_offset(row, k0 * 4 + 16, rb)) = make_float4(y[4], y[5], y[6], y[7]);
    } else {
        const uint32_t rb = row_k * 2;
        const int half = 128 * row_k * 2;
        __align__(16) __nv_bfloat162 h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
            const float2 hf = __bfloat1622float2(h[i]);
            l[i] = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
        }
        *reinterpret_cast<uint4*>(A + tc::cm_offset(row, k0 * 2, rb)) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(A + half + tc::cm_offset(row, k0 * 2, rb)) = *reinterpret_cast<const uint4*>(l);
    }
}

// Writes 2 consecutive K values (k0 even) of one row of an A operand, as
// store8 does.
template <int PREC>
__device__ __forceinline__ void store2(unsigned char* A, int row, int k0, int row_k, float x0, float x1) {
    if constexpr (PREC == PREC_TF32) {
        tc::to_tf32x2(x0, x1);
        *reinterpret_cast<float2*>(A + tc::cm_offset(row, k0 * 4, row_k * 4)) = make_float2(x0, x1);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const uint32_t o = tc::cm_offset(row, k0 * 2, row_k * 2);
        *reinterpret_cast<__nv_bfloat162*>(A + o) = h;
        *reinterpret_cast<__nv_bfloat162*>(A + 128 * row_k * 2 + o) = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    }
}

// Writes 8 consecutive K values (k0 multiple of 8, k0 < 32) of one row of a
// G2 operand chunk (an A2 buffer): 128 rows of 128 bytes in the 128-byte
// swizzled layout.  TF32: the 32 values of a row, rounded; BF16X3: the high
// parts of the 32 values in bytes 0..63 and the low parts in bytes 64..127.
// Two 16-byte stores either way.
template <int PREC>
__device__ __forceinline__ void store8_a2(unsigned char* A, int row, int k0, const float x[8]) {
    if constexpr (PREC == PREC_TF32) {
        float y[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            y[i] = x[i];
            y[i + 1] = x[i + 1];
            tc::to_tf32x2(y[i], y[i + 1]);
        }
        *reinterpret_cast<float4*>(A + tc::sw128_offset(row, k0 * 4)) = make_float4(y[0], y[1], y[2], y[3]);
        *reinterpret_cast<float4*>(A + tc::sw128_offset(row, k0 * 4 + 16)) = make_float4(y[4], y[5], y[6], y[7]);
    } else {
        __align__(16) __nv_bfloat162 h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
            const float2 hf = __bfloat1622float2(h[i]);
            l[i] = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
        }
        *reinterpret_cast<uint4*>(A + tc::sw128_offset(row, k0 * 2)) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(A + tc::sw128_offset(row, 64 + k0 * 2)) = *reinterpret_cast<const uint4*>(l);
    }
}

// Writes 4 consecutive K values (k0 multiple of 4, k0 < 32) of one row of
// an A2 buffer, as store8_a2 does: one 16-byte store (TF32) or two 8-byte
// stores (BF16X3: high and low parts).
template <int PREC>
__device__ __forceinline__ void store4_a2(unsigned char* A, int row, int k0, const float x[4]) {
    if constexpr (PREC == PREC_TF32) {
        float y0 = x[0], y1 = x[1], y2 = x[2], y3 = x[3];
        tc::to_tf32x2(y0, y1);
        tc::to_tf32x2(y2, y3);
        *reinterpret_cast<float4*>(A + tc::sw128_offset(row, k0 * 4)) = make_float4(y0, y1, y2, y3);
    } else {
        __align__(8) __nv_bfloat162 h[2], l[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
            const float2 hf = __bfloat1622float2(h[i]);
            l[i] = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
        }
        *reinterpret_cast<uint2*>(A + tc::sw128_offset(row, k0 * 2)) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(A + tc::sw128_offset(row, 64 + k0 * 2)) = *reinterpret_cast<const uint2*>(l);
    }
}

// Issue the products D += A2 x B^T of one G2 chunk (K = 32): A2 an A2
// buffer (128-byte swizzled, see store8_a2), B n rows of 32 values in the
// core-matrix layout.
template <int PREC>
__device__ __forceinline__ void issue_mma_a2(uint32_t d_tmem, const unsigned char* A, const unsigned char* B, int n,
                                             bool accumulate) {
    const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
    if constexpr (PREC == PREC_TF32) {
        const uint32_t idesc = tc::instr_desc(2, 128, n);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
            tc::mma_tf32(d_tmem, tc::smem_desc_sw128(a0 + ks * 32), tc::smem_desc(b0 + ks * 256, 128u), idesc,
                         (accumulate || ks > 0) ? 1u : 0u);
    } else {
        const uint32_t idesc = tc::instr_desc(1, 128, n);
        const uint32_t bh = b0, bl = b0 + n * 64;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ah = tc::smem_desc_sw128(a0 + ks * 32), al = tc::smem_desc_sw128(a0 + 64 + ks * 32);
            tc::mma_bf16(d_tmem, ah, tc::smem_desc(bh + ks * 256, 64u), idesc, (accumulate || ks > 0) ? 1u : 0u);
            tc::mma_bf16(d_tmem, ah, tc::smem_desc(bl + ks * 256, 64u), idesc, 1u);
            tc::mma_bf16(d_tmem, al, tc::smem_desc(bh + ks * 256, 64u), idesc, 1u);
        }
    }
}

// Issue the products D += A x B^T over K = row_k values (A: 128 rows, B: n
// rows, both in the core-matrix layout with row_k values per row).
template <int PREC>
__device__ __forceinline__ void issue_mma(uint32_t d_tmem, const unsigned char* A, const unsigned char* B, int n,
                                          int row_k, bool accumulate) {
    if constexpr (PREC == PREC_TF32) {
        const uint32_t rb = row_k * 4;
        const uint32_t idesc = tc::instr_desc(2, 128, n);
        const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
        for (int ks = 0; ks < row_k / 8; ++ks)
            tc::mma_tf32(d_tmem, tc::smem_desc(a0 + ks * 256, rb), tc::smem_desc(b0 + ks * 256, rb), idesc,
                         (accumulate || ks > 0) ? 1u : 0u);
    } else {
        const uint32_t rb = row_k * 2;
        const uint32_t idesc = tc::instr_desc(1, 128, n);
        const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
        const uint32_t ah = a0, al = a0 + 128 * rb, bh = b0, bl = b0 + n * rb;
        for (int ks = 0; ks < row_k / 16; ++ks) {
            const uint32_t o = ks * 256;
            tc::mma_bf16(d_tmem, tc::smem_desc(ah + o, rb), tc::smem_desc(bh + o, rb), idesc,
                         (accumulate || ks > 0) ? 1u : 0u);
            tc::mma_bf16(d_tmem, tc::smem_desc(ah + o, rb), tc::smem_desc(bl + o, rb), idesc, 1u);
            tc::mma_bf16(d_tmem, tc::smem_desc(al + o, rb), tc::smem_desc(bh + o, rb), idesc, 1u);
        }
    }
}

// Per-element data of a tensor-core tile, by one warp (tid: its lane), from the staged copies
// of x_r, x_s, y_r, y_s, the connectivity words and eps: affine geometry,
// connectivity word, sqrt(eps) (when av), and two compact face lists (count
// first, then element * 3 + face): sList the faces whose neighbour lies
// outside the tile, sFL the faces whose flux the tile computes -- boundary
// and out-of-tile faces by the element itself, an in-tile pair by its
// lower-numbered element, so that each face point is computed once.
__device__ __forceinline__ void tile_info(int tid, long long e0, int ne, bool av, const float* stG, const int4* stC,
                                          const float* stE, float* sGeo, int4* sNb, float* sSe, int* sList,
                                          int* sFL) {
    int mout = 0, mown = 0;   // bit f: face f is out of tile / computed here
    if (tid < ne) {
        const int4 c = stC[tid];
        const float se = av ? sqrtf(stE[tid]) : 0.f;
        affine_geometry(stG + tid * 4, sGeo + tid * 16);
        sNb[tid] = c;
        sSe[tid] = se;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const long long nbl = (long long)((f == 0) ? c.x : (f == 1) ? c.y : c.z) - e0;
            const bool bnd = code_bc(c.w, f) != 0;
            const bool out = !bnd && (nbl < 0 || nbl >= ne);
            if (out) mout |= 1 << f;
            if (bnd || out || nbl > tid) mown |= 1 << f;
        }
    } else {  // padding element: unit geometry, farfield faces, never stored
#pragma unroll
        for (int i = 0; i < 16; ++i) sGeo[tid * 16 + i] = (i == 4 || i == 7 || i == 10 || i == 13) ? 1.f : 0.f;
        sNb[tid] = make_int4(0, 0, 0, 0x888);
        sSe[tid] = 0.f;
    }
    const int nout = __popc(mout), nown = __popc(mown);
    // both lists by one warp scan of the packed counts
    int incl = nout | (nown << 16);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
    }
    int po = (incl & 0xffff) - nout, pw = (incl >> 16) - nown;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        if (mout & (1 << f)) sList[1 + po++] = tid * 3 + f;
        if (mown & (1 << f)) sFL[1 + pw++] = tid * 3 + f;
    }
    if (tid == 31) {
        sList[0] = incl & 0xffff;
        sFL[0] = incl >> 16;
    }
}

// The 256 threads (8 warps) that work on one tile: a whole CTA, or one of
// the tile pipelines of a larger CTA that share its operator tables.  tid:
// index within the group; bar: the group's named barrier (0 in a CTA of 256
// threads); toff: byte offset of the group's per-tile shared-memory regions.
// hbar: the first of the two named barriers of the group's halves (threads
// 0..127 and 128..255), which work on alternate G2 chunks.
struct TcGroup {
    int tid;
    uint32_t bar;
    uint32_t toff;
    uint32_t hbar;
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, %1;" :: "r"(bar), "n"(THREADS) : "memory");
    }
    __device__ __forceinline__ void half_sync(int h) const {
        asm volatile("bar.sync %0, %1;" :: "r"(hbar + (uint32_t)h), "n"(THREADS / 2) : "memory");
    }
};

// Optional per-phase cycle counts of the tensor-core tile body (a build with
// DGC_PHASE_CLOCKS): thread 0 of each group adds the clock64 cycles of every
// phase of every tile to g_tc_phase_cycles (phase k ends at mark k: 0 tile
// inputs and G1 operand, 1 G1 and neighbour records, 2 neighbour traces, 3
// own traces, 4 face fluxes, 5 face chunk, 6 cubature chunks, 7 epilogue);
// slot 8 counts the tiles; the persistent kernel adds, per pipeline, the
// cycles of its curved tiles (9) and their count (10), of the prologue up to
// the first claim (11), of its lifetime (12) and the number of pipelines (13).
#ifdef DGC_PHASE_CLOCKS
static __device__ unsigned long long g_tc_phase_cycles[16];
template <int N>
int tc_phase_cycles(unsigned long long* out16, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out16, g_tc_phase_cycles, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess && reset) {
        const unsigned long long z[16] = {};
        e = cudaMemcpyToSymbol(g_tc_phase_cycles, z, sizeof(z));
    }
    return (int)e;
}
#define DGC_PHASE_BEGIN() long long dgc_t0 = clock64()
#define DGC_PHASE_MARK(k)                                                     \
    do {                                                                      \
        if (g.tid == 0) {                                                     \
            const long long dgc_t1 = clock64();                               \
            atomicAdd(&g_tc_phase_cycles[k], (unsigned long long)(dgc_t1 - dgc_t0)); \
            if ((k) == 7) atomicAdd(&g_tc_phase_cycles[8], 1ull);             \
            dgc_t0 = dgc_t1;                                                  \
        }                                                                     \
    } while (0)
#else
#define DGC_PHASE_BEGIN() \
    do {                  \
    } while (0)
#define DGC_PHASE_MARK(k) \
    do {                  \
    } while (0)
#endif

// Tile body: one tile of up to 32 affine elements.  The operator tables,
// mbarriers and TMEM are set up once per CTA by the persistent kernel;
// ph tracks the phases of the mbarriers across tiles.
struct TcPhase {
    uint32_t ld = 0;            // completions consumed on the bulk-copy barrier
    uint32_t g1 = 0;            // completions consumed on the G1 barrier
    uint32_t c0 = 0, c1 = 0;    // products committed on the A2 buffer barriers 0, 1
    uint32_t w0 = 0, w1 = 0;    // completions consumed on them
    // (scalars rather than arrays: a runtime index would put them in local memory)
    __device__ __forceinline__ void commit(int b) {
        if (b) ++c1; else ++c0;
    }
};

// Bulk copies of one tile's inputs into the staging region, signalled on bar
// (one thread).  eps is copied for all 32 slots of the tile: its device array
// is padded to a multiple of 32 elements.
template <int N, bool Q, bool EPS>
__device__ __forceinline__ void issue_tile_rows(const StageArgs<float>& p, long long e0, int ne, float* dst,
                                                uint64_t* bar) {
    using T = TileStage<N, Q>;
    constexpr int NP = TcDims<N>::NP;
    tc::fence_async_smem();
    const uint32_t bu = (uint32_t)ne * 4 * NP * 4, bq = Q ? (uint32_t)ne * 8 * NP * 4 : 0u, bg = (uint32_t)ne * 16;
    tc::mbar_expect_tx(bar, bu + bq + 2 * bg + (EPS ? 128u : 0u));
    tc::bulk_g2s(dst + T::U, p.Us + e0 * 4 * NP, bu, bar);
    if constexpr (Q) tc::bulk_g2s(dst + T::QR, p.q + e0 * 8 * NP, bq, bar);
    tc::bulk_g2s(dst + T::G, p.geoA + e0 * 4, bg, bar);
    tc::bulk_g2s(dst + T::C, p.conn + e0, bg, bar);
    if constexpr (EPS) tc::bulk_g2s(dst + T::E, p.eps + e0, 128u, bar);
}

// The 16 D1 columns of one cubature chunk from the 16-lane halves of a
// warp's 32 TMEM lanes (t: the warp's lane base and the chunk's first
// column): a, b the columns 2 (lane % 4) and + 1 of lanes 0..15 and 16..31,
// c, d the same 8 columns further.
__device__ __forceinline__ void tmem_ld_chunk(uint32_t t, float a[4], float b[4], float c[4], float d[4]) {
    tc::tmem_ld16x256(t, a);
    tc::tmem_ld16x256(t + (16u << 16), b);
    tc::tmem_ld16x256(t + 8, c);
    tc::tmem_ld16x256(t + (16u << 16) + 8, d);
    tc::tmem_ld_wait4(a, b);
    tc::tmem_ld_wait4(c, d);
}

// Tile body.  rows_ready: this tile's rows were requested by the previous
// tile.  claim: in the last thread, the index of this CTA's next tile from
// the atomic counter; it is stored to *next_tile once the face phase is
// done (its latency is long hidden by then) and read after the cubature
// chunks.  bars: the CTA's four mbarriers (A2 buffers 0 and 1, G1, bulk
// copies).  Returns true if the next tile's rows were requested here.
template <int N, bool AV, int PREC, bool SENSE = AV, bool LEAN = false>
__device__ __forceinline__ bool stage_tile_tc(const StageArgs<float>& p, long long e0, int ne, unsigned char* smem,
                                              uint32_t tmem, TcPhase& ph, int* err, bool rows_ready,
                                              int claim, int* next_tile, long long nCur, long long nAff,
                                              uint64_t* bars, const TcGroup& g) {
    using D = TcDims<N>;
    using S = TcSmem<N, AV, SENSE, LEAN>;
    constexpr int NP = D::NP, NQ = D::NQ, NG = D::NG, NF = D::NF, NPK = D::NPK, FOFF = D::FOFF;
    constexpr int N1 = D::N1, NFP = D::NFP, N2 = D::N2, NFS = D::NFS, CF = D::CF, CQ = D::CQ, CA = D::CA;
    constexpr int B2C = TcLayout<N>::B2_CHUNK;
    const int tid = g.tid, warp = tid >> 5, lane = tid & 31;
    // TMEM lane / operand row: within each warp's 32 lanes, variable-major
    // (row = 32 q + 8 v + element % 8 for the element 8 q + element % 8);
    // shared-memory arrays keep the element-major order lrow = 4 e + v
    const int row = (warp & 3) * 32 + lane;
    const int half = warp >> 2;                 // which half of the columns this thread loads
    const int e = (warp & 3) * 8 + (lane & 7), v = lane >> 3, lrow = e * 4 + v;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    // lean layout: D2 over D1's face columns, which are read before the
    // first G2 product (the cubature columns lie below FOFF)
    static_assert(!LEAN || FOFF + N2 <= N1, "D2 fits over D1's face columns");
    static_assert(!LEAN || S::LEAN_OK, "the G1 operand region holds an A2 buffer");
    const uint32_t tD1 = tmem, tD1q = tmem + N1, tD2 = LEAN ? tmem + FOFF : tmem + N1 + (AV ? 2 * NFP : 0);
    // the cubature chunks of the second half accumulate into D2b over D1's
    // first N2 columns (those of cubature chunks 0 and 1), once both halves
    // have read their first chunk
    static_assert(N2 <= 32 && (CQ < 2 || N2 <= 32), "D2b lies over the columns of cubature chunks 0 and 1");
    // with an odd number of cubature chunks the last one is shared by the
    // halves (each thread 2 of its points) so that both halves finish together
    constexpr bool JOINT = CQ % 2 == 1;
    constexpr int CP = JOINT ? CQ - 1 : CQ;   // the chunks the halves take in turn
    constexpr bool D2B = CP >= 2;
    const uint32_t tD2b = tmem;

    float* sMean = reinterpret_cast<float*>(smem + g.toff + S::sMEAN);
    float* sGeo = reinterpret_cast<float*>(smem + g.toff + S::sGEO);
    float* sSe = reinterpret_cast<float*>(smem + g.toff + S::sSE);
    int4* sNb = reinterpret_cast<int4*>(smem + g.toff + S::sNB);
    float* sTr = reinterpret_cast<float*>(smem + g.toff + S::sTR);
    float* sQn = sTr + S::TR_FLOATS;            // AV: sqrt(eps) q.n at own face points
    const float* sIgF = reinterpret_cast<const float*>(smem + S::sIGF);
    unsigned char* A1 = smem + g.toff + S::sA1;
    int* sList = reinterpret_cast<int*>(smem + g.toff + S::sLIST);
    int* sFL = reinterpret_cast<int*>(smem + g.toff + S::sFL);
    float* sND = reinterpret_cast<float*>(smem + g.toff + S::sND);
    float* sFC = reinterpret_cast<float*>(smem + g.toff + S::sFC);
    float* sFbnJ = reinterpret_cast<float*>(smem + g.toff + S::sFBN);
    int4* sRec = reinterpret_cast<int4*>(smem + g.toff + S::sREC);

    // G2 runs as a sequence of K chunks; chunk number s uses A2 buffer s % 2.
    auto buf_of = [](int s) { return s & 1; };
    auto a2_buf = [&](int s) { return smem + g.toff + ((s & 1) ? S::sBUF1 : S::sA2); };
    auto wait_buf = [&](int b) {   // every product issued from buffer b has completed
        uint32_t& w = b ? ph.w1 : ph.w0;
        const uint32_t c = b ? ph.c1 : ph.c0;
        while (w < c) {
            if (!tc::mbar_wait(&bars[b], w & 1)) atomicOr(err, 2);
            ++w;
        }
    };
    auto issue_chunk = [&](int s, int op_chunk) {   // thread 0, after the operand is visible
        issue_mma_a2<PREC>(tD2, a2_buf(s), smem + S::sB2 + op_chunk * B2C, N2, s > 0);
        tc::mma_commit(&bars[buf_of(s)]);
    };
    int seq = 0;
    DGC_PHASE_BEGIN();

    // ---------------- tile inputs: the U (and q) rows of the tile by TMA bulk
    // copies into the trace region; per-element data and face lists by warp 4
    if (tid == 32 && !rows_ready) issue_tile_rows<N, AV, AV>(p, e0, ne, sTr, &bars[3]);
    const long long k = e0 + e;
    const bool live = e < ne;
    using TS = TileStage<N, AV>;
    if (!tc::mbar_wait(&bars[3], ph.ld & 1)) atomicOr(err, 8);
    ph.ld++;
    if (warp == 4)   // per-element data by a warp of the half that does not build the G1 operand
        tile_info(tid - 128, e0, ne, AV, sTr + TS::G, reinterpret_cast<const int4*>(sTr + TS::C), sTr + TS::E, sGeo,
                  sNb, sSe, sList, sFL);
    // out-of-tile neighbours: their U (and q) records by 16-byte asynchronous
    // copies into the trace region, in batches of NBB faces (the first batch
    // overlaps G1), then their traces at the reversed face points into the G1
    // operand region, one item per (face, variable, half of the face points)
    float* sRecs = sTr;
    constexpr int NBB = S::NBB;
    auto issue_batch = [&](int b0, int t0, int nt) {
        // 16-byte pieces: U rows, then q rows; with AV one more item per face
        // copies its eps (4 bytes) to the last word of the record
        constexpr int CU = NP, CH = (AV ? 12 : 4) * NP / 4 + (AV ? 1 : 0);
        const int nc = min(NBB, sList[0] - b0) * CH;
        for (int c = t0; c < nc; c += nt) {
            const int i = c / CH, j = c - i * CH;
            const int entry = sList[1 + b0 + i];
            const int ee = entry / 3, f = entry - ee * 3;
            const int4 nbw = sNb[ee];
            const long long nb = (f == 0) ? nbw.x : (f == 1) ? nbw.y : nbw.z;
            if (AV && j == CH - 1) {
                tc::cp_async4(sRecs + i * S::REC + 12 * NP, p.eps + nb);
                continue;
            }
            const float* src = (j < CU) ? p.Us + nb * 4 * NP + j * 4 : p.q + nb * 8 * NP + (j - CU) * 4;
            tc::cp_async16(sRecs + i * S::REC + j * 4, src);
        }
    };

    if (half == 0) {   // the G1 operand
        float u[NP];
        float mean = 0.f;
        if (live) {
            const float* src = sTr + TS::U + lrow * NP;
            if constexpr (NP % 4 == 0) {   // rows on 16-byte boundaries
#pragma unroll
                for (int j = 0; j < NP; j += 4) {
                    const float4 q4 = *reinterpret_cast<const float4*>(src + j);
                    u[j] = q4.x;
                    u[j + 1] = q4.y;
                    u[j + 2] = q4.z;
                    u[j + 3] = q4.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < NP; ++j) u[j] = src[j];
            }
#pragma unroll
            for (int j = 0; j < NP; ++j) mean += u[j];
            mean *= (1.0f / NP);
        } else {
            mean = (v == 0) ? 1.f : (v == 3) ? 2.5f : 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j) u[j] = mean;
        }
        sMean[lrow] = mean;
#pragma unroll
        for (int j0 = 0; j0 < NPK; j0 += 8) {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = (j0 + i < NP) ? u[j0 + i] - mean : 0.f;
            store8<PREC>(A1, row, j0, NPK, x);
        }
    } else if constexpr (AV) {
        // q rows: the G1 operands for the q traces, and the viscous chunks
        // sqrt(eps) (J r_x q_x + J r_y q_y), sqrt(eps) (J s_x q_x + J s_y q_y)
        // at the nodes, written straight into the first A2 buffers
        float qx[NP], qy[NP];
        const float* src = sTr + TS::QR + (e * 8 + v) * NP;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            qx[j] = live ? src[j] : 0.f;
            qy[j] = live ? src[4 * NP + j] : 0.f;
        }
        // J r_x = y_s, J r_y = -x_s, J s_x = -y_r, J s_y = x_r (zero for padding rows)
        const float4 gk = live ? *reinterpret_cast<const float4*>(sTr + TS::G + e * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float g[4] = {gk.w, -gk.y, -gk.z, gk.x};
        const float se = live ? sqrtf(sTr[TS::E + e]) : 0.f;
#pragma unroll
        for (int j0 = 0; j0 < NPK; j0 += 8) {
            float x[8], y[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                x[i] = (j0 + i < NP) ? qx[j0 + i] : 0.f;
                y[i] = (j0 + i < NP) ? qy[j0 + i] : 0.f;
            }
            store8<PREC>(A1 + S::A1_BYTES, row, j0, NPK, x);
            store8<PREC>(A1 + 2 * S::A1_BYTES, row, j0, NPK, y);
        }
#pragma unroll
        for (int ca = 0; ca < CA; ++ca) {
#pragma unroll
            for (int k0 = 0; k0 < 16; k0 += 8) {
                float ar[8], as[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int j = ca * 16 + k0 + i;
                    const float a = (j < NP) ? qx[j] : 0.f, b = (j < NP) ? qy[j] : 0.f;
                    ar[i] = se * (g[0] * a + g[1] * b);
                    as[i] = se * (g[2] * a + g[3] * b);
                }
                store8_a2<PREC>(a2_buf(ca), row, k0, ar);
                store8_a2<PREC>(a2_buf(ca), row, 16 + k0, as);
            }
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    if constexpr (!AV) {
        // G1 as soon as half 0 has written its operand, while warp 4 may
        // still be forming the per-element data
        if (half == 0) {
            g.half_sync(0);
            if (tid == 0) {
                tc::fence_after_sync();
                issue_mma<PREC>(tD1, A1, smem + S::sB1, N1, NPK, false);
                tc::mma_commit(&bars[2]);
            }
        }
    }
    g.sync();
    DGC_PHASE_MARK(0);
    tc::fence_after_sync();

    // ---------------- G1: state deviations to cubature and face points (AV:
    // here, after the q operands; the viscous chunks of G2 start at once)
    if (AV && tid == 0) {
        issue_mma<PREC>(tD1, A1, smem + S::sB1, N1, NPK, false);
        if constexpr (AV) {
            issue_mma<PREC>(tD1q, A1 + S::A1_BYTES, smem + S::sB1Q, NFP, NPK, false);
            issue_mma<PREC>(tD1q + NFP, A1 + 2 * S::A1_BYTES, smem + S::sB1Q, NFP, NPK, false);
        }
        tc::mma_commit(&bars[2]);
        if constexpr (AV)
            for (int ca = 0; ca < CA; ++ca) issue_chunk(ca, CF + CQ + ca);
    }
    if constexpr (AV) {
        for (int ca = 0; ca < CA; ++ca) ph.commit(buf_of(ca));
        seq = CA;
    }

    float* sNbv = reinterpret_cast<float*>(smem + g.toff + S::sA1);
    const int nlist = sList[0];
    if (nlist > 0) issue_batch(0, tid, THREADS);
    if (tid < 128) {   // flux of the element-mean state, one (element, variable) per thread
        float Ub[4], Fb[4], Gb[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) Ub[w] = sMean[e * 4 + w];
        euler_flux(Ub, p.gamma, Fb, Gb);
        // and its contravariant forms with the element's metric, and its
        // normal flux times sJ on each face
        const float* ge = sGeo + e * 16;
        sFC[e * 8 + v] = ge[0] * Fb[v] + ge[1] * Gb[v];
        sFC[e * 8 + 4 + v] = ge[2] * Fb[v] + ge[3] * Gb[v];
#pragma unroll
        for (int f = 0; f < 3; ++f)
            sFbnJ[(e * 3 + f) * 4 + v] = (Fb[v] * ge[5 + 3 * f] + Gb[v] * ge[6 + 3 * f]) * ge[7 + 3 * f];
    }
    if (!tc::mbar_wait(&bars[2], ph.g1 & 1)) atomicOr(err, 1);
    ph.g1++;
    tc::fence_after_sync();
    DGC_PHASE_MARK(1);
    {
        constexpr int GH = (NG + 1) / 2;
        for (int b0 = 0; b0 < nlist; b0 += NBB) {
            if (b0 > 0) {
                g.sync();   // the previous batch is consumed
                issue_batch(b0, tid, THREADS);
            }
            tc::cp_async_wait_all();
            g.sync();
            const int nitems = min(NBB, nlist - b0) * 8;
            for (int it = tid; it < nitems; it += THREADS) {
                const int fi = it >> 3, w = it & 3, hp = (it >> 2) & 1;
                const int entry = sList[1 + b0 + fi];
                const int ee = entry / 3, f = entry - ee * 3;
                const int4 nbw = sNb[ee];
                const int fn = code_face(nbw.w, f);
                const float* rec = sRecs + fi * S::REC;
                // the neighbour's values at the nodes of its face fn
                constexpr int NE = D::NE;
                const int* fmask = reinterpret_cast<const int*>(sIgF + 3 * NG * NE) + fn * NE;
                float un[NE], qx[AV ? NE : 1], qy[AV ? NE : 1];
#pragma unroll
                for (int k = 0; k < NE; ++k) un[k] = rec[w * NP + fmask[k]];
                float sen = 0.f, nx = 0.f, ny = 0.f;
                if constexpr (AV) {
#pragma unroll
                    for (int k = 0; k < NE; ++k) {
                        qx[k] = rec[(4 + w) * NP + fmask[k]];
                        qy[k] = rec[(8 + w) * NP + fmask[k]];
                    }
                    sen = sqrtf(rec[12 * NP]);
                    nx = sGeo[ee * 16 + 5 + 3 * f];
                    ny = sGeo[ee * 16 + 6 + 3 * f];
                }
                const int g1 = hp ? NG : GH;
#pragma unroll 1
                for (int gg = hp * GH; gg < g1; ++gg) {
                    const int fg = f * NG + gg;
                    const float* eg = sIgF + (fn * NG + (NG - 1 - gg)) * NE;
                    float* dst = sNbv + (ee * NF + fg) * S::NBV_C;
                    float a = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
                    for (int k = 0; k < NE; ++k) {
                        const float g = eg[k];
                        a += g * un[k];
                        if constexpr (AV) {
                            ax += g * qx[k];
                            ay += g * qy[k];
                        }
                    }
                    dst[w] = a;
                    if constexpr (AV) dst[4 + w] = sen * (ax * nx + ay * ny);
                }
            }
        }
    }
    g.sync();   // the trace region is free again
    DGC_PHASE_MARK(2);

    // ---------------- own traces (and sqrt(eps) q.n) to shared memory
    const float mean_v = sMean[lrow];
    if (half == 0) {
#pragma unroll
        for (int c0 = 0; c0 < NF; c0 += 8) {
            float x[8];
            tc::tmem_ld8(tD1 + lane_base + FOFF + c0, x);
            tc::tmem_ld_wait(x);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (c0 + i < NF) sTr[lrow * NFS + c0 + i] = x[i] + mean_v;
        }
        if constexpr (D::NQF > 0) {   // the folded cubature points' values
            float x[8];
            tc::tmem_ld8(tD1 + lane_base + CQ * 16, x);
            tc::tmem_ld_wait(x);
#pragma unroll
            for (int m = 0; m < D::NQF; ++m) sTr[lrow * NFS + NF + 2 * m] = x[m] + mean_v;
        }
    } else if constexpr (AV) {
        const float se = sSe[e];
#pragma unroll
        for (int c0 = 0; c0 < NF; c0 += 8) {
            float qx[8], qy[8];
            tc::tmem_ld8(tD1q + lane_base + c0, qx);
            tc::tmem_ld8(tD1q + NFP + lane_base + c0, qy);
            tc::tmem_ld_wait(qx, qy);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int fg = c0 + i;
                if (fg < NF) {
                    const int f = fg / NG;
                    sQn[lrow * NFS + fg] = se * (qx[i] * sGeo[e * 16 + 5 + 3 * f] + qy[i] * sGeo[e * 16 + 6 + 3 * f]);
                }
            }
        }
    }
    // face records, one thread per face the tile computes: where each side's
    // values are, the normal, sJ of both sides and their mean-flux indices
    {
        const int rt = AV ? tid : tid - 128;
        if (rt >= 0 && rt < sFL[0]) {
            const int entry = sFL[1 + rt];
            const int ee = entry / 3, f = entry - ee * 3;
            const int4 nbw = sNb[ee];
            const int bc = code_bc(nbw.w, f);
            const int nb = (f == 0) ? nbw.x : (f == 1) ? nbw.y : nbw.z;
            const int fn = code_face(nbw.w, f);
            const long long nbll = (long long)nb - e0;
            const bool in_tile = (bc == 0) && nbll >= 0 && nbll < ne;
            const int nbl = in_tile ? (int)nbll : 0;
            const int own = ee * 4 * NFS + f * NG;
            int up = own, step = 0, vstr = NFS;
            if (in_tile) {
                up = nbl * 4 * NFS + fn * NG + (NG - 1);
                step = -1;
            } else if (bc == 0) {
                up = (ee * NF + f * NG) * S::NBV_C;
                step = S::NBV_C;
                vstr = 1;
            }
            const float* ge = sGeo + ee * 16;
            const float sJn = in_tile ? sGeo[nbl * 16 + 7 + 3 * fn] : 0.f;
            sRec[3 * rt] = make_int4(own, up, (bc | (in_tile ? 4 : 0)) | ((step + 128) << 8) | (vstr << 16),
                                     (ee * 3 + f) | ((in_tile ? nbl * 3 + fn : 0) << 16));
            sRec[3 * rt + 1] = make_int4(__float_as_int(ge[5 + 3 * f]), __float_as_int(ge[6 + 3 * f]),
                                         __float_as_int(ge[7 + 3 * f]), __float_as_int(sJn));
        }
    }
    if constexpr (LEAN) tc::fence_before_sync();   // D1's face columns are read: D2 may overwrite them
    g.sync();
    DGC_PHASE_MARK(3);

    // ---------------- face fluxes, once per face point, in place:
    // (F*.n - (sqrt(eps) q)*.n - F(Ubar).n) sJ replaces the trace of each
    // side.  F* from the other side of an in-tile face is -F*.
    // (one loop per numerical flux, so that each carries only its own code)
    auto face_phase = [&](auto flux_tag) {
        constexpr int FLUX = decltype(flux_tag)::value;
        const int nface = sFL[0] * NG;
        const int nitems = nface + 32 * D::NQF;
        for (int it = tid; it < nitems; it += THREADS) {
            if (D::NQF > 0 && it >= nface) {
                // a folded cubature point of one element: its contravariant
                // flux deviations into the two slots after the face points
                const int ee = (it - nface) & 31, m = (it - nface) >> 5;
                float* tr = sTr + ee * 4 * NFS + NF + 2 * m;
                const float Uc[4] = {tr[0], tr[NFS], tr[2 * NFS], tr[3 * NFS]};
                float Fr[4], Fs[4];
                contra_flux_dev(Uc, p.gamma, sGeo + ee * 16, sFC + ee * 8, sFC + ee * 8 + 4, Fr, Fs);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    tr[w * NFS] = Fr[w];
                    tr[w * NFS + 1] = Fs[w];
                }
                continue;
            }
            const int fi = it / NG, gg = it - fi * NG;
            const int4 r0 = sRec[3 * fi], r1 = sRec[3 * fi + 1];
            const int bc = r0.z & 3;
            const bool in_tile = (r0.z & 4) != 0;
            const int step = ((r0.z >> 8) & 255) - 128, vstr = r0.z >> 16;
            const float nx = __int_as_float(r1.x), ny = __int_as_float(r1.y), sJ = __int_as_float(r1.z);
            const int om = r0.x + gg, op = r0.y + step * gg;
            float Um[4], Up[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) Um[w] = sTr[om + w * NFS];
            if (bc != 0) {
                ghost_state(Um, bc, nx, ny, p.uinf, Up);
            } else {
                // the neighbour's trace: in the tile's own rows (reversed
                // along the face) or among the out-of-tile neighbour traces
                const float* src = in_tile ? sTr : sNbv;
#pragma unroll
                for (int w = 0; w < 4; ++w) Up[w] = src[op + w * vstr];
            }
            float Fn[4];
            if constexpr (FLUX == 1)
                hllc_flux(Um, Up, nx, ny, p.gamma, Fn);
            else
                llf_flux(Um, Up, nx, ny, p.gamma, Fn);
            if constexpr (AV) {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const float own = sQn[om + w * NFS];
                    float other;   // the neighbour's sqrt(eps) q.n' with n' = -n, negated
                    if (bc != 0) {
                        other = own;
                    } else if (in_tile) {
                        other = -sQn[op + w * NFS];
                    } else {
                        other = sNbv[op + 4 + w];
                    }
                    Fn[w] -= 0.5f * (own + other);
                }
            }
            const float4 fo = *reinterpret_cast<const float4*>(sFbnJ + 4 * (r0.w & 0xffff));
            sTr[om] = fmaf(Fn[0], sJ, -fo.x);
            sTr[om + NFS] = fmaf(Fn[1], sJ, -fo.y);
            sTr[om + 2 * NFS] = fmaf(Fn[2], sJ, -fo.z);
            sTr[om + 3 * NFS] = fmaf(Fn[3], sJ, -fo.w);
            if (in_tile) {
                const float sJn = __int_as_float(r1.w);
                const float4 fm = *reinterpret_cast<const float4*>(sFbnJ + 4 * (r0.w >> 16));
                sTr[op] = fmaf(-Fn[0], sJn, -fm.x);
                sTr[op + NFS] = fmaf(-Fn[1], sJn, -fm.y);
                sTr[op + 2 * NFS] = fmaf(-Fn[2], sJn, -fm.z);
                sTr[op + 3 * NFS] = fmaf(-Fn[3], sJn, -fm.w);
            }
        }
    };
    if (p.flux == 1)
        face_phase(std::integral_constant<int, 1>{});
    else
        face_phase(std::integral_constant<int, 0>{});
    if (tid == THREADS - 1) *next_tile = claim;
    g.sync();
    DGC_PHASE_MARK(4);

    // ---------------- face chunk: the rows of the flux region, 16 slots per half
    static_assert(CF == 1, "one face chunk");
    {
        wait_buf(buf_of(seq));
        unsigned char* A2 = a2_buf(seq);
#pragma unroll
        for (int s0 = 0; s0 < 16; s0 += 8) {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = half * 16 + s0 + i;
                x[i] = (c < NF + 2 * D::NQF) ? sTr[lrow * NFS + c] : 0.f;
            }
            store8_a2<PREC>(A2, row, half * 16 + s0, x);
        }
        tc::fence_async_smem();
        g.sync();
    DGC_PHASE_MARK(5);
        if (tid == 0) {
            tc::fence_after_sync();
            issue_chunk(seq, 0);
        }
        ph.commit(buf_of(seq));
        ++seq;
    }

    // the epilogue's inputs from global memory (U_s, and U^n or the
    // low-storage register) into L2 while the cubature chunks run
    if (tid == 64 && !p.rhs_only) {
        const uint32_t nb = (uint32_t)ne * 4 * NP * 4;
        tc::prefetch_l2(p.Us + e0 * 4 * NP, nb);
        if (p.a != 0.f) tc::prefetch_l2((p.dU ? p.dU : p.Un) + e0 * 4 * NP, nb);
    }

    // ---------------- the next tile's rows into the trace region, free now
    // that the face chunk's operand is written
    bool pre = false;
    {
        const long long tn = *next_tile;
        if (tn >= nCur && tn < nCur + nAff) {
            pre = true;
            if (tid == 32) {
                const long long en = (tn - nCur) * D::E;
                issue_tile_rows<N, AV, AV>(p, en, (int)min((long long)D::E, p.Kaff - en), sTr, &bars[3]);
            }
        }
    }

    // ---------------- cubature chunks: contravariant flux deviations.  The
    // two halves of the group work on alternate chunks (half h: chunks h,
    // h + 2, ...), each with its own A2 buffer (h), named barrier and MMA
    // issuer (its thread 0); half 0 accumulates into D2 after the face
    // chunk, half 1 into D2b.  Each warp of a half owns 8 elements (its 32
    // rows); with the rows ordered (variable, element) within the warp's 32
    // lanes, 16-lane TMEM loads hand each thread the 4 variables of one
    // element at 4 points of the chunk (2g, 2g + 1, 2g + 8, 2g + 9 with g =
    // lane % 4).  The chunk's K slots are ordered so that each pair of these
    // points has its r and s parts in 4 consecutive slots (the operator
    // table is packed to match): each row's values of a pair go out in one
    // 16-byte store, which the swizzled layout spreads over all banks.
    {
        const int el = lane >> 2, gq = lane & 3;          // element within the warp, point group
        const int ec = (warp & 3) * 8 + el;               // element in the tile
        const uint32_t tq = tD1 + ((uint32_t)((warp & 3) * 32) << 16);
        // the element's mean state, metric and negated contravariant mean
        // flux, each value in both halves of a pair (the flux of two points
        // is formed with packed pair instructions), in registers for all chunks
        float2 mu[4], cg[4], nfr[4], nfs[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float m = sMean[ec * 4 + i], gi = sGeo[ec * 16 + i];
            const float fr = -sFC[ec * 8 + i], fs = -sFC[ec * 8 + 4 + i];
            mu[i] = make_float2(m, m);
            cg[i] = make_float2(gi, gi);
            nfr[i] = make_float2(fr, fr);
            nfs[i] = make_float2(fs, fs);
        }
        const float2 gm1 = make_float2(p.gamma - 1.f, p.gamma - 1.f);
        // the fluxes of a pair of points (o = 0, 1) from its TMEM values:
        // lo = (v0 at o = 0, v0 at o = 1, v1 at 0, v1 at 1), hi the same for
        // variables 2 and 3
        auto pair_flux = [&](const float lo[4], const float hi[4], float2 Fr[4], float2 Fs[4]) {
            const float2 Uc[4] = {__fadd2_rn(make_float2(lo[0], lo[1]), mu[0]),
                                  __fadd2_rn(make_float2(lo[2], lo[3]), mu[1]),
                                  __fadd2_rn(make_float2(hi[0], hi[1]), mu[2]),
                                  __fadd2_rn(make_float2(hi[2], hi[3]), mu[3])};
            contra_flux2_dev(Uc, gm1, cg, nfr, nfs, Fr, Fs);
        };
        const int r0 = (warp & 3) * 32 + el;              // the element's row of variable 0
        unsigned char* A2 = smem + g.toff + (half ? S::sBUF1 : S::sA2);
        const uint32_t tDh = half ? tD2b : tD2;
        // a: variables 0, 1 at points 2g, 2g + 1; b: variables 2, 3 at
        // them; c, d: the same at points 2g + 8, 2g + 9
        float a[4], b[4], c[4], d[4];
        if constexpr (JOINT) {
            // the shared last chunk: half h forms the pair h of every
            // thread's points, into the buffer after the face chunk's
            tc::tmem_ld16x256(tq + (CQ - 1) * 16 + 8 * half, a);
            tc::tmem_ld16x256(tq + (16u << 16) + (CQ - 1) * 16 + 8 * half, b);
            tc::tmem_ld_wait4(a, b);
            float2 Fr[4], Fs[4];   // [variable], the two points in .x, .y
            pair_flux(a, b, Fr, Fs);
            wait_buf(buf_of(seq));
            unsigned char* AJ = a2_buf(seq);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const float x[4] = {Fr[w].x, Fr[w].y, Fs[w].x, Fs[w].y};
                store4_a2<PREC>(AJ, r0 + 8 * w, 8 * gq + 4 * half, x);
            }
            tc::fence_async_smem();
        }
        if (half < CP) tmem_ld_chunk(tq + half * 16, a, b, c, d);
        if constexpr (D2B || JOINT) {
            // the shared chunk's operand is complete, and D2b (over the
            // columns of chunks 0 and 1) is read before half 1's first product
            tc::fence_before_sync();
            g.sync();
            tc::fence_after_sync();
        }
        if constexpr (JOINT) {
            if (tid == 0) issue_chunk(seq, CF + CQ - 1);
            ph.commit(buf_of(seq));
            ++seq;
        }
        bool first = true;
#pragma unroll 1
        for (int cq = half; cq < CP; cq += 2) {
            if (LEAN && !first) tmem_ld_chunk(tq + cq * 16, a, b, c, d);
            // the next chunk's TMEM loads are issued now and waited for after
            // this chunk's products are issued: their latency overlaps the
            // flux arithmetic (the registers are read only after the wait).
            // Not in the lean layout's kernels, whose 80 registers a thread
            // (three pipelines per SM) leave no room for the 16 values.
            float na[4], nb[4], nc[4], nd[4];
            const bool more = !LEAN && cq + 2 < CP;
            if (more) {
                const uint32_t tn = tq + (cq + 2) * 16;
                tc::tmem_ld16x256(tn, na);
                tc::tmem_ld16x256(tn + (16u << 16), nb);
                tc::tmem_ld16x256(tn + 8, nc);
                tc::tmem_ld16x256(tn + (16u << 16) + 8, nd);
            }
            // the points in two pairs, each pair's fluxes stored as soon as
            // they are formed: (2g, 2g + 1) from a, b into slots 8g..8g+3,
            // (2g + 8, 2g + 9) from c, d into slots 8g+4..8g+7.  Padded
            // points (beyond NQ) carry the element mean, a finite value, and
            // meet zero operator columns.
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                float2 Fr[4], Fs[4];   // [variable], the two points in .x, .y
                pair_flux(pr ? c : a, pr ? d : b, Fr, Fs);
                if (pr == 0) wait_buf(half);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const float x[4] = {Fr[w].x, Fr[w].y, Fs[w].x, Fs[w].y};
                    store4_a2<PREC>(A2, r0 + 8 * w, 8 * gq + 4 * pr, x);
                }
            }
            tc::fence_async_smem();
            g.half_sync(half);
            if ((tid & 127) == 0) {
                tc::fence_after_sync();
                // half 0 accumulates onto the face (and viscous) chunks
                issue_mma_a2<PREC>(tDh, A2, smem + S::sB2 + (CF + cq) * B2C, N2, half == 0 || !first);
                tc::mma_commit(&bars[half]);
            }
            ph.commit(half);
            first = false;
            if (more) {
                tc::tmem_ld_wait4(na, nb);
                tc::tmem_ld_wait4(nc, nd);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    a[i] = na[i];
                    b[i] = nb[i];
                    c[i] = nc[i];
                    d[i] = nd[i];
                }
            }
        }
    }
    DGC_PHASE_MARK(6);

    // ---------------- epilogue: L = D2 / J into shared memory (the G1
    // operand region), then a coalesced pass over the tile for the stage
    // combination, whose inputs from global memory (U_s, and U^n or the
    // low-storage register) are loaded here, while the last products run
    const long long base = e0 * 4 * NP;
    const int n4 = ne * NP;   // float4 groups: ne * 4 * NP / 4
    // the stage combination of 4 values: U_out = a U^n + b (U_s + dt L), or
    // the low-storage form dU <- a dU + dt L (stored to *du), U = U_s + b dU
    auto combine = [&](const float4 L4, const float4 s4, const float4 n4v, float4* du) -> float4 {
        if (p.rhs_only) return L4;
        if (p.dU) {
            const float4 d = make_float4(p.a * n4v.x + p.dt * L4.x, p.a * n4v.y + p.dt * L4.y,
                                         p.a * n4v.z + p.dt * L4.z, p.a * n4v.w + p.dt * L4.w);
            *du = d;
            return make_float4(s4.x + p.b * d.x, s4.y + p.b * d.y, s4.z + p.b * d.z, s4.w + p.b * d.w);
        }
        float4 r = make_float4(p.b * (s4.x + p.dt * L4.x), p.b * (s4.y + p.dt * L4.y), p.b * (s4.z + p.dt * L4.z),
                               p.b * (s4.w + p.dt * L4.w));
        if (p.a != 0.f) {
            r.x += p.a * n4v.x;
            r.y += p.a * n4v.y;
            r.z += p.a * n4v.z;
            r.w += p.a * n4v.w;
        }
        return r;
    };
    // rows on 16-byte boundaries and no sensor in the epilogue: each thread
    // combines its own row's values straight from TMEM (no pass through
    // shared memory); its U_s and U^n values are loaded here
    constexpr bool DIRECT = (NP % 4 == 0) && !SENSE;
    constexpr int per_half = N2 / 2;
    static_assert(!DIRECT || per_half % 8 == 0, "whole 8-column TMEM loads per half row");
    constexpr int NV4 = DIRECT ? per_half / 4 : 1;
    const long long rbase = base + (long long)(e * 4 + v) * NP + half * per_half;   // this thread's first value
    if constexpr (DIRECT) {
        float4 rs[NV4], rn[NV4];
        {
            const float4* us = reinterpret_cast<const float4*>(p.Us + rbase);
            const float4* un = reinterpret_cast<const float4*>((p.dU ? p.dU : p.Un) + rbase);
            const bool need = !p.rhs_only && p.a != 0.f;
#pragma unroll
            for (int k = 0; k < NV4; ++k) {
                const bool ok = live && half * per_half + 4 * k < NP;
                rs[k] = (ok && !p.rhs_only) ? us[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                rn[k] = (ok && need) ? un[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        wait_buf(half);
        {
            constexpr uint32_t n0 = (CP + 1) / 2, n1 = CP / 2;
            if (half) {
                ph.c0 += n0;
            } else {
                ph.c1 += n1;
            }
        }
        tc::fence_before_sync();
        g.sync();
        tc::fence_after_sync();
        ph.w0 = ph.c0;
        ph.w1 = ph.c1;
        const float invJ = sGeo[e * 16 + 4];
        float4* uo = reinterpret_cast<float4*>(p.Uout + rbase);
        float4* du = reinterpret_cast<float4*>(p.dU ? p.dU + rbase : p.Uout + rbase);
#pragma unroll
        for (int c0 = 0; c0 < per_half; c0 += 8) {
            float x[8], y[8];
            const int i0 = half * per_half + c0;
            tc::tmem_ld8(tD2 + lane_base + i0, x);
            if constexpr (D2B) {
                tc::tmem_ld8(tD2b + lane_base + i0, y);
                tc::tmem_ld_wait(x, y);
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] += y[i];
            } else {
                tc::tmem_ld_wait(x);
            }
#pragma unroll
            for (int i = 0; i < 8; i += 4) {
                const int k = (c0 + i) / 4;
                if (live && i0 + i < NP) {
                    const float4 L4 = make_float4(x[i] * invJ, x[i + 1] * invJ, x[i + 2] * invJ, x[i + 3] * invJ);
                    float4 dv;
                    const float4 r = combine(L4, rs[k], rn[k], &dv);
                    if (p.dU && !p.rhs_only) du[k] = dv;
                    uo[k] = r;
                }
            }
        }
        tc::fence_before_sync();   // this tile's TMEM reads precede the next tile's products
        g.sync();                  // staging and per-element data are reused by the next tile
        DGC_PHASE_MARK(7);
        return pre;
    }
    constexpr int NI = (32 * NP + THREADS - 1) / THREADS;
    float4 pre_s[NI], pre_n[NI];
    {
        const float4* us = reinterpret_cast<const float4*>(p.Us + base);
        const float4* un = reinterpret_cast<const float4*>((p.dU ? p.dU : p.Un) + base);
        const bool need = !p.rhs_only && p.a != 0.f;
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int i = tid + k * THREADS;
            pre_s[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            pre_n[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n4) {
                if (!p.rhs_only) pre_s[k] = us[i];
                if (need) pre_n[k] = un[i];
            }
        }
    }
    // every product of this half has completed; those of the other half
    // after the barrier below (their commits are counted here without
    // waiting for them, all of them complete then)
    wait_buf(half);
    {
        constexpr uint32_t n0 = (CP + 1) / 2, n1 = CP / 2;   // cubature chunks of halves 0 and 1
        if (half) {
            ph.c0 += n0;
        } else {
            ph.c1 += n1;
        }
    }
    tc::fence_before_sync();
    g.sync();
    tc::fence_after_sync();
    ph.w0 = ph.c0;
    ph.w1 = ph.c1;
    {
        float* sOut = reinterpret_cast<float*>(smem + g.toff + S::sA1);
        const float invJ = sGeo[e * 16 + 4];
        constexpr int per_half = N2 / 2;
        constexpr int ES = S::ES;
#pragma unroll
        for (int c0 = 0; c0 < per_half; c0 += 8) {
            float x[8], y[8];
            const int i0 = half * per_half + c0;
            tc::tmem_ld8(tD2 + lane_base + i0, x);
            if constexpr (D2B) {
                tc::tmem_ld8(tD2b + lane_base + i0, y);
                tc::tmem_ld_wait(x, y);
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] += y[i];
            } else {
                tc::tmem_ld_wait(x);
            }
            float* orow = sOut + e * ES + v * NP;
            if constexpr (NP % 4 == 0) {   // rows on 16-byte boundaries
#pragma unroll
                for (int i = 0; i < 8; i += 4)
                    if (i0 + i < NP)
                        *reinterpret_cast<float4*>(orow + i0 + i) =
                            make_float4(x[i] * invJ, x[i + 1] * invJ, x[i + 2] * invJ, x[i + 3] * invJ);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < NP) orow[i0 + i] = x[i] * invJ;
            }
        }
        tc::fence_before_sync();
        g.sync();
        float4* uo = reinterpret_cast<float4*>(p.Uout + base);
        float4* lo = reinterpret_cast<float4*>(sOut);
        // float4 group i of the tile in the padded rows of sOut
        auto lo_at = [&](int i) -> int {
            if constexpr (ES == 4 * NP) return i;
            else return i + i / NP;
        };
        const bool sense = SENSE && p.eps_next != nullptr && !p.rhs_only;
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int i = tid + k * THREADS;
            if (i >= n4) break;
            const float4 L4 = lo[lo_at(i)];
            float4 dv;   // low-storage RK: pre_n holds dU (zero when a = 0)
            const float4 r = combine(L4, pre_s[k], pre_n[k], &dv);
            if (p.dU && !p.rhs_only) reinterpret_cast<float4*>(p.dU + base)[i] = dv;
            uo[i] = r;
            if (sense) lo[lo_at(i)] = r;
        }
        if constexpr (SENSE) {
            // the next stage's eps: the sensor of the new state, 4 threads per
            // element over the modes u = V^-1 rho (FP32 sums, FP64 ratio)
            if (sense) {
                g.sync();
                {
                    constexpr int NLOW = N * (N + 1) / 2;
                    constexpr int MT = (NP + 7) / 8;   // modes per thread, 8 threads per element
                    const float* sVinvT = reinterpret_cast<const float*>(smem + S::sVI);
                    const int ee = tid >> 3, sub = tid & 7;
                    const float* rho = sOut + ee * ES;
                    float um[MT];
#pragma unroll
                    for (int t = 0; t < MT; ++t) um[t] = 0.f;
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const float rj = rho[j];
#pragma unroll
                        for (int t = 0; t < MT; ++t) {
                            const int m = sub + 8 * t;
                            if (m < NP) um[t] += sVinvT[j * NP + m] * rj;
                        }
                    }
                    float num = 0.f, den = 0.f;
#pragma unroll
                    for (int t = 0; t < MT; ++t) {
                        const int m = sub + 8 * t;
                        if (m < NP) {
                            den += um[t] * um[t];
                            if (m >= NLOW) num += um[t] * um[t];
                        }
                    }
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        num += __shfl_xor_sync(0xffffffffu, num, o);
                        den += __shfl_xor_sync(0xffffffffu, den, o);
                    }
                    if (sub == 0) {
                        sND[2 * ee] = num;
                        sND[2 * ee + 1] = den;
                    }
                }
                g.sync();
                // the FP64 ratio, log10 and ramp for the 32 elements by one warp
                // (one lane per element): GB300's FP64 pipe is narrow
                if (warp == 7) {
                    float ev = 0.f;
                    if (lane < ne) {
                        ev = sensor_eps(p, sND[2 * lane], sND[2 * lane + 1]);
                        p.eps_next[e0 + lane] = ev;
                    }
                    if (p.visc != nullptr && __any_sync(0xffffffffu, ev > 0.f) && lane == 0) atomicAdd(p.visc, 1);
                }
            }
        }
        tc::fence_before_sync();   // this tile's TMEM reads precede the next tile's products
        g.sync();                  // staging and per-element data are reused by the next tile
    DGC_PHASE_MARK(7);
    }
    return pre;
}

template <int N, bool AV, bool SENSE = AV>
__device__ __forceinline__ void load_tc_operators(const unsigned char* ops_tc, unsigned char* smem,
                                                  bool common = true, bool extra = true) {
    using S = TcSmem<N, AV, SENSE>;
    using L = TcLayout<N>;
    using D = TcDims<N>;
    constexpr int NF = TcDims<N>::NF, NP = TcDims<N>::NP;
    const int tid = threadIdx.x;
    const int4* src = reinterpret_cast<const int4*>(ops_tc);
    int4* dst = reinterpret_cast<int4*>(smem);
    if (common) {   // the part every launch of this kind of kernel uses
        for (int i = tid; i < L::B1_BYTES / 16; i += blockDim.x) dst[i] = src[i];
        constexpr int NC = D::CF + D::CQ;   // face and cubature chunks
        for (int i = tid; i < NC * L::B2_CHUNK / 16; i += blockDim.x) dst[S::sB2 / 16 + i] = src[L::B2 / 16 + i];
        const float* igs = reinterpret_cast<const float*>(ops_tc + L::IGF);
        float* igd = reinterpret_cast<float*>(smem + S::sIGF);
        for (int i = tid; i < NF * NP; i += blockDim.x) igd[i] = igs[i];
        if constexpr (SENSE) {
            const float* vs = reinterpret_cast<const float*>(ops_tc + L::VINV);
            float* vd = reinterpret_cast<float*>(smem + S::sVI);
            for (int i = tid; i < NP * NP; i += blockDim.x) vd[i] = vs[i];
        }
    }
    if constexpr (AV) {
        if (extra) {   // the viscous chunks and I_g for q
            constexpr int NC = D::CF + D::CQ;
            for (int i = tid; i < D::CA * L::B2_CHUNK / 16; i += blockDim.x)
                dst[(S::sB2 + NC * L::B2_CHUNK) / 16 + i] = src[(L::B2 + NC * L::B2_CHUNK) / 16 + i];
            for (int i = tid; i < L::B1Q_BYTES / 16; i += blockDim.x) dst[S::sB1Q / 16 + i] = src[L::B1Q / 16 + i];
        }
    }
}

// Tile pipelines per CTA: as many groups of 256 threads as the shared memory
// holds beside one copy of the operator tables (at most two).  Each group
// works on its own tile with its own regions, mbarriers and TMEM columns; the
// operators are loaded once per CTA and shared.  STRIDE: the byte distance
// between the groups' per-tile regions (the larger of the viscous layout and
// the inviscid one of an AV launch).
// Tile-pipeline configurations of the stage kernel, code = 10 C + P: C CTAs
// per SM (the minimum the launch bounds ask for) of P pipelines of 256
// threads, each pipeline working on its own tile with its own per-tile
// shared-memory region, mbarriers, TMEM columns and named barrier; the
// operator tables are loaded once per CTA and shared.  STRIDE: the byte
// distance between the pipelines' per-tile regions (the larger of the
// viscous layout and the inviscid one of an AV launch).  FITS: the
// configuration fits an SM (shared memory, TMEM).  LEAN_: the lean
// per-tile layout (one A2 buffer, D2 over D1's face columns; inviscid).
template <int N, bool AV, int P_, int C_, bool LEAN_ = false>
struct TcPipes {
    static_assert(!(LEAN_ && AV), "the lean layout is inviscid");
    using SV = TcSmem<N, AV, AV, LEAN_>;
    using SI = TcSmem<N, false, AV, LEAN_>;
    static constexpr int P = P_, MIN_CTAS = C_, CODE = 100 * LEAN_ + 10 * C_ + P_;
    static constexpr int mx(int a, int b) { return a > b ? a : b; }
    static constexpr int STRIDE = (mx(SV::TOTAL - SV::sA1, SI::TOTAL - SI::sA1) + 1023) / 1024 * 1024;
    // TMEM columns of one pipeline: D1, the q traces (AV), D2 (lean: in D1)
    static constexpr int COLS = TcDims<N>::N1 + (LEAN_ ? 0 : (AV ? 2 * TcDims<N>::NFP : 0) + TcDims<N>::N2);
    static constexpr int pow2(int c) { return c <= 32 ? 32 : 2 * pow2((c + 1) / 2); }
    static constexpr int ALLOC = pow2(P * COLS);   // one allocation for all pipelines (a power of two)
    static_assert(STRIDE % 1024 == 0 || P == 1, "pipelines' regions on 1024-byte boundaries");
    // + up to 1 KB to align the dynamic shared memory to 1024 bytes
    static constexpr int BYTES = SV::TOTAL + (P - 1) * STRIDE + 1024;
    static constexpr int CTA_THREADS = P * THREADS;
    // per block: dynamic + static (< 512 B) + the 1 KB the runtime reserves; per SM 228 KB
    static constexpr bool FITS = BYTES + 512 + 1024 <= 232448 && C_ * (BYTES + 512 + 1024) <= 233472 &&
                                 C_ * ALLOC <= 512 && (!LEAN_ || SV::LEAN_OK);
    static_assert(SI::TOTAL <= SV::TOTAL, "the inviscid layout of an AV launch fits the viscous one");
    // elements of a curved tile: a pipeline runs it on the CUDA-core body in
    // its own per-tile region (of the smaller of the two layouts' regions)
    static constexpr int REGION = mx(SV::TOTAL - SV::sA1, 0) < mx(SI::TOTAL - SI::sA1, 0)
                                      ? SV::TOTAL - SV::sA1 : SI::TOTAL - SI::sA1;
    static constexpr int ec_fit(int e) {
        return (e <= 1 || Tile<N, float>::smem_stage(AV, e) <= (size_t)REGION) ? e : ec_fit(e - 1);
    }
    static constexpr int EC = ec_fit(Tile<N, float>::E);
    static_assert(Tile<N, float>::smem_stage(AV, EC) <= (size_t)REGION, "a curved tile fits a pipeline's region");
};

// The candidate configurations of a degree and viscosity setting, fitting
// ones only: two CTAs of one pipeline, one CTA of two or three pipelines,
// three lean pipelines (113) where three full ones do not fit (inviscid),
// and one CTA of one pipeline where nothing larger fits.  The default (the
// first): two single-pipeline CTAs where they fit (measured: they overlap
// the next kernel's start better), else the most pipelines that fit (the
// lean three before two full ones: measured 11% faster at N = 6).
template <int N, bool AV>
struct TcConfigs {
    static constexpr bool f21 = TcPipes<N, AV, 1, 2>::FITS, f12 = TcPipes<N, AV, 2, 1>::FITS,
                          f13 = TcPipes<N, AV, 3, 1>::FITS;
    static constexpr bool lean3() {
        if constexpr (AV) return false;
        else return !f13 && TcPipes<N, false, 3, 1, true>::FITS;
    }
    static constexpr bool f113 = lean3();
    static constexpr bool f11 = !f21 && !f12 && !f13 && !f113;
    static int list(int* out) {
        int n = 0;
        if (f21) out[n++] = 21;
        if (f13) out[n++] = 13;
        if (f113) out[n++] = 113;
        if (f12) out[n++] = 12;
        if (f11) out[n++] = 11;
        return n;
    }
    static constexpr int deflt() { return f21 ? 21 : f13 ? 13 : f113 ? 113 : f12 ? 12 : 11; }
};

// Persistent grid, one CTA per SM.  Each CTA sets up its mbarriers and TMEM
// and loads the operator tables once; each tile pipeline then claims tiles
// from an atomic counter on its own: first the curved tiles (CUDA-core body
// in the pipeline's region), then the affine tiles of 32 elements on the
// tensor cores.  Handing the slow curved tiles out first lets them overlap
// the affine work instead of forming a tail.
//
// With artificial viscosity, a launch whose input state has no element with
// eps > 0 (the count of viscous tiles comes with eps from the kernel that
// wrote it) runs the inviscid tile body with the next stage's sensor in its
// epilogue: the viscous terms are sqrt(eps) q, all zero then.  The last CTA
// resets that count for the slot's next use.
template <int N, bool AV, int PREC, int P_, int C_, bool LEAN_ = false>
__global__ void __launch_bounds__(P_ * THREADS, C_)
    stage_kernel_tc(StageArgs<float> p, const unsigned char* ops_tc, int* err, int* counter, int* done) {
    using PP = TcPipes<N, AV, P_, C_, LEAN_>;
    constexpr int P = PP::P;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // the A2 buffers' 128-byte swizzle works on address bits: the layout
    // starts on a 1024-byte boundary (the launch adds 1 KB for this)
    unsigned char* smem_tc = smem_dyn + ((1024u - (tc::smem_addr(smem_dyn) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t bars[4 * P];
    __shared__ uint32_t slot;
    __shared__ int s_tile[P];
    __shared__ int s_visc;
    constexpr int ET = TcDims<N>::E, EC = PP::EC, COLS = PP::COLS;
    const int tid = threadIdx.x, pipe = tid / THREADS;
    const TcGroup g{tid - pipe * THREADS, (uint32_t)(1 + pipe), (uint32_t)(pipe * PP::STRIDE),
                    (uint32_t)(1 + P + 2 * pipe)};
    const long long nAff = (p.Kaff + ET - 1) / ET;
    const long long nCur = (p.K - p.Kaff + EC - 1) / EC;
#ifdef DGC_PHASE_CLOCKS
    const long long dgc_k0 = clock64();
#endif

    // prologue (barriers, TMEM, operators) overlaps the previous kernel
    tc::pdl_trigger();
    if (tid == 0) {
        for (int b = 0; b < 4 * P; ++b) tc::mbar_init(&bars[b], 1);
        tc::mbar_fence_init();
    }
    if ((tid >> 5) == 0) tc::tmem_alloc(&slot, PP::ALLOC);
    bool viscous = true;
    if constexpr (AV) {
        // the operators both kinds of launch use, then the kind of launch
        // (known once the previous kernel is done) and the viscous extras
        load_tc_operators<N, true>(ops_tc, smem_tc, true, false);
        tc::pdl_wait();
        if (tid == 0) s_visc = (p.visc_in == nullptr) || *reinterpret_cast<volatile int*>(p.visc_in) > 0;
        __syncthreads();
        viscous = s_visc != 0;
        if (viscous) load_tc_operators<N, true>(ops_tc, smem_tc, false, true);
    } else {
        load_tc_operators<N, false>(ops_tc, smem_tc);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = slot + (uint32_t)(pipe * COLS);
    TcPhase ph;
    tc::pdl_wait();

    // each pipeline claims tiles on its own: first the curved tiles (the
    // CUDA-core body in the pipeline's own region; the shared operator
    // tables stay loaded), then affine tiles of 32 elements on the tensor
    // cores
    unsigned char* region = smem_tc + (viscous ? PP::SV::sA1 : PP::SI::sA1) + g.toff;
    const TileThreads th{g.tid, THREADS, g.bar};
#ifdef DGC_PHASE_CLOCKS
    if (g.tid == 0) atomicAdd(&g_tc_phase_cycles[11], (unsigned long long)(clock64() - dgc_k0));
#endif
    if (g.tid == 0) s_tile[pipe] = atomicAdd(counter, 1);
    g.sync();
    long long t = s_tile[pipe];
    bool rows_ready = false;
    while (t < nCur + nAff) {
        g.sync();   // every thread of the pipeline has read its s_tile
        // claim the following tile now; the result is stored late in the tile
        const int claim = (g.tid == THREADS - 1) ? atomicAdd(counter, 1) : 0;
        if (t < nCur) {
            TileRange tr;
            tr.curved = true;
            tr.e0 = p.Kaff + t * EC;
            tr.ne = (int)min((long long)EC, p.K - tr.e0);
#ifdef DGC_PHASE_CLOCKS
            const long long dgc_c0 = clock64();
#endif
            stage_tile_call<N, float, AV>(p, tr, region, th, EC);
#ifdef DGC_PHASE_CLOCKS
            if (g.tid == 0) {
                atomicAdd(&g_tc_phase_cycles[9], (unsigned long long)(clock64() - dgc_c0));
                atomicAdd(&g_tc_phase_cycles[10], 1ull);
            }
#endif
            rows_ready = false;
            if (g.tid == THREADS - 1) s_tile[pipe] = claim;
            g.sync();
        } else {
            const long long e0 = (t - nCur) * ET;
            const int ne = (int)min((long long)ET, p.Kaff - e0);
            uint64_t* pb = bars + 4 * pipe;
            if constexpr (AV) {
                if (viscous)
                    rows_ready = stage_tile_tc<N, true, PREC>(p, e0, ne, smem_tc, tmem, ph, err, rows_ready, claim,
                                                              &s_tile[pipe], nCur, nAff, pb, g);
                else
                    rows_ready = stage_tile_tc<N, false, PREC, true>(p, e0, ne, smem_tc, tmem, ph, err, rows_ready,
                                                                     claim, &s_tile[pipe], nCur, nAff, pb, g);
            } else {
                rows_ready = stage_tile_tc<N, false, PREC, false, LEAN_>(p, e0, ne, smem_tc, tmem, ph, err,
                                                                         rows_ready, claim, &s_tile[pipe], nCur,
                                                                         nAff, pb, g);
            }
        }
        t = s_tile[pipe];
    }
#ifdef DGC_PHASE_CLOCKS
    if (g.tid == 0) {
        atomicAdd(&g_tc_phase_cycles[12], (unsigned long long)(clock64() - dgc_k0));
        atomicAdd(&g_tc_phase_cycles[13], 1ull);
    }
#endif
    // the last CTA to leave resets the counters for the next launch
    __threadfence();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && atomicAdd(done, 1) == (int)gridDim.x - 1) {
        __threadfence();
        *counter = 0;
        *done = 0;
        if (AV && p.visc_in != nullptr) *p.visc_in = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_free(slot, PP::ALLOC);
}

// Persistent grid size per instantiation: SMs x resident CTAs, set by
// prepare_tc before any launch.
template <int N, bool AV, int PREC, int P_, int C_, bool LEAN_ = false>
struct TcGrid {
    static inline int ctas = 0;
};

template <int N, bool AV, int PREC, int P_, int C_, bool LEAN_ = false>
int prepare_tc_t() {
    using PP = TcPipes<N, AV, P_, C_, LEAN_>;
    if constexpr (!PP::FITS) {
        return 0;
    } else {
        auto kern = stage_kernel_tc<N, AV, PREC, P_, C_, LEAN_>;
        const int sm = PP::BYTES;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return (int)e;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
            return (int)e;
        int occ = resident_ctas((const void*)kern, PP::CTA_THREADS, sm), dev = 0, nsm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
        const int by_tmem = 512 / PP::ALLOC;
        occ = occ < by_tmem ? occ : by_tmem;
        if (occ < 1) return (int)cudaErrorInvalidConfiguration;
        if (getenv("DGC_VERBOSE"))
            fprintf(stderr, "dgcurved: stage_kernel_tc N=%d AV=%d config %d: %d CTAs per SM, %d B shared memory\n", N,
                    (int)AV, PP::CODE, occ, sm);
        TcGrid<N, AV, PREC, P_, C_, LEAN_>::ctas = nsm * occ;
        return 0;
    }
}

// err[0]: error word; err[1]: tile counter, err[3]: CTAs done (both zero
// between launches: the last CTA resets them).
template <int N, bool AV, int PREC, int P_, int C_, bool LEAN_ = false>
int launch_stage_tc_t(const StageArgs<float>& a, const unsigned char* ops_tc, int* err, cudaStream_t st) {
    using PP = TcPipes<N, AV, P_, C_, LEAN_>;
    if constexpr (!PP::FITS) {
        return (int)cudaErrorInvalidConfiguration;
    } else {
        constexpr int ET = TcDims<N>::E, EC = PP::EC;
        const long long tiles = (a.Kaff + ET - 1) / ET + (a.K - a.Kaff + EC - 1) / EC;
        if (tiles == 0) return 0;
        const int ctas = TcGrid<N, AV, PREC, P_, C_, LEAN_>::ctas;
        if (ctas <= 0) return (int)cudaErrorNotReady;   // prepare_tc was not called
        // the tile and neighbour records travel by TMA bulk copies: 16-byte aligned
        if (((uintptr_t)a.Us | (uintptr_t)a.Un | (uintptr_t)a.Uout | (uintptr_t)a.q | (uintptr_t)a.dU |
             (uintptr_t)ops_tc) & 15)
            return (int)cudaErrorMisalignedAddress;
        const long long need = (tiles + PP::P - 1) / PP::P;
        const unsigned grid = (unsigned)(need < ctas ? need : ctas);
        return (int)launch_pdl(stage_kernel_tc<N, AV, PREC, P_, C_, LEAN_>, grid, PP::CTA_THREADS, (size_t)PP::BYTES, st, a,
                               ops_tc, err, err + 1, err + 3);
    }
}

// One precision and viscosity setting: the configuration cfg (0: the default).
template <int N, bool AV, int PREC>
int launch_stage_tc_cfg(const StageArgs<float>& a, const unsigned char* ops_tc, int* err, cudaStream_t st, int cfg) {
    if (cfg == 0) cfg = TcConfigs<N, AV>::deflt();
    using C = TcConfigs<N, AV>;
    switch (cfg) {
        case 21:
            if constexpr (C::f21) return launch_stage_tc_t<N, AV, PREC, 1, 2>(a, ops_tc, err, st);
            break;
        case 12:
            if constexpr (C::f12) return launch_stage_tc_t<N, AV, PREC, 2, 1>(a, ops_tc, err, st);
            break;
        case 13:
            if constexpr (C::f13) return launch_stage_tc_t<N, AV, PREC, 3, 1>(a, ops_tc, err, st);
            break;
        case 113:
            if constexpr (C::f113) return launch_stage_tc_t<N, AV, PREC, 3, 1, true>(a, ops_tc, err, st);
            break;
        case 11:
            if constexpr (C::f11) return launch_stage_tc_t<N, AV, PREC, 1, 1>(a, ops_tc, err, st);
            break;
    }
    return (int)cudaErrorInvalidValue;
}

template <int N, bool AV, int PREC>
int prepare_tc_av() {
    using C = TcConfigs<N, AV>;
    int e = 0;
    if constexpr (C::f21) e = e ? e : prepare_tc_t<N, AV, PREC, 1, 2>();
    if constexpr (C::f12) e = e ? e : prepare_tc_t<N, AV, PREC, 2, 1>();
    if constexpr (C::f13) e = e ? e : prepare_tc_t<N, AV, PREC, 3, 1>();
    if constexpr (C::f113) e = e ? e : prepare_tc_t<N, AV, PREC, 3, 1, true>();
    if constexpr (C::f11) e = e ? e : prepare_tc_t<N, AV, PREC, 1, 1>();
    return e;
}

template <int N, int PREC>
int prepare_tc_prec() {
    const int e = prepare_tc_av<N, false, PREC>();
    return e ? e : prepare_tc_av<N, true, PREC>();
}

template <int N>
int tc_configs_n(int av, int* out4) {
    return av ? TcConfigs<N, true>::list(out4) : TcConfigs<N, false>::list(out4);
}

// The per-precision halves (one translation unit each, compiled in parallel).
template <int N, int PREC>
int launch_stage_tc_prec(const StageArgs<float>& a, int av, const unsigned char* ops_tc, int* err, cudaStream_t st,
                         int cfg) {
    return av ? launch_stage_tc_cfg<N, true, PREC>(a, ops_tc, err, st, cfg)
              : launch_stage_tc_cfg<N, false, PREC>(a, ops_tc, err, st, cfg);
}

// ---------------------------------------------------------------------------
// host: operator table of the tensor-core path
// ---------------------------------------------------------------------------
inline uint32_t host_tf32_bits(double x) {
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x1000u;          // round to nearest, ties away from zero, at 10 mantissa bits
    u &= ~0x1FFFu;
    return u;
}
inline uint16_t host_bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even
    return (uint16_t)(u >> 16);
}
inline float host_bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Write an operand matrix M[rows][K] (value(row, k)) into the core-matrix
// layout: TF32 (4-byte, rounded) or BF16 high block followed by low block.
template <typename F>
inline void pack_operand(std::vector<uint8_t>& out, size_t off, int rows, int K, int prec, F value) {
    if (prec == PREC_TF32) {
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < K; ++k) {
                const uint32_t b = host_tf32_bits(value(r, k));
                std::memcpy(&out[off + tc::cm_offset(r, k * 4, K * 4)], &b, 4);
            }
    } else {
        const size_t lo = (size_t)rows * K * 2;
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < K; ++k) {
                const float x = (float)value(r, k);
                const uint16_t h = host_bf16_bits(x);
                const uint16_t l = host_bf16_bits(x - host_bf16_value(h));
                std::memcpy(&out[off + tc::cm_offset(r, k * 2, K * 2)], &h, 2);
                std::memcpy(&out[off + lo + tc::cm_offset(r, k * 2, K * 2)], &l, 2);
            }
    }
}

template <int N>
std::vector<uint8_t> pack_ops_tc(const RefOps& R, int prec) {
    using D = TcDims<N>;
    using L = TcLayout<N>;
    constexpr int NP = D::NP, NQ = D::NQ, NF = D::NF;
    std::vector<uint8_t> out(L::TOTAL, 0);
    auto Icub = [&](int q, int j) { return R.Icub[(size_t)q * NP + j]; };
    auto Ig = [&](int fg, int j) { return R.Ig[(size_t)fg * NP + j]; };
    pack_operand(out, L::B1, D::N1, D::NPK, prec, [&](int r, int k) -> double {
        if (k >= NP) return 0.0;
        if (r < NQ) return Icub(r, k);
        if (r >= D::FOFF && r < D::FOFF + NF) return Ig(r - D::FOFF, k);
        return 0.0;
    });
    pack_operand(out, L::B1Q, D::NFP, D::NPK, prec,
                 [&](int r, int k) -> double { return (r < NF && k < NP) ? Ig(r, k) : 0.0; });
    for (int c = 0; c < D::NCH; ++c) {
        pack_operand(out, L::B2 + (size_t)c * L::B2_CHUNK, D::N2, 32, prec, [&](int i, int s) -> double {
            if (i >= NP) return 0.0;
            if (c < D::CF) {
                const int fg = c * 32 + s;
                if (fg < NF) return -R.MLift[(size_t)i * NF + fg];
                if (fg < NF + 2 * D::NQF) {   // folded cubature point: r part, then s part
                    const int q = D::CQ * 16 + (fg - NF) / 2;
                    return ((fg - NF) & 1) ? R.MsW[(size_t)i * NQ + q] : R.MrW[(size_t)i * NQ + q];
                }
                return 0.0;
            }
            if (c < D::CF + D::CQ) {
                // slots 8 g .. 8 g + 7 hold the points one thread of the
                // tile body forms, in two pairs: the r parts of points 2 g,
                // 2 g + 1, their s parts, then the same of 2 g + 8, 2 g + 9
                const int gq = s >> 3, pair = (s >> 2) & 1, part = (s >> 1) & 1, j = s & 1;
                const int pt = 2 * gq + j + 8 * pair;
                const int q = (c - D::CF) * 16 + pt;
                if (q >= NQ) return 0.0;
                return part == 0 ? R.MrW[(size_t)i * NQ + q] : R.MsW[(size_t)i * NQ + q];
            }
            const int j = (c - D::CF - D::CQ) * 16 + (s & 15);
            if (j >= NP) return 0.0;
            return s < 16 ? -R.Qr[(size_t)i * NP + j] : -R.Qs[(size_t)i * NP + j];
        });
    }
    // the traces as 1D interpolation from each face's N + 1 nodes (the
    // nodes on a face carry the restriction of the degree-N polynomial):
    // E[f][g][k] = I_g[f][g][fmask[f][k]], all other entries of I_g vanish
    {
        constexpr int NG = D::NG, NE = TcDims<N>::NE;
        std::vector<int> fm(3 * NE, -1);
        for (int f = 0; f < 3; ++f) {
            int k = 0;
            for (int j = 0; j < NP; ++j) {
                double mxv = 0.0;
                for (int g = 0; g < NG; ++g) mxv = std::max(mxv, std::fabs(Ig(f * NG + g, j)));
                if (mxv > 1e-9) {
                    if (k >= NE) return {};   // more nodes on a face than a degree-N trace needs
                    fm[f * NE + k++] = j;
                } else if (mxv > 1e-12) {
                    return {};
                }
            }
            if (k != NE) return {};
        }
        for (int f = 0; f < 3; ++f)
            for (int g = 0; g < NG; ++g)
                for (int k = 0; k < NE; ++k) {
                    const float v = (float)Ig(f * NG + g, fm[f * NE + k]);
                    std::memcpy(&out[L::IGF + ((size_t)(f * NG + g) * NE + k) * 4], &v, 4);
                }
        std::memcpy(&out[L::IGF + (size_t)3 * NG * NE * 4], fm.data(), 3 * NE * sizeof(int));
    }
    for (int j = 0; j < NP; ++j)
        for (int m = 0; m < NP; ++m) {
            const float f = (float)R.Vinv[(size_t)m * NP + j];
            std::memcpy(&out[L::VINV + ((size_t)j * NP + m) * 4], &f, 4);
        }
    pack_operand(out, L::B2F3, 3 * D::N2, 32, prec, [&](int r, int c) -> double {
        const int f = r / D::N2, i = r - f * D::N2;
        if (i >= NP || c < f * D::NG || c >= (f + 1) * D::NG) return 0.0;
        return -R.MLift[(size_t)i * NF + c];
    });
    pack_operand(out, L::BQ, 2 * D::N2, D::NPK, prec, [&](int r, int j) -> double {
        if (j >= NP) return 0.0;
        if (r < D::N2) return r < NP ? R.Qr[(size_t)r * NP + j] : 0.0;
        const int i = r - D::N2;
        return i < NP ? R.Qs[(size_t)i * NP + j] : 0.0;
    });
    return out;
}

}  // namespace dgc

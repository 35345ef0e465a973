// Inline-PTX helpers for the fifth-generation tensor cores (tcgen05) and
// mbarriers on sm_103a.  Operands live in shared memory in the K-major,
// no-swizzle core-matrix layout: a core matrix is 8 rows x 16 bytes stored
// contiguously (128 B); core matrices adjacent along K are LBO = 128 B apart
// and 8-row groups are SBO = (row bytes / 16) * 128 B apart.  Accumulators
// live in tensor memory (TMEM), M = 128 lanes x N 32-bit columns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgc {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of an operand tile whose rows hold
// row_bytes bytes of K, in the core-matrix layout above.
__host__ __device__ __forceinline__ uint32_t cm_offset(uint32_t row, uint32_t kbyte, uint32_t row_bytes) {
    return (row >> 3) * (row_bytes / 16) * 128 + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15);
}

// Shared-memory matrix descriptor (SWIZZLE_NONE, version 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t row_bytes) {
    const uint32_t lbo = 128, sbo = (row_bytes / 16) * 128;
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// The same descriptor with explicit strides (bytes, multiples of 128): lbo
// between core matrices adjacent along K, sbo between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// The 128-byte-swizzled K-major layout of an operand whose rows hold
// exactly 128 bytes of K: eight rows form a 1024-byte atom (rows 128 bytes
// apart, atoms 1024 bytes apart), and the 16-byte piece c of row r sits at
// piece position c XOR (r mod 8) of its row.  The swizzle is applied to
// shared-memory address bits, so an operand in this layout must start on a
// 1024-byte boundary.  Byte offset of byte `kbyte` (0..127) of row `row`:
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t kbyte) {
    return (row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ row) & 7) << 4) + (kbyte & 15);
}

// Shared-memory matrix descriptor of that layout (layout type 2 =
// 128-byte swizzle; the stride between 8-row atoms 1024 bytes; the leading
// offset is not used by a K-major swizzled operand and is set to 16 bytes).
// A product over K bytes [32 k, 32 k + 32) of each row starts at saddr + 32 k.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M x N.
// fmt: 2 = TF32 (kind::tf32), 1 = BF16 (kind::f16).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// Arrive on an mbarrier once every previously issued tcgen05.mma of this
// thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;"); }

// Bounded wait for the given phase parity.  Returns false if the limit ran
// out (the caller records an error and skips the dependent work).
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    return done != 0;
}
// Bounded wait for the phase with the given parity: at most `limit` waits,
// each suspending the thread until the phase completes or for up to about
// 1 ms (the suspend-time hint), and at most 2 s in all.  False if the limit
// ran out (the caller records an error and carries on).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = 1u << 26) {
    const uint32_t a = smem_addr(mbar);
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(a), "r"(parity), "r"(1000000u) : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// Transaction-count arrival: the current phase also waits for `bytes`
// bytes of bulk copies signalling this barrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// TMA bulk copy global -> shared (this CTA), completion counted in bytes on
// mbar.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}

// Bulk prefetch of global memory into L2 (no completion to wait for): both
// the address and the size multiples of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}

// Per-thread asynchronous copies global -> shared (16 bytes through L2 only;
// 4 bytes), and the wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Programmatic dependent launch: let the next kernel of the stream start its
// prologue on SMs this grid leaves, and wait for the previous kernel of the
// stream to complete (with its memory visible) before reading its results.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one full warp; the address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

// 8 consecutive 32-bit columns of this thread's lane (warp-wide, aligned).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// 16 lanes x 8 columns (warp-wide, aligned; taddr's lane field is the first
// of the 16 lanes): thread t gets lane t/4 in v[0], v[1] and lane 8 + t/4 in
// v[2], v[3], columns 2 (t % 4) and 2 (t % 4) + 1 of each.
__device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, float v[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait4(float a[4], float b[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile("" : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(b[0]), "+f"(b[1]), "+f"(b[2]), "+f"(b[3])
                 :: "memory");
}
// Wait for this thread's TMEM loads; the loaded registers pass through the
// statements below, so that no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void reg_fence8(float v[8]) {
    asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7])
                 :: "memory");
}
__device__ __forceinline__ void tmem_ld_wait(float a[8]) {
    tmem_ld_wait();
    reg_fence8(a);
}
__device__ __forceinline__ void tmem_ld_wait(float a[8], float b[8]) {
    tmem_ld_wait();
    reg_fence8(a);
    reg_fence8(b);
}
__device__ __forceinline__ void tmem_ld_wait(float a[8], float b[8], float c[8], float d[8]) {
    tmem_ld_wait();
    reg_fence8(a);
    reg_fence8(b);
    reg_fence8(c);
    reg_fence8(d);
}

// Two values rounded to nearest TF32 (11 significant bits) by Veltkamp's
// splitting, s = 8193 x, x' = s - (s - x), in packed FP32 arithmetic: the
// low 13 bits of each result are zero, so that the tensor cores' truncation
// of the operand is exact.  Equal to cvt.rna.tf32.f32 except at exact ties
// (even here, away from zero there); NaN stays NaN, +-inf becomes NaN.
__device__ __forceinline__ void to_tf32x2(float& a, float& b) {
    asm("{\n .reg .b64 x, s, t, c;\n mov.b64 x, {%0, %1};\n mov.b64 c, {%2, %2};\n"
        " fma.rn.f32x2 s, x, c, x;\n sub.rn.f32x2 t, s, x;\n sub.rn.f32x2 s, s, t;\n mov.b64 {%0, %1}, s;\n}"
        : "+f"(a), "+f"(b)
        : "f"(8192.0f));
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace dgc

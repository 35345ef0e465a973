// Persistent batched stage kernel on the tensor cores: one launch per RK
// stage walks a work list of (mesh, tile) items over many meshes of degrees
// NLO..NHI (no artificial viscosity).  Affine tiles of 32 elements run the
// tensor-core tile body of the single-mesh kernel; curved tiles run the
// CUDA-core body.  A CTA reloads the operator tables only when the degree
// of its next affine item differs from the loaded one (the work list is
// grouped by degree).  The mbarriers and the TMEM slot live in static
// shared memory, outside the per-degree layouts.  Items are claimed from an
// atomic counter reset by a memset node of the captured step graph.
#include "dg_batch.h"
#include "tc_kernels.cuh"

namespace dgc {

template <int NLO, int NHI>
constexpr size_t batch_tc_smem() {
    size_t m = 0;
#define DGC_BT_MAX(n) \
    if (n >= NLO && n <= NHI && tc_smem_bytes<n, false>() > m) m = tc_smem_bytes<n, false>();
    DGC_BT_MAX(2) DGC_BT_MAX(3) DGC_BT_MAX(4) DGC_BT_MAX(5) DGC_BT_MAX(6)
#undef DGC_BT_MAX
    return m + 1024;   // + up to 1 KB to align the layout to 1024 bytes
}

template <int NLO, int NHI>
constexpr int batch_tc_tmem_cols() {
    int c = 0;
#define DGC_BT_COLS(n) \
    if (n >= NLO && n <= NHI && TcDims<n>::TMEM_COLS > c) c = TcDims<n>::TMEM_COLS;
    DGC_BT_COLS(2) DGC_BT_COLS(3) DGC_BT_COLS(4) DGC_BT_COLS(5) DGC_BT_COLS(6)
#undef DGC_BT_COLS
    return c;
}

template <int PREC, int NLO, int NHI>
__global__ void __launch_bounds__(THREADS, 2)
    batch_stage_kernel_tc(const StageArgs<float>* args, const BatchItem* items, int nitems,
                          const unsigned char* const* ops_by_n, int* err, int* counter) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // the tile layout starts on a 1024-byte boundary (128-byte swizzled operands)
    unsigned char* smem_bt = smem_dyn + ((1024u - (tc::smem_addr(smem_dyn) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t bars[4];
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile;
    constexpr int COLS = batch_tc_tmem_cols<NLO, NHI>();
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) tc::mbar_init(&bars[b], 1);
        tc::mbar_fence_init();
    }
    if ((tid >> 5) == 0) tc::tmem_alloc(&s_tmem, COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const TcGroup grp{tid, 0u, 0u, 1u};   // one tile at a time, the whole CTA
    TcPhase ph;
    int loaded = 0;   // degree whose operators are in shared memory (0: none)
    if (tid == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    int t = s_tile;
    while (t < nitems) {
        __syncthreads();   // every thread has read s_tile
        const int claim = (tid == THREADS - 1) ? atomicAdd(counter, 1) : 0;
        const BatchItem b = items[t];
        const StageArgs<float> p = args[b.mesh];
        if (b.curved) {
            TileRange tr;
            tr.curved = true;
            tr.e0 = b.e0;
            tr.ne = b.ne;
            switch (b.N) {
#define DGC_BT_CURVED(n) \
    case n:              \
        if constexpr (n >= NLO && n <= NHI) stage_tile_call<n, float, false>(p, tr, smem_bt); \
        break;
                DGC_BT_CURVED(2) DGC_BT_CURVED(3) DGC_BT_CURVED(4) DGC_BT_CURVED(5) DGC_BT_CURVED(6)
#undef DGC_BT_CURVED
            }
            loaded = 0;   // the curved body overwrote the operator region
            if (tid == THREADS - 1) s_tile = claim;
            __syncthreads();
        } else {
            if (loaded != b.N) {
                switch (b.N) {
#define DGC_BT_OPS(n) \
    case n:           \
        if constexpr (n >= NLO && n <= NHI) load_tc_operators<n, false>(ops_by_n[n], smem_bt); \
        break;
                    DGC_BT_OPS(2) DGC_BT_OPS(3) DGC_BT_OPS(4) DGC_BT_OPS(5) DGC_BT_OPS(6)
#undef DGC_BT_OPS
                }
                __syncthreads();
                loaded = b.N;
            }
            // no prefetch across items: the next item may belong to another mesh
            switch (b.N) {
#define DGC_BT_TILE(n)                                                                                      \
    case n:                                                                                                 \
        if constexpr (n >= NLO && n <= NHI)                                                                 \
            stage_tile_tc<n, false, PREC>(p, b.e0, b.ne, smem_bt, tmem, ph, err, false, claim, &s_tile, 0, 0, \
                                          bars, grp);                                                       \
        break;
                DGC_BT_TILE(2) DGC_BT_TILE(3) DGC_BT_TILE(4) DGC_BT_TILE(5) DGC_BT_TILE(6)
#undef DGC_BT_TILE
            }
        }
        t = s_tile;
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((tid >> 5) == 0) tc::tmem_free(tmem, COLS);
}

// Grid (SMs x resident CTAs) of one instantiation; 0 if it cannot run.
template <int PREC, int NLO, int NHI>
int batch_tc_grid_t(int device) {
    auto kern = batch_stage_kernel_tc<PREC, NLO, NHI>;
    const int sm = (int)batch_tc_smem<NLO, NHI>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int occ = resident_ctas((const void*)kern, THREADS, sm), nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    const int by_tmem = 512 / batch_tc_tmem_cols<NLO, NHI>();
    occ = occ < by_tmem ? occ : by_tmem;
    return occ < 1 ? 0 : nsm * occ;
}

int batch_tc_grid(int device, int prec, bool deg6) {
    if (prec == PREC_TF32) return deg6 ? batch_tc_grid_t<PREC_TF32, 6, 6>(device) : batch_tc_grid_t<PREC_TF32, 2, 5>(device);
    return deg6 ? batch_tc_grid_t<PREC_BF16X3, 6, 6>(device) : batch_tc_grid_t<PREC_BF16X3, 2, 5>(device);
}

int launch_batch_stage_tc(int prec, bool deg6, const void* args, const BatchItem* items, int nitems,
                          const unsigned char* const* ops_by_n, int* err, int* counter, int grid, cudaStream_t st) {
    if (nitems <= 0) return 0;
    if (grid <= 0) return (int)cudaErrorInvalidConfiguration;
    const StageArgs<float>* a = (const StageArgs<float>*)args;
    if (prec == PREC_TF32) {
        if (deg6)
            batch_stage_kernel_tc<PREC_TF32, 6, 6><<<grid, THREADS, batch_tc_smem<6, 6>(), st>>>(a, items, nitems,
                                                                                                ops_by_n, err, counter);
        else
            batch_stage_kernel_tc<PREC_TF32, 2, 5><<<grid, THREADS, batch_tc_smem<2, 5>(), st>>>(a, items, nitems,
                                                                                                ops_by_n, err, counter);
    } else {
        if (deg6)
            batch_stage_kernel_tc<PREC_BF16X3, 6, 6><<<grid, THREADS, batch_tc_smem<6, 6>(), st>>>(
                a, items, nitems, ops_by_n, err, counter);
        else
            batch_stage_kernel_tc<PREC_BF16X3, 2, 5><<<grid, THREADS, batch_tc_smem<2, 5>(), st>>>(
                a, items, nitems, ops_by_n, err, counter);
    }
    return (int)cudaGetLastError();
}

}  // namespace dgc

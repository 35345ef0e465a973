// Persistent batched stage kernel: one launch per RK stage walks a work list
// of (mesh, tile) items over many meshes of any degree 2..6, each tile
// running the same fused stage body as the single-mesh kernel (each mesh at
// its own tile size).  Items are claimed from an atomic counter (reset by a
// memset node in the captured step graph), largest tiles first.
#include "kernels.cuh"
#include "dg_batch.h"

namespace dgc {

template <typename Real>
__global__ void __launch_bounds__(THREADS) batch_stage_kernel(const StageArgs<Real>* args, const BatchItem* items,
                                                              int nitems, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int w;
    while (true) {
        if (threadIdx.x == 0) w = atomicAdd(counter, 1);
        __syncthreads();
        const int it = w;
        if (it >= nitems) break;
        const BatchItem b = items[it];
        const StageArgs<Real> p = args[b.mesh];
        TileRange t;
        t.e0 = b.e0;
        t.ne = b.ne;
        t.curved = b.curved != 0;
        switch (b.N) {
            case 2: stage_tile<2, Real, false>(p, t, smem_raw); break;
            case 3: stage_tile<3, Real, false>(p, t, smem_raw); break;
            case 4: stage_tile<4, Real, false>(p, t, smem_raw); break;
            case 5: stage_tile<5, Real, false>(p, t, smem_raw); break;
            case 6: stage_tile<6, Real, false>(p, t, smem_raw); break;
        }
        __syncthreads();
    }
}

// Shared memory of a launch: the largest stage layout among the degrees
// present, each at the tile size its meshes use (e_by_n[N], 0 = absent).
template <typename Real>
size_t batch_smem_bytes(const int* e_by_n) {
    size_t m = 0;
#define DGC_BS(n) \
    if (e_by_n[n] > 0 && Tile<n, Real>::smem_stage(false, e_by_n[n]) > m) m = Tile<n, Real>::smem_stage(false, e_by_n[n]);
    DGC_BS(2) DGC_BS(3) DGC_BS(4) DGC_BS(5) DGC_BS(6)
#undef DGC_BS
    return m;
}

int batch_tile_e(int N, int rsize) {
    switch (N) {
        case 2: return rsize == 8 ? Tile<2, double>::E : Tile<2, float>::E;
        case 3: return rsize == 8 ? Tile<3, double>::E : Tile<3, float>::E;
        case 4: return rsize == 8 ? Tile<4, double>::E : Tile<4, float>::E;
        case 5: return rsize == 8 ? Tile<5, double>::E : Tile<5, float>::E;
        case 6: return rsize == 8 ? Tile<6, double>::E : Tile<6, float>::E;
    }
    return 0;
}

template <typename Real>
int batch_grid(int device, int ctas_per_sm, size_t sm) {
    if (sm + sizeof(int) > SMEM_CTA_MAX) return -1;
    if (allow_max_dynamic_smem((const void*)batch_stage_kernel<Real>) != cudaSuccess) return -1;
    int occ = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_stage_kernel<Real>, THREADS, sm) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    if (occ < 1) return -1;
    const int per = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    return nsm * per;
}

template <typename Real>
int launch_batch_stage(const void* args, const BatchItem* items, int nitems, int* counter, int grid, size_t sm,
                       cudaStream_t st) {
    batch_stage_kernel<Real><<<grid, THREADS, sm, st>>>((const StageArgs<Real>*)args, items, nitems, counter);
    return (int)cudaGetLastError();
}

template size_t batch_smem_bytes<float>(const int*);
template size_t batch_smem_bytes<double>(const int*);
template int batch_grid<float>(int, int, size_t);
template int batch_grid<double>(int, int, size_t);
template int launch_batch_stage<float>(const void*, const BatchItem*, int, int*, int, size_t, cudaStream_t);
template int launch_batch_stage<double>(const void*, const BatchItem*, int, int*, int, size_t, cudaStream_t);

}  // namespace dgc

// Work list of the persistent batched stage kernel.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace dgc {

struct BatchItem {
    int mesh;        // index into the per-stage argument array
    int N;           // degree of that mesh
    long long e0;    // first element (device order)
    int ne;          // elements in the tile
    int curved;      // tile of curved elements
};

int batch_tile_e(int N, int rsize);
template <typename Real> size_t batch_smem_bytes(const int* e_by_n);
template <typename Real> int batch_grid(int device, int ctas_per_sm, size_t smem);
template <typename Real>
int launch_batch_stage(const void* args, const BatchItem* items, int nitems, int* counter, int grid, size_t smem,
                       cudaStream_t st);

// Tensor-core batched stage (kernels_batch_tc.cu): prec 1 = TF32, 2 = BF16x3;
// deg6 selects the instantiation for degree-6 items (the others take 2..5).
int batch_tc_grid(int device, int prec, bool deg6);
int launch_batch_stage_tc(int prec, bool deg6, const void* args, const BatchItem* items, int nitems,
                          const unsigned char* const* ops_by_n, int* err, int* counter, int grid, cudaStream_t st);

}  // namespace dgc

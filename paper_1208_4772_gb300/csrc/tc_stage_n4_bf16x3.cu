// Degree-4 tensor-core stage kernels with split-BF16 products, every tile-pipeline
// configuration that fits (explicit instantiations; one unit per degree and
// precision so that the units compile in parallel).
#include "tc_kernels.cuh"

namespace dgc {
template int launch_stage_tc_prec<4, 2>(const StageArgs<float>&, int, const unsigned char*, int*, cudaStream_t, int);
template int prepare_tc_prec<4, 2>();
}  // namespace dgc

// Degree-6 tensor-core stage kernels with TF32 products, every tile-pipeline
// configuration that fits (explicit instantiations; one unit per degree and
// precision so that the units compile in parallel).
#include "tc_kernels.cuh"

namespace dgc {
template int launch_stage_tc_prec<6, 1>(const StageArgs<float>&, int, const unsigned char*, int*, cudaStream_t, int);
template int prepare_tc_prec<6, 1>();
template int tc_configs_n<6>(int, int*);
#ifdef DGC_PHASE_CLOCKS
template int tc_phase_cycles<6>(unsigned long long*, bool);
#endif
}  // namespace dgc

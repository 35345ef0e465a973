// Degree-2 instantiations of the CUDA-core and tensor-core kernels.
#include "kernels.cuh"
#include "tc_kernels.cuh"
#include "tc_grad.cuh"

namespace dgc {
template int launch_stage<2, float>(const StageArgs<float>&, int, cudaStream_t);
template int launch_stage<2, double>(const StageArgs<double>&, int, cudaStream_t);
template int launch_sensor<2, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_sensor<2, double>(const StageArgs<double>&, double*, cudaStream_t);
template int launch_grad<2, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_grad<2, double>(const StageArgs<double>&, double*, cudaStream_t);
}  // namespace dgc
namespace dgc {
template int prepare_kernels<2, float>();
template int prepare_kernels<2, double>();
template int tile_e_default<2, float>();
template int tile_e_default<2, double>();
template bool tile_e_fits<2, float>(int, int);
template bool tile_e_fits<2, double>(int, int);
}  // namespace dgc
namespace dgc {
template std::vector<uint8_t> pack_ops_tc<2>(const RefOps&, int);
}  // namespace dgc
namespace dgc {
template int launch_grad_tc<2>(const StageArgs<float>&, float*, int, const unsigned char*, int*, cudaStream_t);
template int prepare_grad_tc<2>();
}  // namespace dgc

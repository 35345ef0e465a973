// Degree-3 instantiations of the CUDA-core and tensor-core kernels.
#include "kernels.cuh"
#include "tc_kernels.cuh"
#include "tc_grad.cuh"

namespace dgc {
template int launch_stage<3, float>(const StageArgs<float>&, int, cudaStream_t);
template int launch_stage<3, double>(const StageArgs<double>&, int, cudaStream_t);
template int launch_sensor<3, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_sensor<3, double>(const StageArgs<double>&, double*, cudaStream_t);
template int launch_grad<3, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_grad<3, double>(const StageArgs<double>&, double*, cudaStream_t);
}  // namespace dgc
namespace dgc {
template int prepare_kernels<3, float>();
template int prepare_kernels<3, double>();
template int tile_e_default<3, float>();
template int tile_e_default<3, double>();
template bool tile_e_fits<3, float>(int, int);
template bool tile_e_fits<3, double>(int, int);
}  // namespace dgc
namespace dgc {
template std::vector<uint8_t> pack_ops_tc<3>(const RefOps&, int);
}  // namespace dgc
namespace dgc {
template int launch_grad_tc<3>(const StageArgs<float>&, float*, int, const unsigned char*, int*, cudaStream_t);
template int prepare_grad_tc<3>();
}  // namespace dgc

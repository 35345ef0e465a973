// Degree-2 instantiations of the CUDA-core stage, sensor and gradient kernels.
#include "kernels.cuh"

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
}  // namespace dgc

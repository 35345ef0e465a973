// Degree-3 instantiations of the CUDA-core stage, sensor and gradient kernels.
#include "kernels.cuh"

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
}  // namespace dgc

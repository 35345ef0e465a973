// Degree-5 instantiations of the CUDA-core stage, sensor and gradient kernels.
#include "kernels.cuh"

namespace dgc {
template int launch_stage<5, float>(const StageArgs<float>&, int, cudaStream_t);
template int launch_stage<5, double>(const StageArgs<double>&, int, cudaStream_t);
template int launch_sensor<5, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_sensor<5, double>(const StageArgs<double>&, double*, cudaStream_t);
template int launch_grad<5, float>(const StageArgs<float>&, float*, cudaStream_t);
template int launch_grad<5, double>(const StageArgs<double>&, double*, cudaStream_t);
}  // namespace dgc
namespace dgc {
template int prepare_kernels<5, float>();
template int prepare_kernels<5, double>();
}  // namespace dgc

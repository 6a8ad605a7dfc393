// FP32 instantiations of the z tridiagonal kernels (templates in z_impl.cuh).
#include "z_impl.cuh"

namespace cales {

template size_t zsolve_w_smem<float>(int, int);
template size_t zsolve_reg_smem<float>(int, int, int);
template size_t zsolve_smem<float>(int, int, int);
template cudaError_t launch_zsolve<float>(const ZArgs<float>&, cudaStream_t);

}  // namespace cales

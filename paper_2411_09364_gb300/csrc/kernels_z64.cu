// FP64 instantiations of the z tridiagonal kernels (templates in z_impl.cuh).
#include "z_impl.cuh"

namespace cales {

template size_t zsolve_w_smem<double>(int, int);
template size_t zsolve_reg_smem<double>(int, int, int);
template size_t zsolve_smem<double>(int, int, int);
template cudaError_t launch_zsolve<double>(const ZArgs<double>&, cudaStream_t);

}  // namespace cales

// FP64 residual of the staggered 7-point operator (Eq. 16 on the MAC grid):
//   r = (f - fshift) - (c0 u + c1 L u)
// with Poisson (c0, c1) = (0, 1) and Helmholtz (1, -alpha).  Boundary ghosts
// are applied in-kernel (periodic wrap, Neumann mirror, Dirichlet
// antisymmetric mirror, zero at a Dirichlet node).  Neighbour reuse in x, y
// and z is left to L1/L2: each thread reads its point and six neighbours.
#include "kernels.cuh"

namespace cales {

__device__ __forceinline__ double ghost(int kind, double v0) {
    return kind == KIND_N ? v0 : -v0;   // N mirror, D antisymmetric
}

__global__ void __launch_bounds__(256) k_residual(ResidArgs a) {
    const long nx = a.nx, ny = a.ny, nz = a.nz;
    const long plane = nx * ny;
    const long N = plane * nz;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane;
        const long rem = idx - k * plane;
        const long j = rem / nx;
        const long i = rem - j * nx;
        const double* __restrict__ u = a.u;
        const double uc = u[idx];
        double uw, ue, us, un, ud, uu;
        if (i > 0) uw = u[idx - 1];
        else uw = (a.bcx == KIND_P) ? u[idx + nx - 1] : ghost(a.bcx, uc);
        if (i < nx - 1) ue = u[idx + 1];
        else ue = (a.bcx == KIND_P) ? u[idx - (nx - 1)] : ghost(a.bcx, uc);
        if (j > 0) us = u[idx - nx];
        else us = (a.bcy == KIND_P) ? u[idx + (ny - 1) * nx] : ghost(a.bcy, uc);
        if (j < ny - 1) un = u[idx + nx];
        else un = (a.bcy == KIND_P) ? u[idx - (ny - 1) * nx] : ghost(a.bcy, uc);
        if (k > 0) ud = u[idx - plane];
        else ud = a.zlo == ZBC_N ? uc : (a.zlo == ZBC_D ? -uc : 0.0);
        if (k < nz - 1) uu = u[idx + plane];
        else uu = a.zhi == ZBC_N ? uc : (a.zhi == ZBC_D ? -uc : 0.0);
        const double lu = (ue + uw - 2.0 * uc) * a.idx2 + (un + us - 2.0 * uc) * a.idy2
                        + a.zc[k] * (uu - uc) - a.za[k] * (uc - ud);
        const double r = (a.f[idx] - a.fshift) - (a.c0 * uc + a.c1 * lu);
        if (a.r_is_double) reinterpret_cast<double*>(a.r)[idx] = r;
        else reinterpret_cast<float*>(a.r)[idx] = float(r);
    }
}

cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st) {
    const long N = (long)a.nx * a.ny * a.nz;
    long blocks = (N + 255) / 256;
    if (blocks > 152L * 64) blocks = 152L * 64;
    k_residual<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cales

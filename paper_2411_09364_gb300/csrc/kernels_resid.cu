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

// ---------------------------------------------------------------------------
// Double-float residual (FP32 pipes).  u is stored as (hi, lo) float pairs;
// each difference and product is carried in double-float, and f is split
// into a pair with integer operations, so no FP64 instruction runs per point.  One CTA row of
// the grid per z-plane, so the dzf weight of the gauge sum is uniform in it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff ldu(const float2* __restrict__ u, long i) {
    const float2 v = u[i];
    return ff{v.x, v.y};
}

__device__ __forceinline__ ff ghost_ff(int kind, ff c) { return kind == KIND_N ? c : ff_neg(c); }

__global__ void __launch_bounds__(256) k_residual_ff(ResidFFArgs a) {
    const long nx = a.nx, ny = a.ny;
    const long plane = nx * ny;
    const int k = blockIdx.y;
    const long kbase = (long)k * plane;
    const float2* __restrict__ u = a.u;
    const ff za = ff_from_double(a.c1 * a.za[k]);
    const ff zc = ff_from_double(a.c1 * a.zc[k]);
    const ff cx{a.cxh, a.cxl}, cy{a.cyh, a.cyl};
    const ff csh = a.cshift ? ff_from_double(a.cshift[0]) : ff{0.f, 0.f};
    const ff zero{0.f, 0.f};
    ff sum{0.f, 0.f};
    for (long rem = (long)blockIdx.x * blockDim.x + threadIdx.x; rem < plane; rem += (long)gridDim.x * blockDim.x) {
        const long j = rem / nx, i = rem - j * nx;
        const long idx = kbase + rem;
        const ff pc = ldu(u, idx);
        const ff pw = i > 0 ? ldu(u, idx - 1) : (a.bcx == KIND_P ? ldu(u, idx + nx - 1) : ghost_ff(a.bcx, pc));
        const ff pe = i < nx - 1 ? ldu(u, idx + 1) : (a.bcx == KIND_P ? ldu(u, idx - (nx - 1)) : ghost_ff(a.bcx, pc));
        const ff ps = j > 0 ? ldu(u, idx - nx) : (a.bcy == KIND_P ? ldu(u, idx + (ny - 1) * nx) : ghost_ff(a.bcy, pc));
        const ff pn = j < ny - 1 ? ldu(u, idx + nx) : (a.bcy == KIND_P ? ldu(u, idx - (ny - 1) * nx) : ghost_ff(a.bcy, pc));
        const ff pd = k > 0 ? ldu(u, idx - plane) : (a.zlo == ZBC_N ? pc : (a.zlo == ZBC_D ? ff_neg(pc) : zero));
        const ff pu = k < a.nz - 1 ? ldu(u, idx + plane) : (a.zhi == ZBC_N ? pc : (a.zhi == ZBC_D ? ff_neg(pc) : zero));
        const ff lx = ff_add(ff_sub(pe, pc), ff_sub(pw, pc));
        const ff ly = ff_add(ff_sub(pn, pc), ff_sub(ps, pc));
        ff t = ff_mul(cx, lx);
        t = ff_add(t, ff_mul(cy, ly));
        t = ff_add(t, ff_mul(zc, ff_sub(pu, pc)));
        t = ff_add(t, ff_mul(za, ff_sub(pd, pc)));
        if (a.c0h != 0.f) t = ff_add(t, pc);
        t = ff_add(t, csh);
        const ff r = ff_sub(split_double_int(a.f[idx]), t);
        a.r[idx] = __fadd_rn(r.hi, r.lo);
        if (a.gacc) sum = ff_add(sum, pc);
    }
    if (a.gacc) {
        double v = ff_to_double(sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double red[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            atomicAdd(a.gacc, s * a.dzf[k]);
        }
    }
}

cudaError_t launch_residual_ff(const ResidFFArgs& a, cudaStream_t st) {
    const long plane = (long)a.nx * a.ny;
    long bx = (plane + 255) / 256;
    if (bx > 64) bx = 64;
    dim3 grid((unsigned)bx, (unsigned)a.nz);
    k_residual_ff<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cales

// Kernels around the pressure projection of the fractional-step method
// (Sec. 2.2, Eqs. 12-13) and of a learned closure trained through it.
//
// Staggered layout on a grid periodic in x and y with walls in z: u on
// x-faces (i+1/2), v on y-faces (j+1/2), both [nz][ny][nx]; w on z-faces,
// [nz+1][ny][nx] with the impermeable wall values w[0] = w[nz] = 0; scalars
// at cell centres [nz][ny][nx].
//   div : d = (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy + (w_{k+1} - w_k)/dzf_k
//   grad: gx = (phi_{i+1} - phi_i)/dx, gy likewise, gz_k = (phi_k - phi_{k-1})/dzc_k
//         on interior z-faces, 0 on the walls.
// The transposes (div^T, grad^T) are written out directly, so gradients of a
// loss flow back through the projection u - grad S div u exactly.
//
// Learned closure: a 27-tap stencil per velocity component,
//   out_c = a u_c + sum_t theta[c][t] u_c(x + o_t) + beta tanh(u_c),
// periodic in x, y, zero outside the component's planes in z, wall faces of w
// held at zero; its weight gradient is the 27 x 3 correlation of the output
// gradient with the shifted inputs.
#include "kernels.cuh"

namespace cales {



__device__ __forceinline__ long wrapx(long i, long n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One thread per (i, j) of plane blockIdx.z (blocks of 32 x 8): no index division.
template <typename T>
__global__ void __launch_bounds__(256) k_divergence(GridArgs<T> g, const T* __restrict__ u,
                                                   const T* __restrict__ v, const T* __restrict__ w,
                                                   T* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z, nx = g.nx, ny = g.ny;
    if (i >= nx || j >= ny) return;
    const size_t plane = (size_t)nx * ny, row = (size_t)k * plane + (size_t)j * nx;
    const size_t idx = row + i;
    const T du = (u[idx] - u[row + (i > 0 ? i - 1 : nx - 1)]) * g.idx;
    const T dv = (v[idx] - v[(size_t)k * plane + (size_t)(j > 0 ? j - 1 : ny - 1) * nx + i]) * g.idy;
    const T dw = (w[idx + plane] - w[idx]) * g.idzf[k];
    d[idx] = du + dv + dw;
}

// gx, gy, gz = sub ? (vin - grad phi) : grad phi; plane blockIdx.z = 0..nz (z-faces)
template <typename T>
__global__ void __launch_bounds__(256) k_gradient(GridArgs<T> g, const T* __restrict__ phi,
                                                 const T* __restrict__ uin, const T* __restrict__ vin,
                                                 const T* __restrict__ win, T* __restrict__ gx,
                                                 T* __restrict__ gy, T* __restrict__ gz, int sub) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z, nx = g.nx, ny = g.ny, nz = g.nz;
    if (i >= nx || j >= ny) return;
    const size_t plane = (size_t)nx * ny, row = (size_t)k * plane + (size_t)j * nx;
    const size_t idx = row + i;
    T z = T(0);
    if (k > 0 && k < nz) z = (phi[idx] - phi[idx - plane]) * g.idzc[k];
    gz[idx] = sub ? win[idx] - z : z;
    if (k < nz) {
        const T c = phi[idx];
        const T x = (phi[row + (i + 1 < nx ? i + 1 : 0)] - c) * g.idx;
        const T y = (phi[(size_t)k * plane + (size_t)(j + 1 < ny ? j + 1 : 0) * nx + i] - c) * g.idy;
        gx[idx] = sub ? uin[idx] - x : x;
        gy[idx] = sub ? vin[idx] - y : y;
    }
}

// (u, v, w) = div^T d, or (uin, vin, win) - div^T d when uin != NULL
template <typename T>
__global__ void k_divergence_T(GridArgs<T> g, const T* __restrict__ d, const T* __restrict__ uin,
                               const T* __restrict__ vin, const T* __restrict__ win, T* __restrict__ u,
                               T* __restrict__ v, T* __restrict__ w) {
    const bool sub = uin != nullptr;
    const long nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny, N = plane * (nz + 1);
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane, rem = idx - k * plane, j = rem / nx, i = rem - j * nx;
        T wz = T(0);
        if (k > 0 && k < nz) wz = d[idx - plane] * g.idzf[k - 1] - d[idx] * g.idzf[k];
        w[idx] = sub ? win[idx] - wz : wz;
        if (k < nz) {
            const T c = d[idx];
            const T ux = (c - d[k * plane + j * nx + wrapx(i + 1, nx)]) * g.idx;
            const T vy = (c - d[k * plane + wrapx(j + 1, ny) * nx + i]) * g.idy;
            u[idx] = sub ? uin[idx] - ux : ux;
            v[idx] = sub ? vin[idx] - vy : vy;
        }
    }
}

// phi = grad^T (gx, gy, gz)
template <typename T>
__global__ void k_gradient_T(GridArgs<T> g, const T* __restrict__ gx, const T* __restrict__ gy,
                             const T* __restrict__ gz, T* __restrict__ phi) {
    const long nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny, N = plane * nz;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane, rem = idx - k * plane, j = rem / nx, i = rem - j * nx;
        T out = (gx[k * plane + j * nx + wrapx(i - 1, nx)] - gx[idx]) * g.idx +
                (gy[k * plane + wrapx(j - 1, ny) * nx + i] - gy[idx]) * g.idy;
        if (k > 0) out += gz[idx] * g.idzc[k];              // face k (bottom of cell k)
        if (k < nz - 1) out -= gz[idx + plane] * g.idzc[k + 1];  // face k+1
        phi[idx] = out;
    }
}

// 27-tap stencil closure of one component (blockIdx.y = component).


__global__ void k_stencil27(StencilArgs s) {
    const int comp = blockIdx.y;
    const long nx = s.nx, ny = s.ny, nzc = s.nz + (comp == 2 ? 1 : 0), plane = nx * ny, N = plane * nzc;
    const float* __restrict__ u = s.in[comp];
    float* __restrict__ o = s.out[comp];
    __shared__ float th[27];
    if (threadIdx.x < 27) th[threadIdx.x] = s.theta[comp * 27 + threadIdx.x];
    __syncthreads();
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane, rem = idx - k * plane, j = rem / nx, i = rem - j * nx;
        if (comp == 2 && (k == 0 || k == nzc - 1)) { o[idx] = 0.f; continue; }
        float acc = 0.f;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const long kk = k + dz;
            if (kk < 0 || kk >= nzc) continue;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const long jj = wrapx(j + dy, ny);
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const long ii = wrapx(i + dx, nx);
                    acc = fmaf(th[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)], u[kk * plane + jj * nx + ii], acc);
                }
            }
        }
        const float uc = u[idx];
        o[idx] = s.a * uc + acc + (s.beta != 0.f ? s.beta * tanhf(uc) : 0.f);
    }
}

// gtheta[c][t] += sum_x g_c(x) u_c(x + o_t)   (g at the w walls is ignored)


__global__ void __launch_bounds__(256) k_stencil27_wgrad(WGradArgs s) {
    const int comp = blockIdx.y;
    const long nx = s.nx, ny = s.ny, nzc = s.nz + (comp == 2 ? 1 : 0), plane = nx * ny, N = plane * nzc;
    const float* __restrict__ u = s.in[comp];
    const float* __restrict__ gg = s.g[comp];
    float acc[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) acc[t] = 0.f;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane, rem = idx - k * plane, j = rem / nx, i = rem - j * nx;
        if (comp == 2 && (k == 0 || k == nzc - 1)) continue;
        const float gv = gg[idx];
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const long kk = k + dz;
            const bool in = kk >= 0 && kk < nzc;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const long jj = wrapx(j + dy, ny);
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const long ii = wrapx(i + dx, nx);
                    const float uv = in ? u[kk * plane + jj * nx + ii] : 0.f;
                    acc[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = fmaf(gv, uv, acc[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]);
                }
            }
        }
    }
    __shared__ double red[8][27];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        double v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 27) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        atomicAdd(&s.gtheta[comp * 27 + threadIdx.x], v);
    }
}

// e = pred - target; grad = 2 e / npts; loss_acc += sum e^2 (FP64)


__global__ void __launch_bounds__(256) k_sqerr(SqErrArgs s) {
    const int comp = blockIdx.y;
    const long N = s.n[comp];
    double acc = 0.0;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const float e = s.pred[comp][idx] - s.target[comp][idx];
        if (s.grad[comp]) s.grad[comp][idx] = s.scale * e;
        acc += (double)e * (double)e;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        atomicAdd(s.loss, v);
    }
}

// Adam step on n parameters (gradient given in FP64, scaled by gscale).
__global__ void k_adam(float* theta, const double* grad, float* m, float* v, int n, float lr, float b1, float b2,
                       float eps, int t, float gscale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = (float)grad[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
static unsigned grid_for(long n) {
    long b = (n + 255) / 256;
    if (b > 152L * 32) b = 152L * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t launch_divergence(const GridArgs<T>& g, const T* u, const T* v, const T* w, T* d, cudaStream_t st) {
    if (g.nz > 65535 || g.ny > 8 * 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
    k_divergence<T><<<grid, dim3(32, 8), 0, st>>>(g, u, v, w, d);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gradient(const GridArgs<T>& g, const T* phi, const T* uin, const T* vin, const T* win, T* gx,
                            T* gy, T* gz, int sub, cudaStream_t st) {
    if (g.nz + 1 > 65535 || g.ny > 8 * 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)(g.nz + 1));
    k_gradient<T><<<grid, dim3(32, 8), 0, st>>>(g, phi, uin, vin, win, gx, gy, gz, sub);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_divergence_T(const GridArgs<T>& g, const T* d, const T* uin, const T* vin, const T* win, T* u,
                                T* v, T* w, cudaStream_t st) {
    k_divergence_T<T><<<grid_for((long)g.nx * g.ny * (g.nz + 1)), 256, 0, st>>>(g, d, uin, vin, win, u, v, w);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gradient_T(const GridArgs<T>& g, const T* gx, const T* gy, const T* gz, T* phi, cudaStream_t st) {
    k_gradient_T<T><<<grid_for((long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, gx, gy, gz, phi);
    return cudaGetLastError();
}
cudaError_t launch_stencil27(const StencilArgs& s, cudaStream_t st) {
    dim3 grid(grid_for((long)s.nx * s.ny * (s.nz + 1)) / 3 + 1, 3);
    k_stencil27<<<grid, 256, 0, st>>>(s);
    return cudaGetLastError();
}
cudaError_t launch_stencil27_wgrad(const WGradArgs& s, cudaStream_t st) {
    dim3 grid(grid_for((long)s.nx * s.ny * (s.nz + 1)) / 3 + 1, 3);
    k_stencil27_wgrad<<<grid, 256, 0, st>>>(s);
    return cudaGetLastError();
}
cudaError_t launch_sqerr(const SqErrArgs& s, cudaStream_t st) {
    dim3 grid(grid_for(s.n[2]) / 3 + 1, 3);
    k_sqerr<<<grid, 256, 0, st>>>(s);
    return cudaGetLastError();
}
cudaError_t launch_adam(float* theta, const double* grad, float* m, float* v, int n, float lr, float b1, float b2,
                        float eps, int t, float gscale, cudaStream_t st) {
    k_adam<<<(n + 127) / 128, 128, 0, st>>>(theta, grad, m, v, n, lr, b1, b2, eps, t, gscale);
    return cudaGetLastError();
}

template cudaError_t launch_divergence<float>(const GridArgs<float>&, const float*, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_divergence<double>(const GridArgs<double>&, const double*, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_gradient<float>(const GridArgs<float>&, const float*, const float*, const float*, const float*, float*, float*, float*, int, cudaStream_t);
template cudaError_t launch_gradient<double>(const GridArgs<double>&, const double*, const double*, const double*, const double*, double*, double*, double*, int, cudaStream_t);
template cudaError_t launch_divergence_T<float>(const GridArgs<float>&, const float*, const float*, const float*,
                                               const float*, float*, float*, float*, cudaStream_t);
template cudaError_t launch_divergence_T<double>(const GridArgs<double>&, const double*, const double*, const double*,
                                                const double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_gradient_T<float>(const GridArgs<float>&, const float*, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_gradient_T<double>(const GridArgs<double>&, const double*, const double*, const double*, double*, cudaStream_t);

}  // namespace cales

// Smagorinsky eddy viscosity with van Driest damping (Eq. 4, Sec. 2.1-2.2):
//   nu_t = (C_s Delta D)^2 |S|,  |S| = sqrt(2 S_ij S_ij),  D = 1 - exp(-y*/25),
// at the cell centres of a channel (x, y periodic; no-slip walls in z).  The
// diagonal strain-rate components are formed at the centre, the off-diagonal
// ones on the four surrounding cell edges and averaged to the centre.  Filter
// width Delta_k = (dx dy dzf_k)^(1/3); y* = (distance of the centre to the
// nearer wall) u_tau / nu.  No-slip ghosts: u and v mirror to minus the first
// interior value at the distances dzc[0] and dzc[nz]; w = 0 on the wall faces.
// One thread per cell; a CTA covers part of one z-plane and forms that plane's
// coefficient (C_s Delta D)^2 once, in FP64.
#include "kernels.cuh"

namespace cales {

template <typename T>
__global__ void __launch_bounds__(256) k_eddy_visc(SgsArgs<T> a) {
    const int k = blockIdx.y;
    __shared__ T coef_s;
    if (threadIdx.x == 0) {
        const double zc = a.zcen[k];
        const double d = fmin(zc, a.lz - zc);
        const double damp = 1.0 - exp(-d * a.utau / (25.0 * a.nu));
        const double c = a.cs * cbrt(a.dx * a.dy * a.dzf[k]) * damp;
        coef_s = T(c * c);
    }
    __syncthreads();
    const T coef = coef_s;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long plane = (long)nx * ny;
    const T idx = a.idx, idy = a.idy;
    const T idzf = a.idzf[k], izlo = a.idzc[k], izhi = a.idzc[k + 1];
    const T h = T(0.5), q = T(0.25);
    const T* __restrict__ u = a.u;
    const T* __restrict__ v = a.v;
    const T* __restrict__ w = a.w;
    const long kb = (long)k * plane;
    const long kd = k > 0 ? kb - plane : -1, ku = k < nz - 1 ? kb + plane : -1;   // -1: the wall ghost
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long)j * nx);
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        const int jm = j > 0 ? j - 1 : ny - 1, jp = j < ny - 1 ? j + 1 : 0;
        const long r0 = (long)j * nx, rm = (long)jm * nx, rp = (long)jp * nx;
        // u at (j-1, j, j+1) x (i-1, i) of plane k; v at (j-1, j) x (i-1, i, i+1)
        const T u_c = u[kb + r0 + i], u_w = u[kb + r0 + im];
        const T u_s = u[kb + rm + i], u_sw = u[kb + rm + im], u_n = u[kb + rp + i], u_nw = u[kb + rp + im];
        const T v_c = v[kb + r0 + i], v_s = v[kb + rm + i];
        const T v_w = v[kb + r0 + im], v_sw = v[kb + rm + im], v_e = v[kb + r0 + ip], v_se = v[kb + rm + ip];
        // z neighbours of u (i-1, i) and v (j-1, j), wall ghosts -value
        const T u_d = kd >= 0 ? u[kd + r0 + i] : -u_c, u_dw = kd >= 0 ? u[kd + r0 + im] : -u_w;
        const T u_u = ku >= 0 ? u[ku + r0 + i] : -u_c, u_uw = ku >= 0 ? u[ku + r0 + im] : -u_w;
        const T v_d = kd >= 0 ? v[kd + r0 + i] : -v_c, v_ds = kd >= 0 ? v[kd + rm + i] : -v_s;
        const T v_u = ku >= 0 ? v[ku + r0 + i] : -v_c, v_us = ku >= 0 ? v[ku + rm + i] : -v_s;
        // w on the faces k (below) and k+1 (above): (i-1, i, i+1) at j and (j-1, j+1) at i
        const long wb = kb, wa = kb + plane;
        const T wb_c = w[wb + r0 + i], wb_w = w[wb + r0 + im], wb_e = w[wb + r0 + ip];
        const T wb_s = w[wb + rm + i], wb_n = w[wb + rp + i];
        const T wa_c = w[wa + r0 + i], wa_w = w[wa + r0 + im], wa_e = w[wa + r0 + ip];
        const T wa_s = w[wa + rm + i], wa_n = w[wa + rp + i];
        // diagonal components at the centre
        const T s11 = (u_c - u_w) * idx;
        const T s22 = (v_c - v_s) * idy;
        const T s33 = (wa_c - wb_c) * idzf;
        // S12 on the four z-edges around the centre
        const T e11 = h * ((u_n - u_c) * idy + (v_e - v_c) * idx);
        const T e01 = h * ((u_nw - u_w) * idy + (v_c - v_w) * idx);
        const T e10 = h * ((u_c - u_s) * idy + (v_se - v_s) * idx);
        const T e00 = h * ((u_w - u_sw) * idy + (v_s - v_sw) * idx);
        const T s12 = q * (e00 + e10 + e01 + e11);
        // S13 on the y-edges (x-face i-1/2, i+1/2) x (z-face k, k+1)
        const T f_i_lo = h * ((u_c - u_d) * izlo + (wb_e - wb_c) * idx);
        const T f_i_hi = h * ((u_u - u_c) * izhi + (wa_e - wa_c) * idx);
        const T f_w_lo = h * ((u_w - u_dw) * izlo + (wb_c - wb_w) * idx);
        const T f_w_hi = h * ((u_uw - u_w) * izhi + (wa_c - wa_w) * idx);
        const T s13 = q * (f_i_lo + f_i_hi + f_w_lo + f_w_hi);
        // S23 on the x-edges (y-face j-1/2, j+1/2) x (z-face k, k+1)
        const T g_j_lo = h * ((v_c - v_d) * izlo + (wb_n - wb_c) * idy);
        const T g_j_hi = h * ((v_u - v_c) * izhi + (wa_n - wa_c) * idy);
        const T g_s_lo = h * ((v_s - v_ds) * izlo + (wb_c - wb_s) * idy);
        const T g_s_hi = h * ((v_us - v_s) * izhi + (wa_c - wa_s) * idy);
        const T s23 = q * (g_j_lo + g_j_hi + g_s_lo + g_s_hi);
        const T ss = s11 * s11 + s22 * s22 + s33 * s33 + T(2) * (s12 * s12 + s13 * s13 + s23 * s23);
        a.nut[kb + e] = coef * sqrt(T(2) * ss);
    }
}

template <typename T>
cudaError_t launch_eddy_viscosity(const SgsArgs<T>& a, cudaStream_t st) {
    const long plane = (long)a.nx * a.ny;
    long bx = (plane + 255) / 256;
    if (bx > 2048) bx = 2048;
    dim3 grid((unsigned)bx, (unsigned)a.nz);
    k_eddy_visc<T><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_eddy_viscosity<float>(const SgsArgs<float>&, cudaStream_t);
template cudaError_t launch_eddy_viscosity<double>(const SgsArgs<double>&, cudaStream_t);

}  // namespace cales

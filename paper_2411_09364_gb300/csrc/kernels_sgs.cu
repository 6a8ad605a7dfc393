// Smagorinsky eddy viscosity with van Driest damping (Eq. 4, Sec. 2.1-2.2):
//   nu_t = (C_s Delta D)^2 |S|,  |S| = sqrt(2 S_ij S_ij),  D = 1 - exp(-y*/25),
// at the cell centres of a channel (x, y periodic; no-slip walls in z).  The
// diagonal strain-rate components are formed at the centre, the off-diagonal
// ones on the four surrounding cell edges and averaged to the centre.  Filter
// width Delta_k = (dx dy dzf_k)^(1/3); y* = (distance of the centre to the
// nearer wall) u_tau / nu.  No-slip ghosts: u and v mirror to minus the first
// interior value at the distances dzc[0] and dzc[nz]; w = 0 on the wall faces.
//
// Two launches: the plane coefficients (C_s Delta D)^2 in FP64 (nz threads),
// then one thread per VW consecutive cells of an x-row, reading each of the
// 17 neighbouring rows of u, v, w it needs as one 16-byte vector (plus a
// scalar at either end where the stencil reaches i-1 or i+VW).  The sum of
// the four edge values of S_ij is formed from differences before scaling:
// 8 S_12 = (du/dy summed over the two x-faces) + (dv/dx over the two y-faces),
// and likewise for S_13 and S_23 with the z spacing below and above; the
// x-differences are shared by a thread's neighbouring cells.  Each CTA hints
// plane k+2 into L2, so the demand loads of a plane find it there.
#include "kernels.cuh"

namespace cales {

__global__ void k_sgs_coef(double* __restrict__ coef, const double* __restrict__ zcen,
                           const double* __restrict__ dzf, int nz, double lz, double dx, double dy,
                           double cs, double nu, double utau) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    const double d = fmin(zcen[k], lz - zcen[k]);
    const double damp = 1.0 - exp(-d * utau / (25.0 * nu));
    const double c = cs * cbrt(dx * dy * dzf[k]) * damp;
    coef[k] = c * c;
}

// x[1 .. VW] = row[i0 .. i0+VW-1]  (16-byte vector for VW > 1)
template <typename T, int VW>
__device__ __forceinline__ void sgs_load_mid(T* x, const T* __restrict__ row, int i0) {
    if constexpr (VW == 1) {
        x[1] = row[i0];
    } else if constexpr (VW == 2) {
        const double2 q = *reinterpret_cast<const double2*>(row + i0);
        x[1] = q.x; x[2] = q.y;
    } else {
        const float4 q = *reinterpret_cast<const float4*>(row + i0);
        x[1] = q.x; x[2] = q.y; x[3] = q.z; x[4] = q.w;
    }
}

// x[0] = row[i0-1], x[1 .. VW] = row[i0 ..], x[VW+1] = row[i0+VW] (periodic in x);
// the ends only where the stencil needs them
template <typename T, int VW, bool LEFT, bool RIGHT>
__device__ __forceinline__ void sgs_load_row(T* x, const T* __restrict__ row, int i0, int im, int ip) {
    sgs_load_mid<T, VW>(x, row, i0);
    if constexpr (LEFT) x[0] = row[im];
    if constexpr (RIGHT) x[VW + 1] = row[ip];
}

template <typename T, int VW>
__global__ void __launch_bounds__(256) k_eddy_visc(SgsArgs<T> a) {
    const int k = blockIdx.z;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * VW;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    if (j >= ny || i0 >= nx) return;
    const size_t plane = (size_t)nx * ny;
    const int im = i0 > 0 ? i0 - 1 : nx - 1, ip = i0 + VW < nx ? i0 + VW : 0;
    const int jm = j > 0 ? j - 1 : ny - 1, jp = j < ny - 1 ? j + 1 : 0;
    const size_t r0 = (size_t)j * nx, rs = (size_t)jm * nx, rn = (size_t)jp * nx;
    const T* __restrict__ u = a.u + (size_t)k * plane;
    const T* __restrict__ v = a.v + (size_t)k * plane;
    const T* __restrict__ wb = a.w + (size_t)k * plane;     // face below the centre
    const T* __restrict__ wa = wb + plane;                  // face above
    constexpr int N = VW + 2;
    // u: centre row j and rows j-1, j+1 (i-1 .. i); z neighbours of row j
    T uc[N], us[N], un[N], ud[N], uu[N];
    // v: rows j and j-1 (i-1 .. i+1); their z neighbours (i only)
    T vc[N], vs[N], vd[N], vds[N], vu[N], vus[N];
    // w below / above: row j (i-1 .. i+1) and rows j-1, j+1 (i only)
    T bc[N], bs[N], bn[N], ac[N], as[N], an[N];
    sgs_load_row<T, VW, true, false>(uc, u + r0, i0, im, ip);
    sgs_load_row<T, VW, true, false>(us, u + rs, i0, im, ip);
    sgs_load_row<T, VW, true, false>(un, u + rn, i0, im, ip);
    sgs_load_row<T, VW, true, true>(vc, v + r0, i0, im, ip);
    sgs_load_row<T, VW, true, true>(vs, v + rs, i0, im, ip);
    sgs_load_row<T, VW, true, true>(bc, wb + r0, i0, im, ip);
    sgs_load_row<T, VW, false, false>(bs, wb + rs, i0, im, ip);
    sgs_load_row<T, VW, false, false>(bn, wb + rn, i0, im, ip);
    sgs_load_row<T, VW, true, true>(ac, wa + r0, i0, im, ip);
    sgs_load_row<T, VW, false, false>(as, wa + rs, i0, im, ip);
    sgs_load_row<T, VW, false, false>(an, wa + rn, i0, im, ip);
    if (k > 0) {
        sgs_load_row<T, VW, true, false>(ud, u - plane + r0, i0, im, ip);
        sgs_load_row<T, VW, false, false>(vd, v - plane + r0, i0, im, ip);
        sgs_load_row<T, VW, false, false>(vds, v - plane + rs, i0, im, ip);
    } else {                                                // no-slip ghost below the bottom wall
#pragma unroll
        for (int m = 0; m <= VW; ++m) { ud[m] = -uc[m]; vd[m] = -vc[m]; vds[m] = -vs[m]; }
    }
    if (k < nz - 1) {
        sgs_load_row<T, VW, true, false>(uu, u + plane + r0, i0, im, ip);
        sgs_load_row<T, VW, false, false>(vu, v + plane + r0, i0, im, ip);
        sgs_load_row<T, VW, false, false>(vus, v + plane + rs, i0, im, ip);
    } else {                                                // ghost above the top wall
#pragma unroll
        for (int m = 0; m <= VW; ++m) { uu[m] = -uc[m]; vu[m] = -vc[m]; vus[m] = -vs[m]; }
    }
    // the next CTAs of this column of the grid work on plane k+1, whose rows
    // are all in L2 by now; start plane k+2 (u, v and the face above it) on
    // its way from HBM
    if (k + 2 < nz) {
        prefetch_l2(u + 2 * plane + r0 + i0);
        prefetch_l2(v + 2 * plane + r0 + i0);
        prefetch_l2(wa + 2 * plane + r0 + i0);
    }
    const T coef = T(a.coef[k]);
    const T idx = a.idx, idy = a.idy, idzf = a.idzf[k], izlo = a.idzc[k], izhi = a.idzc[k + 1];
    // differences and sums shared by the x-neighbouring cells of this thread
    T dns[N], dlo[N], dhi[N], sv[N], sw[N];
#pragma unroll
    for (int m = 0; m <= VW; ++m) { dns[m] = un[m] - us[m]; dlo[m] = uc[m] - ud[m]; dhi[m] = uu[m] - uc[m]; }
#pragma unroll
    for (int m = 0; m < N; ++m) { sv[m] = vc[m] + vs[m]; sw[m] = bc[m] + ac[m]; }
    T out[VW];
#pragma unroll
    for (int t = 0; t < VW; ++t) {
        const int c = t + 1, w = t, e = t + 2;              // cells i, i-1, i+1
        const T s11 = (uc[c] - uc[w]) * idx;
        const T s22 = (vc[c] - vs[c]) * idy;
        const T s33 = (ac[c] - bc[c]) * idzf;
        const T a12 = (dns[c] + dns[w]) * idy + (sv[e] - sv[w]) * idx;
        const T a13 = (dlo[c] + dlo[w]) * izlo + (dhi[c] + dhi[w]) * izhi + (sw[e] - sw[w]) * idx;
        const T a23 = ((vc[c] - vd[c]) + (vs[c] - vds[c])) * izlo + ((vu[c] - vc[c]) + (vus[c] - vs[c])) * izhi +
                      ((bn[c] + an[c]) - (bs[c] + as[c])) * idy;
        // 2 S_ij S_ij = 2 (s11^2 + s22^2 + s33^2) + (a12^2 + a13^2 + a23^2) / 16
        const T ss2 = T(2) * (s11 * s11 + s22 * s22 + s33 * s33) + T(0.0625) * (a12 * a12 + a13 * a13 + a23 * a23);
        out[t] = coef * sqrt(ss2);
    }
    T* __restrict__ dst = a.nut + (size_t)k * plane + r0 + i0;
    if constexpr (VW == 1) {
        dst[0] = out[0];
    } else if constexpr (VW == 2) {
        *reinterpret_cast<double2*>(dst) = make_double2(out[0], out[1]);
    } else {
        *reinterpret_cast<float4*>(dst) = make_float4(out[0], out[1], out[2], out[3]);
    }
}

template <typename T>
cudaError_t launch_eddy_viscosity(const SgsArgs<T>& a, cudaStream_t st) {
    if (a.nz > 65535 || a.ny > 8 * 65535) return cudaErrorInvalidValue;
    k_sgs_coef<<<(a.nz + 127) / 128, 128, 0, st>>>(a.coef, a.zcen, a.dzf, a.nz, a.lz, a.dx, a.dy, a.cs, a.nu,
                                                    a.utau);
    constexpr int VV = 16 / (int)sizeof(T);
    const bool aligned = ((uintptr_t)a.u | (uintptr_t)a.v | (uintptr_t)a.w | (uintptr_t)a.nut) % 16 == 0;
    const bool vec = aligned && a.nx % VV == 0;
    const int groups = vec ? a.nx / VV : a.nx;
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((groups + 31) / 32), (unsigned)((a.ny + 7) / 8), (unsigned)a.nz);
    if (vec) k_eddy_visc<T, VV><<<grid, block, 0, st>>>(a);
    else k_eddy_visc<T, 1><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_eddy_viscosity<float>(const SgsArgs<float>&, cudaStream_t);
template cudaError_t launch_eddy_viscosity<double>(const SgsArgs<double>&, cudaStream_t);

}  // namespace cales

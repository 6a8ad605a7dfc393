// Periodic z direction of the eigenfunction expansion: one cyclic tridiagonal
// system per mode (mx, my).  For (sigma - alpha L) u = g with L = L_z + lambda,
//
//   row k:  -A_k u[k-1] + b_k u[k] - C_k u[k+1] = g_k,   b_k = sigma - alpha lambda + A_k + C_k,
//   A_k = alpha / (dzc[k] dzf[k]),  C_k = alpha / (dzc[k+1] dzf[k]),
//
// indices taken modulo nz, so row 0 couples to row nz-1 through A_0 and row
// nz-1 to row 0 through C_{nz-1}.  Row 0 is eliminated last: rows 1..nz-1
// form a tridiagonal T (couplings to u[0] moved to the right-hand side), and
//   u[k] = p[k] + u[0] (1 - q[k]),   T p = g[1..],   T q = b 1,   b = sigma - alpha lambda,
//   u[0] = (g_0 + A_0 p[n-1] + C_0 p[1]) / (b + A_0 q[n-1] + C_0 q[1]).
// (1 - q solves T (1 - q) = the couplings of rows 1 and n-1 to u[0].)  The
// pivots of T are carried in excess form d_k = C~_k + e_k, e_k = b + A_k e_{k-1}
// / d_{k-1} (+ C_k on the last row), q is a positive solve of a positive
// right-hand side and the denominator of u[0] a sum of positive terms, so no
// step cancels even for the near-singular low Poisson modes (a
// Sherman-Morrison form of the same solve loses most FP32 digits there).
// Mode (0, 0) of a singular Poisson problem is projected (dzf-weighted mean
// of g removed), its last unknown pinned to zero (the wrap couplings to it
// drop out) and the result gauged to zero weighted mean.
//
// One thread per mode: consecutive threads own consecutive modes, so every
// row access of a warp is one contiguous run.  The back-substitution ratios
// and q go to two scratch fields of the plan.
#include "z_impl.cuh"

namespace cales {

template <typename T>
__global__ void __launch_bounds__(256) k_zsolve_cyclic(ZArgs<T> a, T* __restrict__ ework, T* __restrict__ zwork) {
    const long nm = (long)a.nx * a.ny;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nm) return;
    const int nz = a.nz;
    const int j = (int)(q / a.nx), i = (int)(q - (long)j * a.nx);
    T* __restrict__ x = a.data + q;
    T* __restrict__ ev = ework + q;
    T* __restrict__ zv = zwork + q;
    const T al = a.alpha, sc = a.scale;
    const T base = a.sigma - al * (a.lamy[j] + a.lamx[i]);
    const T* __restrict__ za = a.za;
    const T* __restrict__ zc = a.zc;

    // right-hand side of row k: scale * data, divided by dzf[k] for the
    // adjoint (S^T = D S D^-1, D = diag(dzf)); the result is then times dzf[k]
    const bool adj = a.adjoint != 0;
    auto rhs = [&](int k) -> T {
        const T v = sc * x[(long)k * nm];
        return adj ? T(double(v) / a.dzf[k]) : v;
    };
    if (a.singular && q == 0) {
        double sum = 0.0, sw = 0.0;
        for (int k = 0; k < nz; ++k) {
            sum += a.dzf[k] * double(rhs(k));
            sw += a.dzf[k];
        }
        const T gmean = T(sum / sw);
        if (a.cacc) a.cacc[0] += (sum / sw) * a.cacc_scale;    // consistency constant (refinement)
        // rows 0..nz-2 with u[nz-1] = 0
        T einv = T(0), d = T(0);
        for (int k = 0; k < nz - 1; ++k) {
            const T A = al * za[k], C = al * zc[k];
            const bool last = k == nz - 2;
            const T e = base + (k == 0 ? A : A * einv) + (last ? C : T(0));
            const T inv = rcp_<T>((last ? T(0) : C) + e);
            ev[k * nm] = last ? T(0) : C * inv;
            d = (rhs(k) - gmean + (k > 0 ? A * d : T(0))) * inv;
            x[k * nm] = d;
            einv = e * inv;
        }
        T u = T(0);
        x[(long)(nz - 1) * nm] = u;
        for (int k = nz - 2; k >= 0; --k) {
            u = x[k * nm] + ev[k * nm] * u;
            x[k * nm] = u;
        }
        sum = 0.0;
        for (int k = 0; k < nz; ++k) sum += a.dzf[k] * double(x[k * nm]);
        // gauge, and the caller's constant shift of the solution
        const T mean = T(sum / sw + (a.shift_acc ? a.shift_acc[0] * a.shift_scale : 0.0));
        for (int k = 0; k < nz; ++k) x[k * nm] -= mean;
        if (adj)
            for (int k = 0; k < nz; ++k) x[k * nm] = T(double(x[k * nm]) * a.dzf[k]);
        return;
    }

    const T g0 = rhs(0);
    T einv = T(0), dp = T(0), dq = T(0);
    for (int k = 1; k < nz; ++k) {
        const T A = al * za[k], C = al * zc[k];
        const bool last = k == nz - 1;
        const T e = base + (k == 1 ? A : A * einv) + (last ? C : T(0));
        const T inv = rcp_<T>((last ? T(0) : C) + e);
        ev[k * nm] = last ? T(0) : C * inv;
        dp = (rhs(k) + (k > 1 ? A * dp : T(0))) * inv;
        dq = (base + (k > 1 ? A * dq : T(0))) * inv;
        x[k * nm] = dp;
        zv[k * nm] = dq;
        einv = e * inv;
    }
    const T plast = dp, qlast = dq;
    T pk = dp, qk = dq;
    for (int k = nz - 2; k >= 1; --k) {
        const T r = ev[k * nm];
        pk = x[k * nm] + r * pk;
        qk = zv[k * nm] + r * qk;
        x[k * nm] = pk;
        zv[k * nm] = qk;
    }
    const T A0 = al * za[0], C0 = al * zc[0];
    const T u0 = (g0 + A0 * plast + C0 * pk) / (base + A0 * qlast + C0 * qk);
    x[0] = adj ? T(double(u0) * a.dzf[0]) : u0;
    for (int k = 1; k < nz; ++k) {
        const T v = x[k * nm] + u0 * (T(1) - zv[k * nm]);
        x[k * nm] = adj ? T(double(v) * a.dzf[k]) : v;
    }
}

template <typename T>
cudaError_t launch_zsolve_cyclic(const ZArgs<T>& a, T* ework, T* zwork, cudaStream_t st) {
    if (a.nz < 3) return cudaErrorInvalidValue;
    const long nm = (long)a.nx * a.ny;
    k_zsolve_cyclic<T><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(a, ework, zwork);
    return cudaGetLastError();
}

template cudaError_t launch_zsolve_cyclic<float>(const ZArgs<float>&, float*, float*, cudaStream_t);
template cudaError_t launch_zsolve_cyclic<double>(const ZArgs<double>&, double*, double*, cudaStream_t);

}  // namespace cales

// z direction of the eigenfunction expansion: one tridiagonal system per mode
// (mx, my), solved by Thomas elimination along the stretched direction
// (Sec. 2.2).  For (sigma - alpha L) u = g with L = L_z + lambda(mx, my):
//
//   row k:  -A_k u[k-1] + (sigma - alpha lambda + A_k + C_k + bc) u[k] - C_k u[k+1] = g_k
//   A_k = alpha / (dzc[k] dzf[k]),  C_k = alpha / (dzc[k+1] dzf[k])
//
// The pivots are carried in "excess" form d_k = C_k + e_k with
//   e_k = (sigma - alpha lambda) + A_k e_{k-1} / d_{k-1}   (+ boundary terms)
// in which every term is non-negative, so the recurrence has no cancellation
// even when the near-singular low modes meet a strongly stretched grid (plain
// d_k = b_k - a_k c_{k-1} / d_{k-1} loses the FP32 digits there).
//
// A CTA owns `tm` consecutive modes (contiguous in memory) and the whole z
// extent: the column tile is loaded once into shared memory, one thread per
// mode runs the forward sweep, and the pivots needed by the backward sweep are
// recomputed chunk by chunk from checkpoints kept every CK rows, so the only
// per-row state is the tile itself.  Mode (0,0) of a singular Poisson problem
// is projected (weighted mean of the right-hand side removed), pinned at its
// last row and gauged to zero weighted mean.
#include "kernels.cuh"

namespace cales {



template <typename T, int CK>
__global__ void __launch_bounds__(128) k_zsolve(ZArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TM = a.tm, nz = a.nz;
    const int nck = (nz + CK - 1) / CK;
    const long nmodes = (long)a.nx * a.ny;
    T* tile = reinterpret_cast<T*>(smem_raw);     // [nz][TM]
    T* ck = tile + (long)nz * TM;                 // [nck][TM]
    T* sA = ck + (long)nck * TM;                  // [nz]
    T* sC = sA + nz;                              // [nz]
    const long q0 = (long)blockIdx.x * TM;
    const int c = threadIdx.x;
    const int w = (int)min((long)TM, nmodes - q0);
    for (int k = c; k < nz; k += blockDim.x) {
        sA[k] = a.alpha * a.za[k];
        sC[k] = a.alpha * a.zc[k];
    }
    T* __restrict__ gp = a.data + q0 + c;
#pragma unroll 8
    for (int k = 0; k < nz; ++k) tile[k * TM + c] = (c < w) ? gp[(long)k * nmodes] : T(0);
    __syncthreads();

    if (c < w) {
        const long q = q0 + c;
        const int my = (int)(q / a.nx), mx = (int)(q - (long)my * a.nx);
        const bool sing0 = a.singular && q == 0;
        const T lam = a.lamx[mx] + a.lamy[my];
        const T base = a.sigma - a.alpha * lam;
        const T ebot = a.zlo == ZBC_D ? T(2) * sA[0] : (a.zlo == ZBC_DF ? sA[0] : T(0));
        const T etop = a.zhi == ZBC_D ? T(2) * sC[nz - 1] : (a.zhi == ZBC_DF ? sC[nz - 1] : T(0));
        const T sc = a.scale;
        T* col = tile + c;
        // right-hand side transform: scale, adjoint D^-1, projection of mode 0
        double gmean = 0.0;
        if (sing0) {
            double s = 0.0, sw = 0.0;
            for (int k = 0; k < nz; ++k) {
                double g = double(col[k * TM]) * double(sc);
                if (a.adjoint) g /= a.dzf[k];
                s += a.dzf[k] * g;
                sw += a.dzf[k];
            }
            gmean = s / sw;
            if (a.cacc) a.cacc[0] += gmean * a.cacc_scale;
        }
        bool bad = false;
        // forward sweep
        T e = base + ebot + (nz == 1 ? etop : T(0));
        T d = (nz > 1 ? sC[0] : T(0)) + e;
        T y;
        {
            T g = col[0] * sc;
            if (a.adjoint) g = T(double(g) / a.dzf[0]);
            if (sing0) g = T(double(g) - gmean);
            y = (sing0 && nz == 1) ? T(0) : g / d;
        }
        col[0] = y;
        ck[c] = e;
        bad |= !(d > T(0)) && !(sing0 && nz == 1);
        for (int k = 1; k < nz; ++k) {
            const T Ak = sA[k];
            e = base + Ak * e / d + (k == nz - 1 ? etop : T(0));
            d = (k < nz - 1 ? sC[k] : T(0)) + e;
            T g = col[k * TM] * sc;
            if (a.adjoint) g = T(double(g) / a.dzf[k]);
            if (sing0) g = T(double(g) - gmean);
            if (sing0 && k == nz - 1) {
                y = T(0);                     // pinned row
            } else {
                y = (g + Ak * y) / d;
                bad |= !(d > T(0));
            }
            col[k * TM] = y;
            if (k % CK == 0) ck[(k / CK) * TM + c] = e;
        }
        // backward sweep, pivots recomputed per chunk from the checkpoints
        T xn = T(0);
        for (int ch = nck - 1; ch >= 0; --ch) {
            const int k0 = ch * CK;
            const int k1 = min(k0 + CK, nz);
            T rr[CK];
            T ee = ck[ch * TM + c];
            T dd = (k0 < nz - 1 ? sC[k0] : T(0)) + ee;
#pragma unroll
            for (int j = 0; j < CK; ++j) {
                const int k = k0 + j;
                if (k < k1) {
                    if (j > 0) {
                        ee = base + sA[k] * ee / dd + (k == nz - 1 ? etop : T(0));
                        dd = (k < nz - 1 ? sC[k] : T(0)) + ee;
                    }
                    rr[j] = (k < nz - 1) ? sC[k] / dd : T(0);
                }
            }
#pragma unroll
            for (int j = CK - 1; j >= 0; --j) {
                const int k = k0 + j;
                if (k < k1) {
                    const T x = col[k * TM] + rr[j] * xn;
                    col[k * TM] = x;
                    xn = x;
                    bad |= !isfinite(x);
                }
            }
        }
        if (sing0) {   // gauge: zero dzf-weighted mean
            double s = 0.0, sw = 0.0;
            for (int k = 0; k < nz; ++k) { s += a.dzf[k] * double(col[k * TM]); sw += a.dzf[k]; }
            const double m = s / sw;
            for (int k = 0; k < nz; ++k) col[k * TM] = T(double(col[k * TM]) - m);
        }
        if (a.adjoint)
            for (int k = 0; k < nz; ++k) col[k * TM] = T(double(col[k * TM]) * a.dzf[k]);
        if (bad && a.status) atomicOr(a.status, ST_BADPIVOT | ST_NONFINITE);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < nz; ++k)
        if (c < w) gp[(long)k * nmodes] = tile[k * TM + c];
}

template <typename T>
cudaError_t launch_zsolve(const ZArgs<T>& a, cudaStream_t st) {
    constexpr int CK = 16;
    const int nck = (a.nz + CK - 1) / CK;
    const size_t sm = ((size_t)a.nz * a.tm + (size_t)nck * a.tm + 2 * (size_t)a.nz) * sizeof(T);
    auto kern = k_zsolve<T, CK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const long nmodes = (long)a.nx * a.ny;
    const unsigned grid = (unsigned)((nmodes + a.tm - 1) / a.tm);
    kern<<<grid, a.tm, sm, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_zsolve<double>(const ZArgs<double>&, cudaStream_t);
template cudaError_t launch_zsolve<float>(const ZArgs<float>&, cudaStream_t);

}  // namespace cales

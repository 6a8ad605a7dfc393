// z direction of the eigenfunction expansion: one tridiagonal system per mode
// (mx, my), solved along the stretched direction (Thomas algorithm, Sec. 2.2).
// For (sigma - alpha L) u = g with L = L_z + lambda(mx, my):
//
//   row k:  -A_k u[k-1] + (sigma - alpha lambda + A_k + C_k + bc) u[k] - C_k u[k+1] = g_k
//   A_k = alpha / (dzc[k] dzf[k]),  C_k = alpha / (dzc[k+1] dzf[k])
//
// Pivots are carried in excess form d_k = C~_k + e_k (C~_k = C_k below the top
// row, 0 on it) with
//   e_k = (sigma - alpha lambda) + A_k e_{k-1} / d_{k-1}   (+ boundary terms)
// in which every term is non-negative: no cancellation even for the
// near-singular low modes on a strongly stretched grid.
//
// Layout and parallelism.  A CTA owns `tm` consecutive modes (contiguous in
// memory) and the whole z extent.  The [nz][tm] tile is moved between global
// and shared memory by TMA bulk copies, one row per copy.  P threads share a
// mode, each owning a segment of about nz/P rows:
//   A  the pivot recurrence of a segment is a product of 2x2 positive matrices
//      (a Moebius map of e), composed in the segment and chained across the P
//      lanes with shuffles;
//   C  the forward elimination y_k = (g_k + A_k y_{k-1}) / d_k is affine in
//      y_{k-1}: composed per segment, chained across lanes;
//   E  the segment is swept with the correct incoming state, writing y_k and
//      composing the back-substitution map x_k0 = Q + R x_k1;
//   F  the back-substitution maps are chained from the top segment down;
//   G  each segment back-substitutes, recomputing its pivots chunk by chunk
//      from checkpoints, so shared memory holds only the tile.
// Mode (0,0) of a singular Poisson problem is redone by one thread: its
// right-hand side is projected (dzf-weighted mean removed), its last row is
// pinned to zero and the result is gauged to zero weighted mean.
#include "kernels.cuh"

namespace cales {

template <typename T> __device__ __forceinline__ T rcp_(T d);
template <> __device__ __forceinline__ float rcp_<float>(float d) { return __frcp_rn(d); }
// FP64: FP32 reciprocal refined by two Newton steps (24 -> 48 -> ~53 bits);
// IEEE FP64 division is far slower on GB300's narrow FP64 pipe.
template <> __device__ __forceinline__ double rcp_<double>(double d) {
    double r = (double)__frcp_rn((float)d);
    r = r * fma(-d, r, 2.0);
    r = r * fma(-d, r, 2.0);
    return r;
}

// Pivot recurrence state: e_k and 1 / d_k of the last row visited.
template <typename T> struct Piv {
    T e, inv;
    const T *sA, *sC;
    T base, ebot, etop;
    int nz;
    __device__ __forceinline__ T ct(int k) const { return k < nz - 1 ? sC[k] : T(0); }
    __device__ __forceinline__ void first() {        // row 0
        e = base + ebot + (nz == 1 ? etop : T(0));
        inv = rcp_<T>(ct(0) + e);
    }
    __device__ __forceinline__ void step(int k) {     // row k >= 1 from row k-1
        e = base + sA[k] * e * inv + (k == nz - 1 ? etop : T(0));
        inv = rcp_<T>(ct(k) + e);
    }
    // start a sweep at row k0 given e of row k0-1 (ignored when k0 == 0)
    __device__ __forceinline__ void start(int k0, T e_prev) {
        if (k0 == 0) {
            first();
        } else {
            e = e_prev;
            inv = rcp_<T>(ct(k0 - 1) + e_prev);
            step(k0);
        }
    }
};

// Serial solve of one line (the singular mode 0): raw g0 -> x into col.
template <typename T>
__device__ void serial_line(T* tile, int stride, int m, int segs, const T* g0, T* r0, const T* sA, const T* sC, const T* sG,
                            const T* sO, const double* dzf, int nz, T base, bool singular, double* cacc,
                            double cacc_scale) {
    double gmean = 0.0;
    if (singular) {
        double s = 0.0, sw = 0.0;
        for (int k = 0; k < nz; ++k) {
            s += dzf[k] * double(g0[k]) * double(sG[k]);
            sw += dzf[k];
        }
        gmean = s / sw;
        if (cacc) cacc[0] += gmean * cacc_scale;
    }
    Piv<T> pv{T(0), T(0), sA, sC, base, T(0), T(0), nz};
    T y = T(0);
    for (int k = 0; k < nz; ++k) {
        if (k == 0) pv.first(); else pv.step(k);
        const T g = T(double(g0[k]) * double(sG[k]) - gmean);
        if (singular && k == nz - 1) y = T(0);
        else y = (g + (k > 0 ? sA[k] : T(0)) * y) * pv.inv;
        tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = y;
        r0[k] = (k < nz - 1) ? pv.ct(k) * pv.inv : T(0);
    }
    T x = T(0);
    for (int k = nz - 1; k >= 0; --k) {
        x = tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] + r0[k] * x;
        tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = x;
    }
    if (singular) {
        double s = 0.0, sw = 0.0;
        for (int k = 0; k < nz; ++k) { s += dzf[k] * double(tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride]); sw += dzf[k]; }
        const double mm = s / sw;
        for (int k = 0; k < nz; ++k) tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = T(double(tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride]) - mm);
    }
    for (int k = 0; k < nz; ++k) tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] *= sO[k];
}

// Segment stride of the shared tile (elements): m*tm rounded so that the P
// segments of a mode fall in different banks (stride = 32/P mod 32 words for
// FP32) while every row stays 16-byte aligned for the bulk copies.
template <typename T> __host__ __device__ __forceinline__ int zseg_stride(int m, int tm, int P) {
    const int words = (int)sizeof(T) / 4;
    const int want = P <= 8 ? (32 / P) / words : 0;     // residue in elements
    const int align = 16 / (int)sizeof(T);
    int st = m * tm;
    if (want > 0) {
        int r = st % (32 / words);
        int add = (want - r + 32 / words) % (32 / words);
        st += add;
    }
    return (st + align - 1) / align * align;
}

template <typename T, int P, int CK>
__global__ void __launch_bounds__(256) k_zsolve(ZArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TM = a.tm, nz = a.nz;
    const int m = (nz + P - 1) / P;
    const int nchs = (m + CK - 1) / CK;
    const long nmodes = (long)a.nx * a.ny;
    const int nthr = blockDim.x;
    const int segs = zseg_stride<T>(m, TM, P);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    T* tile = reinterpret_cast<T*>(smem_raw + 16);
    T* ck = tile + (long)segs * P;
    T* sA = ck + (long)nchs * nthr;
    T* sC = sA + nz;
    T* sG = sC + nz;
    T* sO = sG + nz;
    T* save0 = sO + nz;
    T* r0 = save0 + nz;
    const long q0 = (long)blockIdx.x * TM;
    const int w = (int)min((long)TM, nmodes - q0);
    const int tid = threadIdx.x;

    if (a.bulk && tid == 0) mbar_init(bar, 1);
    for (int k = tid; k < nz; k += nthr) {
        sA[k] = a.alpha * a.za[k];
        sC[k] = a.alpha * a.zc[k];
        double gs = double(a.scale), os = 1.0;
        if (a.adjoint) { gs /= a.dzf[k]; os = a.dzf[k]; }
        sG[k] = T(gs);
        sO[k] = T(os);
    }
    __syncthreads();
    if (a.bulk) {
        if (tid < 32) {
            const uint32_t rowb = (uint32_t)(w * sizeof(T));
            if (tid == 0) mbar_expect_tx(bar, rowb * (uint32_t)nz);
            __syncwarp();
            for (int k = tid; k < nz; k += 32) {
                const int sg = k / m;
                bulk_g2s(tile + (long)sg * segs + (long)(k - sg * m) * TM, a.data + q0 + (long)k * nmodes, rowb, bar);
            }
        }
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, 0);
            return;
        }
    } else {
        for (long e = tid; e < (long)nz * TM; e += nthr) {
            const int k = (int)(e / TM), c = (int)(e - (long)k * TM);
            const int sg = k / m;
            tile[(long)sg * segs + (long)(k - sg * m) * TM + c] = c < w ? a.data[(long)k * nmodes + q0 + c] : T(0);
        }
        __syncthreads();
    }
    const bool sing_tile = a.singular && q0 == 0;
    if (sing_tile && tid == 0)
        for (int k = 0; k < nz; ++k) save0[k] = tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * TM];
    __syncthreads();

    const int c = tid / P, s = tid - c * P;
    const unsigned lane = tid & 31;
    const unsigned gmask = P == 32 ? 0xffffffffu : (((1u << P) - 1u) << (lane & ~(unsigned)(P - 1)));
    bool bad = false;
    if (c < w) {
        const long q = q0 + c;
        const int my = (int)(q / a.nx), mx = (int)(q - (long)my * a.nx);
        const T lam = a.lamx[mx] + a.lamy[my];
        const T base = a.sigma - a.alpha * lam;
        const T ebot = a.zlo == ZBC_D ? T(2) * sA[0] : (a.zlo == ZBC_DF ? sA[0] : T(0));
        const T etop = a.zhi == ZBC_D ? T(2) * sC[nz - 1] : (a.zhi == ZBC_DF ? sC[nz - 1] : T(0));
        const int k0 = s * m, k1 = min(k0 + m, nz);
        T* col = tile + (long)s * segs + c - (long)k0 * TM;   // row k of this segment at col[k * TM]
        Piv<T> pv{T(0), T(0), sA, sC, base, ebot, etop, nz};

        // A: composite pivot map of the segment
        T g11 = T(1), g12 = T(0), g21 = T(0), g22 = T(1);
        T e_end = T(0);
        if (s == 0) {
            if (k1 > 0) {
                pv.first();
                for (int k = 1; k < k1; ++k) pv.step(k);
                e_end = pv.e;
            }
        } else {
            for (int k = k0; k < k1; ++k) {
                const T x = (k == nz - 1) ? etop : T(0);
                const T am = base + sA[k] + x, bm = (base + x) * sC[k - 1], cm = sC[k - 1];
                const T n11 = am * g11 + bm * g21, n12 = am * g12 + bm * g22;
                const T n21 = g11 + cm * g21, n22 = g12 + cm * g22;
                g11 = n11; g12 = n12; g21 = n21; g22 = n22;
                if (((k - k0) & 3) == 3) {
                    const T nrm = rcp_<T>(g11 + g12 + g21 + g22);
                    g11 *= nrm; g12 *= nrm; g21 *= nrm; g22 *= nrm;
                }
            }
        }
        // B: chain the pivot maps across the lanes of the mode
        T e_in = T(0);
        for (int j = 1; j < P; ++j) {
            const T t = __shfl_up_sync(gmask, e_end, 1, P);
            if (s == j) {
                e_in = t;
                e_end = (g11 * t + g12) * rcp_<T>(g21 * t + g22);
            }
        }
        // C: affine composite of the forward elimination over the segment
        T al = T(1), be = T(0);
        for (int k = k0; k < k1; ++k) {
            if (k == k0) pv.start(k0, e_in); else pv.step(k);
            const T ak = k > 0 ? sA[k] : T(0);
            const T g = col[(long)k * TM] * sG[k];
            al = ak * pv.inv * al;
            be = (g + ak * be) * pv.inv;
        }
        T y_end = (s == 0) ? be : T(0);
        T y_in = T(0);
        for (int j = 1; j < P; ++j) {
            const T t = __shfl_up_sync(gmask, y_end, 1, P);
            if (s == j) {
                y_in = t;
                y_end = al * t + be;
            }
        }
        // E: forward sweep writing y, checkpoints, back-substitution composite
        T y = y_in, Q = T(0), R = T(1);
        for (int k = k0; k < k1; ++k) {
            if (k == k0) pv.start(k0, e_in); else pv.step(k);
            if (((k - k0) % CK) == 0) ck[((k - k0) / CK) * nthr + tid] = pv.e;
            const T ak = k > 0 ? sA[k] : T(0);
            y = (col[(long)k * TM] * sG[k] + ak * y) * pv.inv;
            col[(long)k * TM] = y;
            Q += R * y;
            R *= pv.ct(k) * pv.inv;
            bad |= !(pv.inv > T(0));
        }
        // F: chain the back-substitution maps from the top segment down
        T xs = Q, x_next = T(0);
        for (int j = P - 2; j >= 0; --j) {
            const T t = __shfl_down_sync(gmask, xs, 1, P);
            if (s == j) {
                x_next = t;
                xs = Q + R * t;
            }
        }
        // G: back-substitute the segment, chunks from the top
        T x = x_next;
        for (int ch = nchs - 1; ch >= 0; --ch) {
            const int kc0 = k0 + ch * CK;
            if (kc0 >= k1) continue;
            const int kc1 = min(kc0 + CK, k1);
            T rr[CK];
            Piv<T> qv{ck[ch * nthr + tid], T(0), sA, sC, base, ebot, etop, nz};
            qv.inv = rcp_<T>(qv.ct(kc0) + qv.e);
#pragma unroll
            for (int j = 0; j < CK; ++j) {
                const int k = kc0 + j;
                if (k < kc1) {
                    if (j > 0) qv.step(k);
                    rr[j] = qv.ct(k) * qv.inv;
                }
            }
#pragma unroll
            for (int j = CK - 1; j >= 0; --j) {
                const int k = kc0 + j;
                if (k < kc1) {
                    x = col[(long)k * TM] + rr[j] * x;
                    col[(long)k * TM] = x * sO[k];
                    bad |= !isfinite(x);
                }
            }
        }
        if (sing_tile && c == 0) bad = false;
    }
    if (bad && a.status) atomicOr(a.status, ST_BADPIVOT | ST_NONFINITE);
    __syncthreads();
    if (sing_tile && tid == 0) {
        const T base0 = a.sigma - a.alpha * (a.lamx[0] + a.lamy[0]);
        serial_line<T>(tile, TM, m, segs, save0, r0, sA, sC, sG, sO, a.dzf, nz, base0, true, a.cacc, a.cacc_scale);
        for (int k = 0; k < nz; ++k)
            if (!isfinite(tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * TM])) {
                if (a.status) atomicOr(a.status, ST_NONFINITE);
                break;
            }
    }
    if (a.bulk) {
        fence_proxy_async();
        __syncthreads();
        if (tid < 32) {
            const uint32_t rowb = (uint32_t)(w * sizeof(T));
            for (int k = tid; k < nz; k += 32) {
                const int sg = k / m;
                bulk_s2g(a.data + q0 + (long)k * nmodes, tile + (long)sg * segs + (long)(k - sg * m) * TM, rowb);
            }
            bulk_commit();
            bulk_wait_read_all();
        }
    } else {
        __syncthreads();
        for (long e = tid; e < (long)nz * TM; e += nthr) {
            const int k = (int)(e / TM), cc = (int)(e - (long)k * TM);
            const int sg = k / m;
            if (cc < w) a.data[(long)k * nmodes + q0 + cc] = tile[(long)sg * segs + (long)(k - sg * m) * TM + cc];
        }
    }
}

template <typename T>
size_t zsolve_smem(int nz, int tm, int P) {
    constexpr int CK = 16;
    const int m = (nz + P - 1) / P;
    const int nchs = (m + CK - 1) / CK;
    const size_t segs = (size_t)zseg_stride<T>(m, tm, P);
    return 16 + (segs * P + (size_t)nchs * tm * P + 6 * (size_t)nz) * sizeof(T);
}

template <typename T, int P>
static cudaError_t launch_zsolve_p(const ZArgs<T>& a, cudaStream_t st) {
    constexpr int CK = 16;
    const size_t sm = zsolve_smem<T>(a.nz, a.tm, P);
    auto kern = k_zsolve<T, P, CK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const long nmodes = (long)a.nx * a.ny;
    const unsigned grid = (unsigned)((nmodes + a.tm - 1) / a.tm);
    kern<<<grid, a.tm * P, sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zsolve(const ZArgs<T>& a, cudaStream_t st) {
    switch (a.P) {
        case 1: return launch_zsolve_p<T, 1>(a, st);
        case 2: return launch_zsolve_p<T, 2>(a, st);
        case 4: return launch_zsolve_p<T, 4>(a, st);
        case 8: return launch_zsolve_p<T, 8>(a, st);
        default: return launch_zsolve_p<T, 16>(a, st);
    }
}

template size_t zsolve_smem<double>(int, int, int);
template size_t zsolve_smem<float>(int, int, int);
template cudaError_t launch_zsolve<double>(const ZArgs<double>&, cudaStream_t);
template cudaError_t launch_zsolve<float>(const ZArgs<float>&, cudaStream_t);

}  // namespace cales

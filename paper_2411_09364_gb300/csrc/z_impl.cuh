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
#pragma once
#include "kernels.cuh"

namespace cales {

template <typename T> __device__ __forceinline__ T rcp_(T d);
template <> __device__ __forceinline__ float rcp_<float>(float d) { return __frcp_rn(d); }
// FP64: FP32 reciprocal refined by two Newton steps (24 -> 48 -> ~53 bits);
// IEEE FP64 division is far slower on GB300's narrow FP64 pipe.  The FP32
// seed needs 1/d to be a normal float: |d| in [2^-125, 2^125), tested on the
// exponent bits with integer operations; anything else (zero, tiny, huge,
// non-finite) takes the division.
template <> __device__ __forceinline__ double rcp_<double>(double d) {
    const unsigned e = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
    if (e - 898u > 249u) return 1.0 / d;
    double r = (double)__frcp_rn((float)d);
    r = __dmul_rn(r, __fma_rn(-d, r, 2.0));
    r = __dmul_rn(r, __fma_rn(-d, r, 2.0));
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
__device__ __noinline__ void serial_line(T* tile, int stride, int m, int segs, const T* g0, T* r0, const T* sA, const T* sC, const T* sG,
                            const T* sO, const double* dzf, int nz, T base, bool singular, double* cacc,
                            double cacc_scale, int sk, double shift = 0.0) {
    // coefficient tables may be skewed by one slot per segment of sk rows
#define SKI(k) ((sk) > 0 ? (k) + (k) / (sk) : (k))
    double gmean = 0.0;
    if (singular) {
        double s = 0.0, sw = 0.0;
        for (int k = 0; k < nz; ++k) {
            s += dzf[k] * double(g0[k]) * double(sG[SKI(k)]);
            sw += dzf[k];
        }
        gmean = s / sw;
        if (cacc) cacc[0] += gmean * cacc_scale;
    }
    T e = T(0), inv = T(0), y = T(0);
    for (int k = 0; k < nz; ++k) {
        const T ct = k < nz - 1 ? sC[SKI(k)] : T(0);
        e = (k == 0) ? base : base + sA[SKI(k)] * e * inv;
        inv = rcp_<T>(ct + e);
        const T g = T(double(g0[k]) * double(sG[SKI(k)]) - gmean);
        if (singular && k == nz - 1) y = T(0);
        else y = (g + (k > 0 ? sA[SKI(k)] : T(0)) * y) * inv;
        tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = y;
        r0[k] = (k < nz - 1) ? ct * inv : T(0);
    }
    T x = T(0);
    for (int k = nz - 1; k >= 0; --k) {
        x = tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] + r0[k] * x;
        tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = x;
    }
    if (singular) {
        double s = 0.0, sw = 0.0;
        for (int k = 0; k < nz; ++k) { s += dzf[k] * double(tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride]); sw += dzf[k]; }
        const double mm = s / sw + shift;      // gauge, and the caller's constant shift
        for (int k = 0; k < nz; ++k) tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] = T(double(tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride]) - mm);
    }
    for (int k = 0; k < nz; ++k) tile[(long)(k / m) * segs + (long)(k - (k / m) * m) * stride] *= sO[SKI(k)];
#undef SKI
}

// The same line by one warp, for Neumann sides on both ends of z and a zero
// diagonal shift (sigma = 0, lambda(0, 0) = 0).  Then every pivot excess is
// zero: d_k = C_k below the pinned last row, so the forward elimination
// y_k = (g_k + A_k y_{k-1}) / C_k and the back-substitution
// x_k = y_k + (C_k / d_k) x_{k+1} are affine recurrences.  Lane l takes rows
// [l R, l R + R) (R = ceil(nz / 32)); each recurrence is composed per chunk,
// the chunk maps are combined by a shuffle scan (lane order forward, reverse
// order backward) and the chunk is swept again from its incoming value.  The
// per-row arithmetic is that of serial_line; projection and gauge sums are
// warp reductions of the same FP64 terms.
template <typename T>
__device__ __noinline__ void singular_line_warp(T* tile, int stride, const T* g0, const T* sA, const T* sC, const T* sG, const T* sO,
                                   const double* dzf, int nz, double* cacc, double cacc_scale, double shift,
                                   int* status) {
    const unsigned FULLM = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int R = (nz + 31) / 32;
    const int k0 = min(nz, lane * R), k1 = min(nz, k0 + R);
    double sg = 0.0, sw = 0.0;
    for (int k = k0; k < k1; ++k) {
        sg += dzf[k] * double(g0[k]) * double(sG[k]);
        sw += dzf[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sg += __shfl_xor_sync(FULLM, sg, o);
        sw += __shfl_xor_sync(FULLM, sw, o);
    }
    const double gmean = sg / sw;
    if (lane == 0 && cacc) cacc[0] += gmean * cacc_scale;
    // forward: chunk map y_out = al * y_in + be
    T al = T(1), be = T(0);
    for (int k = k0; k < k1; ++k) {
        if (k == nz - 1) { al = T(0); be = T(0); continue; }
        const T inv = rcp_<T>(sC[k]);
        const T ak = k > 0 ? sA[k] : T(0);
        const T g = T(double(g0[k]) * double(sG[k]) - gmean);
        al = ak * inv * al;
        be = (g + ak * be) * inv;
    }
    for (int o = 1; o < 32; o <<= 1) {
        const T pa = __shfl_up_sync(FULLM, al, o), pb = __shfl_up_sync(FULLM, be, o);
        if (lane >= o) { be = al * pb + be; al = al * pa; }
    }
    T y = __shfl_up_sync(FULLM, be, 1);
    if (lane == 0) y = T(0);
    for (int k = k0; k < k1; ++k) {
        if (k == nz - 1) {
            y = T(0);
        } else {
            const T inv = rcp_<T>(sC[k]);
            const T ak = k > 0 ? sA[k] : T(0);
            const T g = T(double(g0[k]) * double(sG[k]) - gmean);
            y = (g + ak * y) * inv;
        }
        tile[(long)k * stride] = y;
    }
    // backward: chunk map x_top = Q + Rm * x_in (x_in: first row of the next chunk)
    T Q = T(0), Rm = T(1);
    for (int k = k1 - 1; k >= k0; --k) {
        const T r = k < nz - 1 ? sC[k] * rcp_<T>(sC[k]) : T(0);
        Q = tile[(long)k * stride] + r * Q;
        Rm = r * Rm;
    }
    for (int o = 1; o < 32; o <<= 1) {
        const T nq = __shfl_down_sync(FULLM, Q, o), nr = __shfl_down_sync(FULLM, Rm, o);
        if (lane + o < 32) { Q = Q + Rm * nq; Rm = Rm * nr; }
    }
    T x = __shfl_down_sync(FULLM, Q, 1);
    if (lane == 31) x = T(0);
    double sx = 0.0;
    for (int k = k1 - 1; k >= k0; --k) {
        const T r = k < nz - 1 ? sC[k] * rcp_<T>(sC[k]) : T(0);
        x = tile[(long)k * stride] + r * x;
        tile[(long)k * stride] = x;
        sx += dzf[k] * double(x);
    }
    for (int o = 16; o > 0; o >>= 1) sx += __shfl_xor_sync(FULLM, sx, o);
    const double mm = sx / sw + shift;      // gauge, and the caller's constant shift
    bool bad = false;
    for (int k = k0; k < k1; ++k) {
        const T v = T(double(tile[(long)k * stride]) - mm) * sO[k];
        tile[(long)k * stride] = v;
        bad |= !isfinite(v);
    }
    if (__any_sync(FULLM, bad) && lane == 0 && status) atomicOr(status, ST_NONFINITE);
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
        const T base0 = a.sigma - mul_(a.alpha, a.lamx[0] + a.lamy[0]);
        serial_line<T>(tile, TM, m, segs, save0, r0, sA, sC, sG, sO, a.dzf, nz, base0, true, a.cacc, a.cacc_scale, 0,
                       a.shift_acc ? a.shift_acc[0] * a.shift_scale : 0.0);
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


// Fast reciprocal: FP32 hardware approximation + one Newton step (about 1 ulp);
// FP64 as rcp_ (FP32 seed + two Newton steps).
template <typename T> __device__ __forceinline__ T frcp(T d);
template <> __device__ __forceinline__ float frcp<float>(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return __fmul_rn(r, __fmaf_rn(-d, r, 2.0f));
}
template <> __device__ __forceinline__ double frcp<double>(double d) { return rcp_<double>(d); }

// Segmented Thomas with the segment's pivot reciprocals held in registers
// (MAXM >= rows per segment).  Same phases as k_zsolve; the pivot recurrence
// runs once per row (phase C) instead of being recomputed.  Coefficient
// tables are skewed by one slot per segment so the P segments of a warp read
// different banks.
template <typename T, int P, int MAXM>
__global__ void __launch_bounds__(256) k_zsolve_reg(ZArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TM = a.tm, nz = a.nz;
    const int m = (nz + P - 1) / P;
    const long nmodes = (long)a.nx * a.ny;
    const int nthr = blockDim.x;
    const int segs = zseg_stride<T>(m, TM, P);
    const int nsk = nz + P;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    T* tile = reinterpret_cast<T*>(smem_raw + 16);
    T* sA = tile + segs * P;
    T* sC = sA + nsk;
    T* sG = sC + nsk;
    T* sO = sG + nsk;
    T* save0 = sO + nsk;
    T* r0 = save0 + nz;
    const long q0 = (long)blockIdx.x * TM;
    const int w = (int)min((long)TM, nmodes - q0);
    const int tid = threadIdx.x;

    if (a.bulk && tid == 0) mbar_init(bar, 1);
    for (int k = tid; k < nz; k += nthr) {
        const int pk = k + k / m;
        sA[pk] = a.alpha * a.za[k];
        sC[pk] = a.alpha * a.zc[k];
        double gs = double(a.scale), os = 1.0;
        if (a.adjoint) { gs /= a.dzf[k]; os = a.dzf[k]; }
        sG[pk] = T(gs);
        sO[pk] = T(os);
    }
    __syncthreads();
    if (a.bulk) {
        if (tid < 32) {
            const uint32_t rowb = (uint32_t)(w * sizeof(T));
            if (tid == 0) mbar_expect_tx(bar, rowb * (uint32_t)nz);
            __syncwarp();
            for (int k = tid; k < nz; k += 32) {
                const int sg = k / m;
                bulk_g2s(tile + sg * segs + (k - sg * m) * TM, a.data + q0 + (long)k * nmodes, rowb, bar);
            }
        }
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, 0);
            return;
        }
    } else {
        for (int e = tid; e < nz * TM; e += nthr) {
            const int k = e / TM, c = e - k * TM;
            const int sg = k / m;
            tile[sg * segs + (k - sg * m) * TM + c] = c < w ? a.data[(long)k * nmodes + q0 + c] : T(0);
        }
        __syncthreads();
    }
    const bool sing_tile = a.singular && q0 == 0;
    if (sing_tile && tid == 0)
        for (int k = 0; k < nz; ++k) save0[k] = tile[(k / m) * segs + (k - (k / m) * m) * TM];
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
        const int ktop = (nz - 1) + (nz - 1) / m;
        const T etop = a.zhi == ZBC_D ? T(2) * sC[ktop] : (a.zhi == ZBC_DF ? sC[ktop] : T(0));
        const int k0 = s * m;
        const int mseg = max(0, min(m, nz - k0));
        const T* A = sA + k0 + s;
        const T* Cc = sC + k0 + s;
        const T* G = sG + k0 + s;
        const T* O = sO + k0 + s;
        T* col = tile + s * segs + c;
        const T cprev = s > 0 ? sC[(k0 - 1) + (s - 1)] : T(0);
#define CT(j) ((k0 + (j) < nz - 1) ? Cc[j] : T(0))
#define XT(j) ((k0 + (j) == nz - 1) ? etop : T(0))

        // A: composite pivot map of the segment (2x2 positive matrices)
        T g11 = T(1), g12 = T(0), g21 = T(0), g22 = T(1);
        T e_end = T(0);
        if (s == 0) {
            if (mseg > 0) {
                T e = base + ebot + (nz == 1 ? etop : T(0));
#pragma unroll
                for (int j = 1; j < MAXM; ++j)
                    if (j < mseg) e = base + A[j] * e * frcp<T>(CT(j - 1) + e) + XT(j);
                e_end = e;
            }
        } else {
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                if (j < mseg) {
                    const T x = XT(j);
                    const T cm = j > 0 ? Cc[j - 1] : cprev;
                    const T am = base + A[j] + x, bm = (base + x) * cm;
                    const T n11 = am * g11 + bm * g21, n12 = am * g12 + bm * g22;
                    const T n21 = g11 + cm * g21, n22 = g12 + cm * g22;
                    g11 = n11; g12 = n12; g21 = n21; g22 = n22;
                    if ((j & 3) == 3) {
                        const T nrm = frcp<T>(g11 + g12 + g21 + g22);
                        g11 *= nrm; g12 *= nrm; g21 *= nrm; g22 *= nrm;
                    }
                }
            }
        }
        // B: chain the pivot maps across the lanes
        T e_in = T(0);
#pragma unroll
        for (int j = 1; j < P; ++j) {
            const T t = __shfl_up_sync(gmask, e_end, 1, P);
            if (s == j) {
                e_in = t;
                e_end = (g11 * t + g12) * frcp<T>(g21 * t + g22);
            }
        }
        // C: pivots of the segment (kept in registers) and the affine
        //    composite of the forward elimination
        T inv[MAXM];
        T al = T(1), be = T(0);
        {
            T e;
            if (k0 == 0) e = base + ebot + (nz == 1 ? etop : T(0));
            else e = base + A[0] * e_in * frcp<T>(cprev + e_in) + XT(0);
#pragma unroll
            for (int j = 0; j < MAXM; ++j) {
                if (j < mseg) {
                    if (j > 0) e = base + A[j] * e * inv[j - 1] + XT(j);
                    inv[j] = frcp<T>(CT(j) + e);
                    const T ak = (k0 + j > 0) ? A[j] : T(0);
                    al = ak * inv[j] * al;
                    be = (col[j * TM] * G[j] + ak * be) * inv[j];
                    bad |= !(inv[j] > T(0));
                }
            }
        }
        T y_end = (s == 0) ? be : T(0);
        T y_in = T(0);
#pragma unroll
        for (int j = 1; j < P; ++j) {
            const T t = __shfl_up_sync(gmask, y_end, 1, P);
            if (s == j) {
                y_in = t;
                y_end = al * t + be;
            }
        }
        // E: forward sweep writing y; back-substitution composite
        T y = y_in, Q = T(0), R = T(1);
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            if (j < mseg) {
                const T ak = (k0 + j > 0) ? A[j] : T(0);
                y = (col[j * TM] * G[j] + ak * y) * inv[j];
                col[j * TM] = y;
                Q += R * y;
                R *= CT(j) * inv[j];
            }
        }
        // F: chain the back-substitution maps from the top segment down
        T xs = Q, x_next = T(0);
#pragma unroll
        for (int j = P - 2; j >= 0; --j) {
            const T t = __shfl_down_sync(gmask, xs, 1, P);
            if (s == j) {
                x_next = t;
                xs = Q + R * t;
            }
        }
        // G: back-substitution
        T x = x_next;
#pragma unroll
        for (int j = MAXM - 1; j >= 0; --j) {
            if (j < mseg) {
                x = col[j * TM] + CT(j) * inv[j] * x;
                col[j * TM] = x * O[j];
                bad |= !isfinite(x);
            }
        }
#undef CT
#undef XT
        if (sing_tile && c == 0) bad = false;
    }
    if (bad && a.status) atomicOr(a.status, ST_BADPIVOT | ST_NONFINITE);
    __syncthreads();
    if (sing_tile && tid == 0) {
        const T base0 = a.sigma - mul_(a.alpha, a.lamx[0] + a.lamy[0]);
        serial_line<T>(tile, TM, m, segs, save0, r0, sA, sC, sG, sO, a.dzf, nz, base0, true, a.cacc, a.cacc_scale, m,
                       a.shift_acc ? a.shift_acc[0] * a.shift_scale : 0.0);
        for (int k = 0; k < nz; ++k)
            if (!isfinite(tile[(k / m) * segs + (k - (k / m) * m) * TM])) {
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
                bulk_s2g(a.data + q0 + (long)k * nmodes, tile + sg * segs + (k - sg * m) * TM, rowb);
            }
            bulk_commit();
            bulk_wait_read_all();
        }
    } else {
        __syncthreads();
        for (int e = tid; e < nz * TM; e += nthr) {
            const int k = e / TM, cc = e - k * TM;
            const int sg = k / m;
            if (cc < w) a.data[(long)k * nmodes + q0 + cc] = tile[sg * segs + (k - sg * m) * TM + cc];
        }
    }
}

template <typename T>
size_t zsolve_reg_smem(int nz, int tm, int P) {
    const int m = (nz + P - 1) / P;
    const size_t segs = (size_t)zseg_stride<T>(m, tm, P);
    return 16 + (segs * P + 4 * (size_t)(nz + P) + 2 * (size_t)nz) * sizeof(T);
}

template <typename T, int P, int MAXM>
static cudaError_t launch_zsolve_reg(const ZArgs<T>& a, cudaStream_t st) {
    const size_t sm = zsolve_reg_smem<T>(a.nz, a.tm, P);
    auto kern = k_zsolve_reg<T, P, MAXM>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const long nmodes = (long)a.nx * a.ny;
    const unsigned grid = (unsigned)((nmodes + a.tm - 1) / a.tm);
    kern<<<grid, a.tm * P, sm, st>>>(a);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Warp-per-segment variant: a CTA owns 32 consecutive modes; warp s owns rows
// [s*m, s*m + m) of all 32 modes, so every shared-memory row access of a warp
// is one contiguous 128-byte (FP32) row and every coefficient read is a
// broadcast.  The tile moves by 16-byte cp.async copies (all in flight at
// once) and vector stores.  Segment states pass through shared memory: warp 0
// chains the pivot maps, each warp the elimination maps before and after its
// own segment.  Pivot reciprocals of a segment stay in registers.
// Every product that feeds a sum is rounded explicitly (mul_ / fma_), so the
// compiler's FMA contraction cannot differ between the instantiations (full
// or ragged segments, one-tile, grouped, persistent): all of them give
// bit-identical solves.
// ---------------------------------------------------------------------------
template <typename T> struct alignas(2 * sizeof(T)) ZPair { T a, c; };

// Coefficient tables of the warp-per-segment kernels in shared memory:
// sA, sC (alpha-scaled couplings), sG, sO (adjoint weights), the (A_k, C_k)
// pairs sAC with A_0 = 0 and C_{nz-1} = 0 (one 8-byte (FP32) or 16-byte
// (FP64) load per row and no first/last-row tests), and two nz-long scratch
// lines of the singular mode (save0, r0).
template <typename T> struct ZwTables {
    T *sA, *sC, *sG, *sO, *save0, *r0;
    ZPair<T>* sAC;
    __device__ ZwTables(T* base, int nz) {
        sA = base; sC = sA + nz; sG = sC + nz; sO = sG + nz; save0 = sO + nz; r0 = save0 + nz;
        sAC = reinterpret_cast<ZPair<T>*>(r0 + nz);
    }
    __device__ void fill(const ZArgs<T>& a) {
        const int nz = a.nz;
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            sA[k] = a.alpha * a.za[k];
            sC[k] = a.alpha * a.zc[k];
            ZPair<T> pr;
            pr.a = k > 0 ? sA[k] : T(0);
            pr.c = k < nz - 1 ? sC[k] : T(0);
            sAC[k] = pr;
            double gs = double(a.scale), os = 1.0;
            if (a.adjoint) { gs /= a.dzf[k]; os = a.dzf[k]; }
            sG[k] = T(gs);
            sO[k] = T(os);
        }
    }
};

// Rows [0, nz) of the 32 modes q0 .. q0+31 of `in` into the tile [nz][32] with
// 16-byte cp.async copies (zero-filled past the w live modes); completion by
// the caller's commit / wait.
template <typename T>
__device__ __forceinline__ void zw_load_async(T* tile, const T* __restrict__ in, long nmodes, long q0, int w, int nz) {
    constexpr int TM = 32, EPC = 16 / (int)sizeof(T), CPR = TM / EPC;
    for (int e = threadIdx.x; e < nz * CPR; e += blockDim.x) {
        const int k = e / CPR, c0 = (e - k * CPR) * EPC;
        cp_async16(tile + k * TM + c0, in + (long)k * nmodes + q0 + (c0 < w ? c0 : 0), c0 < w);
    }
}

template <typename T>
__device__ __forceinline__ void zw_store(T* __restrict__ out, const T* tile, long nmodes, long q0, int w, int nz) {
    constexpr int TM = 32, EPC = 16 / (int)sizeof(T), CPR = TM / EPC;
    for (int e = threadIdx.x; e < nz * CPR; e += blockDim.x) {
        const int k = e / CPR, c0 = (e - k * CPR) * EPC;
        if (c0 < w)
            *reinterpret_cast<float4*>(out + (long)k * nmodes + q0 + c0) = *reinterpret_cast<const float4*>(tile + k * TM + c0);
    }
}

// The solve of one tile of 32 modes (q0 .. q0 + w - 1) already in shared
// memory, in place; every thread of the CTA takes part (P warps, warp s owns
// rows [s m, s m + m)).  Phases as in the header of this file; the segment
// states pass through `ch` (6 x [P][32]).
// FULL: every segment has exactly MAXM rows (nz = P * MAXM), so the row
// predicates and the first/last-row conditions reduce to compile-time tests
// on j plus one warp-uniform test on s.  ADJ: the adjoint weights (Eq. 16
// transposed) instead of the uniform forward scale.
template <typename T, int MAXM, bool FULL, bool ADJ>
__device__ __forceinline__ void zw_solve_tile(const ZArgs<T>& a, T* tile, T* ch, const ZwTables<T>& tb, long q0,
                                              int w, const int P, const int Pb, const bool pending = false) {
    // pending: the tile's cp.async copies and the table fill may still be in
    // flight; the per-mode global loads below are issued first, then the CTA
    // waits for its copies and synchronises.
    // P: segments of this line; Pb = blockDim.x / 32 >= P warps, the chain
    // arrays hold Pb slots.  Warps s >= P (grouped launches over lines of
    // different depth) own no rows and only take part in the barriers.
    constexpr int TM = 32;
    const int nz = a.nz;
    const int m = (nz + P - 1) / P;
    const int tid = threadIdx.x;
    const T* sA = tb.sA;
    const T* sC = tb.sC;
    const ZPair<T>* sAC = tb.sAC;
    const bool sing_tile = a.singular && q0 == 0;
    const int s = tid >> 5, c = tid & 31;
    const long q = q0 + (c < w ? c : 0);
    int my, mx;
    if ((long)a.nx * a.ny < (1L << 31)) { my = (int)q / a.nx; mx = (int)q - my * a.nx; }
    else { my = (int)(q / a.nx); mx = (int)(q - (long)my * a.nx); }
    const T lam = a.lamx[mx] + a.lamy[my];
    // cached segment-entry pivot (stride 0: every lane of every CTA reads the same slot)
    const T e_cached = (a.ecache_mode == 2 && s > 0)
                           ? a.ecache[a.ecache_stride ? (long)s * a.ecache_stride + q : (long)s] : T(0);
    if (pending) {
        cp_async_wait_all();
        __syncthreads();
    }
    if (sing_tile && tid == 0)
        for (int k = 0; k < nz; ++k) tb.save0[k] = tile[k * TM];
    const T base = a.sigma - mul_(a.alpha, lam);
    const T ebot = a.zlo == ZBC_D ? mul_(T(2), sA[0]) : (a.zlo == ZBC_DF ? sA[0] : T(0));
    const T etop = a.zhi == ZBC_D ? mul_(T(2), sC[nz - 1]) : (a.zhi == ZBC_DF ? sC[nz - 1] : T(0));
    const bool act = s < P;
    const int k0 = act ? s * m : 0;
    const int mseg = act ? max(0, min(m, nz - k0)) : 0;
    const ZPair<T>* AC = sAC + k0;
    const T* G = tb.sG + k0;
    const T* O = tb.sO + k0;
    const T gsc = T(a.scale);
    const bool lastseg = s == P - 1, firstseg = s == 0;
    (void)lastseg; (void)firstseg;
    T* col = tile + k0 * TM + c;
    T* c11 = ch;
    T* c12 = ch + Pb * TM;
    T* c21 = ch + 2 * Pb * TM;
    T* c22 = ch + 3 * Pb * TM;
    T* cin = ch + 4 * Pb * TM;
    const int me = s * TM + c;
#define XT(j) (FULL ? (((j) == MAXM - 1 && lastseg) ? etop : T(0)) : ((k0 + (j) == nz - 1) ? etop : T(0)))
#define GW(j) (ADJ ? G[j] : gsc)
#define INSEG(j) (FULL || (j) < mseg)
    bool bad = false;

    T e_in;
    if (a.ecache_mode == 2) {
        e_in = e_cached;
    } else {
        // A: composite pivot map of the segment
        {
            T g11 = T(1), g12 = T(0), g21 = T(0), g22 = T(1);
            if (s == 0) {
                T e = base + ebot + (nz == 1 ? etop : T(0));
    #pragma unroll
                for (int j = 1; j < MAXM; ++j)
                    if (INSEG(j)) e = fma_(mul_(AC[j].a, e), frcp<T>(AC[j - 1].c + e), base) + XT(j);
                g11 = T(0); g12 = e; g21 = T(0); g22 = T(1);         // constant map -> e_end
            } else {
    #pragma unroll
                for (int j = 0; j < MAXM; ++j) {
                    if (INSEG(j)) {
                        const T x = XT(j);
                        const T cm = AC[j - 1].c;              // k0 + j - 1 >= 0 for s > 0
                        const T am = base + AC[j].a + x, bm = mul_(base + x, cm);
                        const T n11 = fma_(am, g11, mul_(bm, g21)), n12 = fma_(am, g12, mul_(bm, g22));
                        const T n21 = fma_(cm, g21, g11), n22 = fma_(cm, g22, g12);
                        g11 = n11; g12 = n12; g21 = n21; g22 = n22;
                        if ((j & 3) == 3) {
                            const T nrm = frcp<T>(g11 + g12 + g21 + g22);
                            g11 = mul_(g11, nrm); g12 = mul_(g12, nrm); g21 = mul_(g21, nrm); g22 = mul_(g22, nrm);
                        }
                    }
                }
            }
            c11[me] = g11; c12[me] = g12; c21[me] = g21; c22[me] = g22;
        }
        __syncthreads();
        if (s == 0) {       // chain: e entering segment t = map_{t-1}(...map_0)
            T e = T(0);
            for (int t = 0; t < P; ++t) {
                const int i = t * TM + c;
                cin[i] = e;
                e = mul_(fma_(c11[i], e, c12[i]), frcp<T>(fma_(c21[i], e, c22[i])));
            }
        }
        __syncthreads();
        e_in = cin[me];
        // (stride 0: every lane of every CTA stores the same value)
        if (a.ecache_mode == 1 && act && s > 0 && c < w)
            a.ecache[a.ecache_stride ? (long)s * a.ecache_stride + q : (long)s] = e_in;
    }
    // C: pivots (registers) and the affine composite of the forward sweep
    T inv[MAXM];
    T al = T(1), be = T(0);
    {
        T e;
        if (k0 == 0) e = base + ebot + (nz == 1 ? etop : T(0));
        else e = fma_(mul_(AC[0].a, e_in), frcp<T>(AC[-1].c + e_in), base) + XT(0);
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            if (INSEG(j)) {
                const ZPair<T> ac = AC[j];
                if (j > 0) e = fma_(mul_(ac.a, e), inv[j - 1], base) + XT(j);
                inv[j] = frcp<T>(ac.c + e);
                al = mul_(mul_(ac.a, inv[j]), al);
                be = mul_(fma_(ac.a, be, mul_(col[j * TM], GW(j))), inv[j]);
                bad |= !(inv[j] > T(0));
            }
        }
    }
    c11[me] = al;
    c12[me] = be;
    __syncthreads();
    // E: forward sweep writing y, back-substitution composite.  Each warp
    // chains the affine maps of the segments before its own (in segment
    // order, four segments' coefficients loaded ahead of their dependent
    // steps), so no warp waits for a serial chain and a second barrier.
    {
        T y = T(0);
        for (int t0 = 0; t0 < s && act; t0 += 4) {
            T ka[4], kb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (t0 + u < s) { ka[u] = c11[(t0 + u) * TM + c]; kb[u] = c12[(t0 + u) * TM + c]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (t0 + u < s) y = fma_(ka[u], y, kb[u]);
        }
        T Q = T(0), R = T(1);
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            if (INSEG(j)) {
                const ZPair<T> ac = AC[j];
                y = mul_(fma_(ac.a, y, mul_(col[j * TM], GW(j))), inv[j]);
                col[j * TM] = y;
                Q = fma_(R, y, Q);
                R = mul_(R, mul_(ac.c, inv[j]));
            }
        }
        c21[me] = Q;
        c22[me] = R;
    }
    __syncthreads();
    // G: back-substitution; each warp chains the back-substitution maps of
    // the segments above its own, from the top segment down
    {
        T x = T(0), xs = T(0);
        for (int t0 = P - 1; t0 > s && act; t0 -= 4) {
            T kq[4], kr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (t0 - u > s) { kq[u] = c21[(t0 - u) * TM + c]; kr[u] = c22[(t0 - u) * TM + c]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (t0 - u > s) x = fma_(kr[u], x, kq[u]);
        }
#pragma unroll
        for (int j = MAXM - 1; j >= 0; --j) {
            if (INSEG(j)) {
                x = fma_(mul_(AC[j].c, inv[j]), x, col[j * TM]);
                col[j * TM] = ADJ ? mul_(x, O[j]) : x;
                xs += x;
            }
        }
        bad |= !isfinite(xs);
    }
#undef XT
#undef GW
#undef INSEG
    if ((sing_tile && c == 0) || c >= w) bad = false;
    if (bad && a.status) atomicOr(a.status, ST_BADPIVOT | ST_NONFINITE);
    __syncthreads();
    if (sing_tile && s == 0) {
        const T base0 = a.sigma - mul_(a.alpha, a.lamx[0] + a.lamy[0]);
        const double shift = a.shift_acc ? a.shift_acc[0] * a.shift_scale : 0.0;
        if (base0 == T(0) && a.zlo == ZBC_N && a.zhi == ZBC_N) {
            singular_line_warp<T>(tile, TM, tb.save0, sA, sC, tb.sG, tb.sO, a.dzf, nz, a.cacc, a.cacc_scale, shift,
                                  a.status);
        } else if (c == 0) {
            serial_line<T>(tile, TM, nz, 0, tb.save0, tb.r0, sA, sC, tb.sG, tb.sO, a.dzf, nz, base0, true, a.cacc,
                           a.cacc_scale, 0, shift);
            for (int k = 0; k < nz; ++k)
                if (!isfinite(tile[k * TM])) {
                    if (a.status) atomicOr(a.status, ST_NONFINITE);
                    break;
                }
        }
    }
    __syncthreads();
}

// One tile of 32 consecutive modes per CTA: load (16-byte cp.async, all in
// flight), solve, store.  P segments (warps) of the line, Pb = blockDim / 32.
template <typename T, int MAXM, bool FULL, bool ADJ>
__device__ __forceinline__ void zw_kernel_body(const ZArgs<T>& a, const int bx, const int P, const int Pb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TM = 32;
    const int nz = a.nz;
    const int m = (nz + P - 1) / P;
    const long nmodes = (long)a.nx * a.ny;
    T* tile = reinterpret_cast<T*>(smem_raw);          // [P*m][32]
    T* ch = tile + (long)P * m * TM;                   // 6 x [Pb][32] chain states
    ZwTables<T> tb(ch + 6 * Pb * TM, nz);
    const long q0 = (long)bx * TM;
    const int w = (int)min((long)TM, nmodes - q0);
    const T* __restrict__ in = a.src ? a.src : a.data;
    // the tile copy is issued first; the coefficient tables are filled and
    // the per-mode values loaded while it is in flight
    if (a.bulk) {
        zw_load_async<T>(tile, in, nmodes, q0, w, nz);
    } else {
        for (int e = threadIdx.x; e < nz * TM; e += blockDim.x) {
            const int k = e / TM, c = e - k * TM;
            tile[e] = c < w ? in[(long)k * nmodes + q0 + c] : T(0);
        }
    }
    tb.fill(a);
    zw_solve_tile<T, MAXM, FULL, ADJ>(a, tile, ch, tb, q0, w, P, Pb, true);
    if (a.bulk) {
        zw_store<T>(a.data, tile, nmodes, q0, w, nz);
    } else {
        for (int e = threadIdx.x; e < nz * TM; e += blockDim.x) {
            const int k = e / TM, cc = e - k * TM;
            if (cc < w) a.data[(long)k * nmodes + q0 + cc] = tile[e];
        }
    }
}

template <typename T, int MAXM, bool FULL, bool ADJ>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_zsolve_w(const __grid_constant__ ZArgs<T> a) {
    zw_kernel_body<T, MAXM, FULL, ADJ>(a, blockIdx.x, blockDim.x / 32, blockDim.x / 32);
}

// Grouped launch (z stage of many solves): CTA b solves tile work[b].y of
// item work[b].x with that item's P segments; blockDim = 32 x the largest P.
template <typename T, int MAXM, bool ADJ>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_zsolve_w_grp(const ZArgs<T>* __restrict__ items,
                                                                             const int2* __restrict__ work) {
    __shared__ __align__(16) ZArgs<T> sa;
    const int2 wk = work[blockIdx.x];
    {
        const int* src = reinterpret_cast<const int*>(items + wk.x);
        int* d = reinterpret_cast<int*>(&sa);
        for (int i = threadIdx.x; i < (int)(sizeof(ZArgs<T>) / 4); i += blockDim.x) d[i] = src[i];
    }
    __syncthreads();
    zw_kernel_body<T, MAXM, false, ADJ>(sa, wk.y, sa.P, blockDim.x / 32);
}

// Shared memory of one tile of a line of nz rows in P segments, chain slots
// for Pb warps.
template <typename T>
size_t zsolve_w_smem_pb(int nz, int P, int Pb) {
    const int m = (nz + P - 1) / P;
    return ((size_t)P * m * 32 + 6 * (size_t)Pb * 32 + 8 * (size_t)nz) * sizeof(T);
}

// Persistent variant (16-byte aligned rows only): each CTA walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... with two tile buffers, so the
// cp.async load of the next tile is in flight while the current one is
// solved and stored.  One CTA per SM.
template <typename T, int MAXM, bool FULL, bool ADJ>
__global__ void __launch_bounds__(512, 1) k_zsolve_wp(ZArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TM = 32;
    const int nz = a.nz;
    const int P = blockDim.x / 32;
    const int m = (nz + P - 1) / P;
    const long nmodes = (long)a.nx * a.ny;
    const long tsz = (long)P * m * TM;                 // elements of one tile buffer
    T* tiles = reinterpret_cast<T*>(smem_raw);         // 2 x [P*m][32]
    T* ch = tiles + 2 * tsz;
    ZwTables<T> tb(ch + 6 * P * TM, nz);
    const T* __restrict__ in = a.src ? a.src : a.data;
    const long ntiles = (nmodes + TM - 1) / TM;
    tb.fill(a);
    long t = blockIdx.x;
    if (t < ntiles) zw_load_async<T>(tiles, in, nmodes, t * TM, (int)min((long)TM, nmodes - t * TM), nz);
    cp_async_commit();
    for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
        T* cur = tiles + (it & 1) * tsz;
        const long tn = t + gridDim.x;
        if (tn < ntiles)
            zw_load_async<T>(tiles + ((it + 1) & 1) * tsz, in, nmodes, tn * TM, (int)min((long)TM, nmodes - tn * TM), nz);
        cp_async_commit();
        cp_async_wait_prev();                          // the current tile's group has landed
        __syncthreads();
        const long q0 = t * TM;
        const int w = (int)min((long)TM, nmodes - q0);
        zw_solve_tile<T, MAXM, FULL, ADJ>(a, cur, ch, tb, q0, w, P, P);
        zw_store<T>(a.data, cur, nmodes, q0, w, nz);
        __syncthreads();                               // the buffer is free for the load after next
    }
    cp_async_wait_none();
}

template <typename T>
size_t zsolve_w_smem(int nz, int P) {
    const int m = (nz + P - 1) / P;
    return ((size_t)P * m * 32 + 6 * (size_t)P * 32 + 8 * (size_t)nz) * sizeof(T);
}

// Shared memory of the persistent variant: two tile buffers.
template <typename T>
size_t zsolve_wp_smem(int nz, int P) {
    const int m = (nz + P - 1) / P;
    return zsolve_w_smem<T>(nz, P) + (size_t)P * m * 32 * sizeof(T);
}

// Streaming-multiprocessor count of the current device (cached).
static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
        if (n <= 0) { cudaGetLastError(); return 1; }
    }
    return n;
}

template <typename T, int MAXM>
static cudaError_t launch_zsolve_w(const ZArgs<T>& a, cudaStream_t st) {
    const bool full = a.nz == a.P * MAXM;
    const long nmodes = (long)a.nx * a.ny;
    const long ntiles = (nmodes + 31) / 32;
    const int nsm = sm_count();
    // persistent double-buffered kernel when every SM gets several tiles and
    // two tile buffers fit
    const size_t smp = zsolve_wp_smem<T>(a.nz, a.P);
    if (a.bulk && a.persist != 0 && ntiles >= 8L * nsm && smp <= 227 * 1024) {
        auto kern = full ? (a.adjoint ? k_zsolve_wp<T, MAXM, true, true> : k_zsolve_wp<T, MAXM, true, false>)
                         : (a.adjoint ? k_zsolve_wp<T, MAXM, false, true> : k_zsolve_wp<T, MAXM, false, false>);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * a.P, smp) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const long slots = (long)nsm * per_sm;
        const unsigned grid = (unsigned)(ntiles < slots ? ntiles : slots);
        kern<<<grid, 32 * a.P, smp, st>>>(a);
        return cudaGetLastError();
    }
    const size_t sm = zsolve_w_smem<T>(a.nz, a.P);
    auto kern = full ? (a.adjoint ? k_zsolve_w<T, MAXM, true, true> : k_zsolve_w<T, MAXM, true, false>)
                     : (a.adjoint ? k_zsolve_w<T, MAXM, false, true> : k_zsolve_w<T, MAXM, false, false>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<(unsigned)ntiles, 32 * a.P, sm, st>>>(a);
    return cudaGetLastError();
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
    if (a.warp_mode) {
        switch (a.maxm) {
            case 16: return launch_zsolve_w<T, 16>(a, st);
            case 32: return launch_zsolve_w<T, 32>(a, st);
            case 64: return launch_zsolve_w<T, 64>(a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.maxm > 0) {
        const int key = a.P * 1000 + a.maxm;
        switch (key) {
            case 1016: return launch_zsolve_reg<T, 1, 16>(a, st);
            case 2016: return launch_zsolve_reg<T, 2, 16>(a, st);
            case 2032: return launch_zsolve_reg<T, 2, 32>(a, st);
            case 4016: return launch_zsolve_reg<T, 4, 16>(a, st);
            case 4032: return launch_zsolve_reg<T, 4, 32>(a, st);
            case 8016: return launch_zsolve_reg<T, 8, 16>(a, st);
            case 8032: return launch_zsolve_reg<T, 8, 32>(a, st);
            case 8064: return launch_zsolve_reg<T, 8, 64>(a, st);
            case 16032: return launch_zsolve_reg<T, 16, 32>(a, st);
            case 16064: return launch_zsolve_reg<T, 16, 64>(a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.P) {
        case 1: return launch_zsolve_p<T, 1>(a, st);
        case 2: return launch_zsolve_p<T, 2>(a, st);
        case 4: return launch_zsolve_p<T, 4>(a, st);
        case 8: return launch_zsolve_p<T, 8>(a, st);
        default: return launch_zsolve_p<T, 16>(a, st);
    }
}

}  // namespace cales

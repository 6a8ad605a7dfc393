// Transform kernels of the two uniform directions (eigenfunction expansion,
// Sec. 2.2), as templates: LS > 0 and KS >= 0 give the compile-time-size and
// compile-time-kind variants, LS = 0, KS = -1 the run-time ones.
//
// Row kernels (x): a CTA moves `rpc` consecutive rows (contiguous in memory)
// with one TMA bulk copy each way, packs them into complex pairs in shared
// memory, runs the Stockham passes and the post-processing, and writes the
// rows back.  The paper's pencil transposes (Sec. 3.1) are not needed: the
// column kernels (y) stage a tile of TX consecutive columns x all ny rows of
// one z-plane through shared memory with 16-byte cp.async copies, so every
// global access is a contiguous run of TX elements while the FFT runs along y
// inside shared memory.  Twiddles are staged in shared memory; every division
// by a run-time size is a multiply-high by a precomputed magic.
#pragma once
#include "kernels.cuh"

#include <type_traits>

namespace cales {

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// x / D for a compile-time D > 0, else the multiply-high magic of the table
template <int D> __device__ __forceinline__ int sdiv(int x, unsigned mag) {
    return D > 0 ? (int)((unsigned)x / (unsigned)(D > 0 ? D : 1)) : (int)fdivu((unsigned)x, mag);
}

// Number of table entries staged in shared memory: the per-pass twiddles
// (twlen), the post-processing factors W_n^m (L + 1) and, for the cosine and
// sine kinds, exp(-i pi m/(2n)) (L + 1).
__host__ __device__ __forceinline__ int table_len(int twlen, int L, int kind) {
    return twlen + L + 1 + (kind != KIND_P ? L + 1 : 0);
}

// Shared-memory layout of the row kernels: [mbarrier 16 B | b0 | b1 | tw | extra];
// b0 and b1 hold a multiple of 16 complex elements (swizzle blocks).
template <typename T> struct RowLayout {
    size_t b0, b1, tw, extra, total;
    __host__ __device__ RowLayout(int rpc, int L, int n, int kind, int twlen, size_t extra_per_elem) {
        const size_t C = sizeof(cpx<T>);
        const size_t nel = ((size_t)rpc * L + 15) & ~size_t(15);
        b0 = 16;
        b1 = al16(b0 + nel * C);
        tw = al16(b1 + nel * C);
        extra = al16(tw + (size_t)table_len(twlen, L, kind) * C);
        total = al16(extra + (size_t)rpc * n * extra_per_elem);
    }
};

// The per-pass twiddles (twlen), then the post-processing tables W_n^m and
// (cosine and sine kinds) exp(-i pi m/(2n)) (L + 1 each), staged
// contiguously in shared memory.
template <typename T>
__device__ __forceinline__ void stage_twiddles(cpx<T>* tw_s, const DirTab<T>& t) {
    const int L = t.L, tl = t.twlen;
    for (int i = threadIdx.x; i < tl; i += blockDim.x) tw_s[i] = t.tw[i];
    if (t.kind != KIND_P) {
        for (int i = threadIdx.x; i <= L; i += blockDim.x) {
            tw_s[tl + i] = t.post[i];
            tw_s[tl + L + 1 + i] = t.mak[i];
        }
    } else {
        for (int i = threadIdx.x; i <= L; i += blockDim.x) tw_s[tl + i] = t.post[i];
    }
}

// ---------------------------------------------------------------------------
// x direction
// ---------------------------------------------------------------------------
template <typename T, typename TIn, int LS = 0, int KS = -1>
__device__ __forceinline__ void rows_forward_body(const RowArgs<T>& a, const int bx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = LS ? 2 * LS : t.n, L = LS ? LS : t.L;
    const int kind = KS >= 0 ? KS : t.kind;
    const int nrad = LS ? sf_nrad(LS) : t.nrad;
    const long row0 = (long)bx * a.rpc;
    const int nr = (int)min((long)a.rpc, a.nrows - row0);
    constexpr bool RUP = std::is_same<TIn, RUIn>::value;
    using TLd = typename std::conditional<RUP, T, TIn>::type;     // element type of `in`
    const TLd* __restrict__ in = reinterpret_cast<const TLd*>(a.in) + row0 * n;
    T* __restrict__ out = reinterpret_cast<T*>(a.out) + row0 * n;
    const T sc = T(a.in_scale);
    const int tid = threadIdx.x;
    if (!RUP && n == 1) {
        for (int e = tid; e < nr; e += blockDim.x) out[e] = T(in[e]) * sc;
        return;
    }
    // FP64 input of an FP32 solve is read by the first Stockham pass straight
    // from global memory (prefetched into L2 while the tables are staged);
    // input of the compute type arrives by one TMA bulk copy into b0.
    constexpr bool IN64 = sizeof(TIn) == 8 && sizeof(T) == 4;
    const RowLayout<T> lay(a.rpc, L, n, kind, t.twlen, 0);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw + lay.b0);
    cpx<T>* b1 = reinterpret_cast<cpx<T>*>(smem_raw + lay.b1);
    cpx<T>* tw_s = reinterpret_cast<cpx<T>*>(smem_raw + lay.tw);
    const cpx<T>* pst = tw_s + t.twlen;
    const cpx<T>* mkt = tw_s + t.twlen + L + 1;
    const int tot = nr * n;
    if constexpr (RUP) {
        // the fused residual update: the CTA's rows formed in b0 (natural
        // order), as the bulk copy of the standalone transform would leave them
        if constexpr (sizeof(T) == 4) {
            float* xs = reinterpret_cast<float*>(b0);
            const ResidUpdArgs& u = a.ru;
            // L2 prefetch of the rows the update reads: r and the correction
            // at the CTA's rows, the correction one row before and after
            // (y neighbours) and one plane below and above (z neighbours)
            if (tid < 4) {
                const long plane = (long)n * u.ny, N = plane * u.nz;
                long lo = row0 * n, hi = lo + (long)nr * n;
                const float* base = tid == 0 ? u.r : u.d;
                if (tid == 1) { lo -= n; hi += n; }
                if (tid == 2) { lo -= plane; hi -= plane; }
                if (tid == 3) { lo += plane; hi += plane; }
                lo = max(lo, 0L);
                hi = min(hi, N);
                if (hi > lo) bulk_prefetch_l2(base + lo, (uint32_t)((hi - lo) * sizeof(float)));
            }
            const float dshift = u.acc ? (float)(u.acc[0] - u.acc[2]) : 0.f;
            const int ng = n / 4, tg = nr * ng;
            const unsigned gmag = div_magic((unsigned)ng), ymag = div_magic((unsigned)u.ny);
            // two groups per thread in flight
            for (int e0 = tid; e0 < tg; e0 += 2 * blockDim.x) {
                float v[2][4];
                int off[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = e0 + h * blockDim.x;
                    off[h] = -1;
                    if (e < tg) {
                        const int rr = (int)fdivu((unsigned)e, gmag), g = e - rr * ng;
                        const unsigned R = (unsigned)(row0 + rr);
                        const int k = (int)fdivu(R, ymag), j = (int)R - k * u.ny;
                        resupd_group<4>(u, ru_plane(u, k), 4 * g, j, k, dshift, v[h]);
                        off[h] = rr * n + 4 * g;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (off[h] >= 0)
                        *reinterpret_cast<float4*>(xs + off[h]) = make_float4(v[h][0], v[h][1], v[h][2], v[h][3]);
            }
        }
        stage_twiddles(tw_s, t);
        __syncthreads();
    } else if (IN64) {
        if (tid == 0 && a.bulk) bulk_prefetch_l2(in, (uint32_t)(tot * sizeof(TIn)));
        stage_twiddles(tw_s, t);
        __syncthreads();
    } else if (a.bulk) {
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (uint32_t)(tot * sizeof(TIn)));
            bulk_g2s(b0, in, (uint32_t)(tot * sizeof(TIn)), bar);
        }
        stage_twiddles(tw_s, t);
        __syncthreads();
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, 0);
            return;
        }
    } else {
        TIn* stage = reinterpret_cast<TIn*>(b0);
        for (int e = tid; e < tot; e += blockDim.x) stage[e] = in[e];
        stage_twiddles(tw_s, t);
        __syncthreads();
    }
    NatIO<T> nat{reinterpret_cast<const T*>(b0), nullptr, n, 1, reinterpret_cast<const double*>(in)};
    if (KS < 0 && kind >= KIND_DF) {
        // DST-I / DCT-IV / DST-IV: explicit packing with the pre-twiddles,
        // FFT, post-processing (natural-order input staged in b0)
        T* xs = reinterpret_cast<T*>(b0);
        if (IN64) {
            for (int e = tid; e < tot; e += blockDim.x) xs[e] = T(trunc_double_int(double(in[e])));
            __syncthreads();
        }
        for (int idx = tid; idx < nr * L; idx += blockDim.x) {
            const int r = (int)fdivu((unsigned)idx, t.lmag), j = idx - r * L;
            b1[r * L + j] = pack_new<T>(kind, n, xs + r * n, 1, mkt, j, sc);
        }
        __syncthreads();
        cpx<T>* Zn = fft_lines<T, false, 0, false, false, LS, KS>(b1, b0, t, nr, L, 1, tw_s, nat);
        T* obn = reinterpret_cast<T*>(Zn == b0 ? b1 : b0);
        const int kb = kind == KIND_DF ? 1 : 0, nk = kind == KIND_DF ? n : L;
        const unsigned kmag = kind == KIND_DF ? t.nmag : t.lmag;
        for (int idx = tid; idx < nr * nk; idx += blockDim.x) {
            const int r = (int)fdivu((unsigned)idx, kmag), k = idx - r * nk + kb;
            post_new<T>(kind, n, L, Zn + r * L, 1, obn + r * n, 1, pst, k);
        }
        if (a.bulk) {
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                bulk_s2g(out, obn, (uint32_t)(tot * sizeof(T)));
                bulk_commit();
                bulk_wait_read_all();
            }
        } else {
            __syncthreads();
            for (int e = tid; e < tot; e += blockDim.x) out[e] = obn[e];
        }
        return;
    }
    // (the fused FP64 read uses 16-byte loads: only with aligned rows)
    const bool fused = nrad > 0 && sc == T(1) && (!IN64 || a.bulk);
    if (!fused) {
        // explicit packing (n == 2, or a scaled input)
        T* r0 = reinterpret_cast<T*>(IN64 ? b0 : b1);
        const T* s32 = reinterpret_cast<const T*>(b0);
        for (int e = tid; e < tot; e += blockDim.x) {
            const int r = sdiv<LS ? 2 * LS : 0>(e, t.nmag), s = e - r * n;
            T v;
            if (IN64) v = T(trunc_double_int(double(in[e])));
            else v = s32[e];
            r0[r * n + pack_index(kind, n, s)] = v * sc * pack_sign<T>(kind, s);
        }
        __syncthreads();
    }
    cpx<T>* Z;
    if (fused && IN64) Z = fft_lines<T, false, 0, true, false, LS, KS, true>(b0, b1, t, nr, L, 1, tw_s, nat);
    else if (fused && kind == KIND_P) Z = fft_lines<T, false, 0, false, false, LS, KS>(b0, b1, t, nr, L, 1, tw_s, nat);
    else if (fused) Z = fft_lines<T, false, 0, true, false, LS, KS>(b0, b1, t, nr, L, 1, tw_s, nat);
    else if (!IN64) Z = fft_lines<T, false, 0, false, false, LS, KS>(b1, b0, t, nr, L, 1, tw_s, nat);
    else Z = fft_lines<T, false, 0, false, false, LS, KS>(b0, b1, t, nr, L, 1, tw_s, nat);
    T* ob = reinterpret_cast<T*>(Z == b0 ? b1 : b0);
    const int half = L / 2 + 1;
    const int npost = nr * half;
    for (int idx = tid; idx < npost; idx += blockDim.x) {
        const int r = sdiv<LS ? LS / 2 + 1 : 0>(idx, t.hmag), m = idx - r * half;
        post_forward_pair<T, LS, KS>(Z + r * L, 1, ob + r * n, 1, t, pst, mkt, m);
    }
    if (a.bulk) {
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(out, ob, (uint32_t)(tot * sizeof(T)));
            bulk_commit();
            bulk_wait_read_all();
        }
    } else {
        __syncthreads();
        for (int e = tid; e < tot; e += blockDim.x) out[e] = ob[e];
    }
}

template <typename T, typename TIn, int LS = 0, int KS = -1>
__global__ void __launch_bounds__(256) k_rows_forward(const __grid_constant__ RowArgs<T> a) {
    rows_forward_body<T, TIn, LS, KS>(a, blockIdx.x);
}

// pair + (v - shift) as a normalised pair; without a shift (every sweep but
// the last of a singular problem) the single float v joins by one TwoSum.
__device__ __forceinline__ ff pair_update(float2 pr, float v, ff shift, bool has_shift) {
    if (!has_shift) {
        const ff sm = two_sum(pr.x, v);
        return fast_two_sum(sm.hi, sm.lo + pr.y);
    }
    return ff_add(ff{pr.x, pr.y}, ff_sub(ff{v, 0.f}, shift));
}

// One inverse-x result into an 8-byte slot according to the output mode.
template <typename T, int MODE>
__device__ __forceinline__ void store8(unsigned char* slot, T v, ff shift) {
    if (MODE == OUT_F64) {
        *reinterpret_cast<double*>(slot) = double(v);
    } else if (MODE == OUT_FF_INIT) {
        *reinterpret_cast<float2*>(slot) = make_float2(float(v), 0.f);
    } else {
        const float2 pr = *reinterpret_cast<const float2*>(slot);
        const ff x = pair_update(pr, float(v), shift, shift.hi != 0.f || shift.lo != 0.f);
        if (MODE == OUT_FF_ACC) *reinterpret_cast<float2*>(slot) = make_float2(x.hi, x.lo);
        else *reinterpret_cast<double*>(slot) = ff_to_double_bits(x);
    }
}

// The 8-byte results of a CTA's rows (row0 .. of row length n): pair updates
// load U pairs per thread before computing any (more loads in flight per
// thread).  OUT_FF_ACC_D also stores each correction as FP32 to a.dout and,
// with a.gacc, adds the dzf-weighted sum of the updated pairs to a.gacc[0].
template <typename T, int MODE>
__device__ __forceinline__ void store8_rows(unsigned char* outp, const T* vals, int tot, ff shift, const RowArgs<T>& a,
                                            long row0, int n) {
    if (MODE == OUT_FF_ACC_D) {
        // row by row, so the gauge sum of a row takes its plane's weight once
        constexpr int U = 4;
        const int bd = blockDim.x;
        float2* po = reinterpret_cast<float2*>(outp);
        float* dout = reinterpret_cast<float*>(a.dout) + row0 * n;
        const bool gauge = a.gacc != nullptr;
        const int nrow = tot / n;
        double dacc = 0.0;
        for (int r = 0; r < nrow; ++r) {
            float ghi = 0.f, glo = 0.f;
            const int rb = r * n;
            for (int s0 = threadIdx.x; s0 < n; s0 += U * bd) {
                float2 pr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int sx = s0 + u * bd;
                    if (sx < n) pr[u] = po[rb + sx];
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int sx = s0 + u * bd;
                    if (sx < n) {
                        const float v = float(vals[rb + sx]);
                        const ff x = pair_update(pr[u], v, shift, false);
                        po[rb + sx] = make_float2(x.hi, x.lo);
                        dout[rb + sx] = v;
                        if (gauge) {
                            const ff g = two_sum(ghi, x.hi);
                            ghi = g.hi;
                            glo += g.lo + x.lo;
                        }
                    }
                }
            }
            if (gauge) dacc += ((double)ghi + (double)glo) * a.gw[(int)fdivu((unsigned)(row0 + r), a.nymag)];
        }
        if (gauge) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dacc += __shfl_down_sync(0xffffffffu, dacc, o);
            __shared__ double red[32];
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) red[wid] = dacc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += red[w2];
                atomicAdd(a.gacc, t);
            }
        }
    } else if (MODE == OUT_FF_ACC || MODE == OUT_FF_FINAL) {
        constexpr int U = 4;
        const int bd = blockDim.x;
        const bool has_shift = shift.hi != 0.f || shift.lo != 0.f;     // uniform per CTA
        float2* po = reinterpret_cast<float2*>(outp);
        for (int e0 = threadIdx.x; e0 < tot; e0 += U * bd) {
            float2 pr[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * bd;
                if (e < tot) pr[u] = po[e];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * bd;
                if (e < tot) {
                    const ff x = pair_update(pr[u], float(vals[e]), shift, has_shift);
                    if (MODE == OUT_FF_ACC) po[e] = make_float2(x.hi, x.lo);
                    else reinterpret_cast<double*>(outp)[e] = ff_to_double_bits(x);
                }
            }
        }
    } else {
        for (int e = threadIdx.x; e < tot; e += blockDim.x) store8<T, MODE>(outp + (long)e * 8, vals[e], shift);
    }
}


// Inverse along x; the output mode decides how the result is stored.
template <typename T, int MODE, int LS = 0, int KS = -1>
__device__ __forceinline__ void rows_inverse_body(const RowArgs<T>& a, const int bx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = LS ? 2 * LS : t.n, L = LS ? LS : t.L;
    const int kind = KS >= 0 ? KS : t.kind;
    const int nrad = LS ? sf_nrad(LS) : t.nrad;
    const long row0 = (long)bx * a.rpc;
    const int nr = (int)min((long)a.rpc, a.nrows - row0);
    const T* __restrict__ in = reinterpret_cast<const T*>(a.in) + row0 * n;
    constexpr int OSZ = MODE == OUT_T ? (int)sizeof(T) : 8;
    unsigned char* outp = reinterpret_cast<unsigned char*>(a.out) + row0 * n * OSZ;
    ff shift{0.f, 0.f};
    if (MODE >= OUT_FF_ACC && a.shift_acc) shift = ff_from_double(a.shift_acc[0] * a.shift_scale);
    const int tot = nr * n;
    const int tid = threadIdx.x;
    if (n == 1) {
        if (MODE == OUT_T) {
            for (int e = tid; e < tot; e += blockDim.x) reinterpret_cast<T*>(outp)[e] = in[e];
        } else {
            store8_rows<T, MODE>(outp, in, tot, shift, a, row0, n);
        }
        return;
    }
    // Shared memory holds the spectra and the FFT buffers only; the 8-byte
    // results (FP64 or double-float pairs) are read-modified-written in
    // global memory by coalesced accesses, the pairs to update having been
    // prefetched into L2 at the start so they arrive during the FFT.
    const RowLayout<T> lay(a.rpc, L, n, kind, t.twlen, 0);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw + lay.b0);
    cpx<T>* b1 = reinterpret_cast<cpx<T>*>(smem_raw + lay.b1);
    cpx<T>* tw_s = reinterpret_cast<cpx<T>*>(smem_raw + lay.tw);
    T* x0 = reinterpret_cast<T*>(b0);
    constexpr bool LOAD_OUT = MODE == OUT_FF_ACC || MODE == OUT_FF_FINAL || MODE == OUT_FF_ACC_D;
    if (a.bulk) {
        if (tid == 0) {
            if (LOAD_OUT) bulk_prefetch_l2(outp, (uint32_t)(tot * 8));
            mbar_init(bar, 1);
            const uint32_t b_in = (uint32_t)(tot * sizeof(T));
            mbar_expect_tx(bar, b_in);
            bulk_g2s(x0, in, b_in, bar);
        }
        stage_twiddles(tw_s, t);
        __syncthreads();
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, 0);
            return;
        }
    } else {
        for (int e = tid; e < tot; e += blockDim.x) x0[e] = in[e];
        stage_twiddles(tw_s, t);
        __syncthreads();
    }
    const cpx<T>* pst = tw_s + t.twlen;
    const cpx<T>* mkt = tw_s + t.twlen + L + 1;
    T* ob;
    if (KS < 0 && kind >= KIND_DF) {
        // DST-I / DCT-IV / DST-IV are their own inverses up to a constant:
        // the forward steps, scaled so that inverse(forward(x)) = n x
        const T isc = kind == KIND_DF ? T(2.0 * n / (n + 1)) : T(2);
        for (int idx = tid; idx < nr * L; idx += blockDim.x) {
            const int r = (int)fdivu((unsigned)idx, t.lmag), j = idx - r * L;
            b1[r * L + j] = pack_new<T>(kind, n, x0 + r * n, 1, mkt, j, isc);
        }
        __syncthreads();
        const NatIO<T> nat0{nullptr, nullptr, n, 1};
        cpx<T>* Zn = fft_lines<T, false, 0, false, false, LS, KS>(b1, b0, t, nr, L, 1, tw_s, nat0);
        T* natout = reinterpret_cast<T*>(Zn == b0 ? b1 : b0);
        const int kb = kind == KIND_DF ? 1 : 0, nk = kind == KIND_DF ? n : L;
        const unsigned kmag = kind == KIND_DF ? t.nmag : t.lmag;
        for (int idx = tid; idx < nr * nk; idx += blockDim.x) {
            const int r = (int)fdivu((unsigned)idx, kmag), k = idx - r * nk + kb;
            post_new<T>(kind, n, L, Zn + r * L, 1, natout + r * n, 1, pst, k);
        }
        __syncthreads();
        if (MODE != OUT_T) {
            store8_rows<T, MODE>(outp, natout, tot, shift, a, row0, n);
            return;
        }
        ob = natout;
    } else {
    const int half = L / 2 + 1;
    const int npre = nr * half;
    for (int idx = tid; idx < npre; idx += blockDim.x) {
        const int r = sdiv<LS ? LS / 2 + 1 : 0>(idx, t.hmag), m = idx - r * half;
        pre_inverse_pair<T, LS, KS>(x0 + r * n, 1, b1 + r * L, 1, t, pst, mkt, m);
    }
    __syncthreads();
    if (nrad > 0) {
        // the last pass unpacks straight into natural order (real rows); a
        // periodic row's packed pairs already are its natural order
        T* natout = reinterpret_cast<T*>((nrad & 1) ? b0 : b1);
        const NatIO<T> nat{nullptr, natout, n, 1};
        if (kind == KIND_P) fft_lines<T, true, 0, false, false, LS, KS>(b1, b0, t, nr, L, 1, tw_s, nat);
        else fft_lines<T, true, 0, false, true, LS, KS>(b1, b0, t, nr, L, 1, tw_s, nat);
        if (MODE != OUT_T) {
            store8_rows<T, MODE>(outp, natout, tot, shift, a, row0, n);
            return;
        }
        ob = natout;
    } else {
        const T* zr = reinterpret_cast<const T*>(b1);
        ob = reinterpret_cast<T*>(b0);
        for (int e = tid; e < tot; e += blockDim.x) {
            const int r = sdiv<LS ? 2 * LS : 0>(e, t.nmag), s2 = e - r * n;
            ob[e] = zr[r * n + pack_index(kind, n, s2)] * pack_sign<T>(kind, s2);
        }
        if (MODE != OUT_T) {
            __syncthreads();
            store8_rows<T, MODE>(outp, ob, tot, shift, a, row0, n);
            return;
        }
    }
    }
    if (a.bulk) {
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(outp, ob, (uint32_t)(tot * sizeof(T)));
            bulk_commit();
            bulk_wait_read_all();
        }
    } else {
        __syncthreads();
        for (int e = tid; e < tot; e += blockDim.x) reinterpret_cast<T*>(outp)[e] = ob[e];
    }
}

template <typename T, int MODE, int LS = 0, int KS = -1>
__global__ void __launch_bounds__(256) k_rows_inverse(const __grid_constant__ RowArgs<T> a) {
    rows_inverse_body<T, MODE, LS, KS>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// y direction: tiles of TX columns of one z-plane, in place.  With `bulk`, the
// tile moves by 16-byte cp.async copies (all in flight), else by plain loads.
// Shared memory: [16 B | b0 | b1 | tw].
// ---------------------------------------------------------------------------
template <typename T> __host__ __device__ __forceinline__ size_t col_smem(int TX, int L, int kind, int twlen) {
    return al16(16 + 2 * (size_t)TX * L * sizeof(cpx<T>)) + (size_t)table_len(twlen, L, kind) * sizeof(cpx<T>);
}

template <typename T, int TX, bool INV, int LS = 0, int KS = -1>
__device__ __forceinline__ void cols_body(const ColArgs<T>& a, const int bx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = LS ? 2 * LS : t.n, L = LS ? LS : t.L;     // n = ny
    const int kind = KS >= 0 ? KS : t.kind;
    const int nrad = LS ? sf_nrad(LS) : t.nrad;
    const int nx = a.nx;
    const int tiles_x = (nx + TX - 1) / TX;
    const int plane = bx / tiles_x;
    const int x0 = (bx - plane * tiles_x) * TX;
    const int wx = min(TX, nx - x0);
    const int tid = threadIdx.x;
    T* __restrict__ base = reinterpret_cast<T*>(a.data) + (long)plane * n * nx + x0;
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw + 16);
    cpx<T>* b1 = b0 + TX * L;
    cpx<T>* tw_s = reinterpret_cast<cpx<T>*>(smem_raw + al16(16 + 2 * (size_t)TX * L * sizeof(cpx<T>)));
    const int tot = n * TX;
    T* nat = reinterpret_cast<T*>(b0);                 // natural-order tile [ny][TX]
    const cpx<T>* pst = tw_s + t.twlen;
    const cpx<T>* mkt = tw_s + t.twlen + L + 1;
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int CPR = TX / EPC > 0 ? TX / EPC : 1;
    if (a.bulk) {
        for (int e = tid; e < n * CPR; e += blockDim.x) {
            const int s = e / CPR, c0 = (e - s * CPR) * EPC;
            cp_async16(nat + s * TX + c0, base + (long)s * nx + (c0 < wx ? c0 : 0), c0 < wx);
        }
        stage_twiddles(tw_s, t);
        cp_async_wait_all();
    } else {
        for (int e = tid; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            nat[e] = (c < wx) ? base[(long)s * nx + c] : T(0);
        }
        stage_twiddles(tw_s, t);
    }
    __syncthreads();
    T* ob;
    const int half = L / 2 + 1;
    if (KS < 0 && kind >= KIND_DF) {
        // DST-I / DCT-IV / DST-IV: explicit packing, forward FFT, post-processing;
        // the inverse is the same transform scaled so that inverse(forward(x)) = n x
        const T sc = INV ? (kind == KIND_DF ? T(2.0 * n / (n + 1)) : T(2)) : T(1);
        for (int idx = tid; idx < TX * L; idx += blockDim.x) {
            const int q = idx / TX, c = idx - q * TX;
            b1[q * TX + c] = pack_new<T>(kind, n, nat + c, TX, mkt, q, sc);
        }
        __syncthreads();
        const NatIO<T> nat0{nullptr, nullptr, 1, TX};
        cpx<T>* Zn = fft_lines<T, false, TX, false, false, LS, KS>(b1, b0, t, TX, 1, TX, tw_s, nat0);
        ob = reinterpret_cast<T*>(Zn == b0 ? b1 : b0);
        const int kb = kind == KIND_DF ? 1 : 0, nk = kind == KIND_DF ? n : L;
        for (int idx = tid; idx < nk * TX; idx += blockDim.x) {
            const int k = idx / TX, c = idx - k * TX;
            post_new<T>(kind, n, L, Zn + c, TX, ob + c, TX, pst, k + kb);
        }
    } else if (!INV) {
        cpx<T>* Z;
        if (nrad > 0) {
            const NatIO<T> natio{nat, nullptr, 1, TX};
            Z = fft_lines<T, false, TX, true, false, LS, KS>(b0, b1, t, TX, 1, TX, tw_s, natio);
        } else {
            T* r1 = reinterpret_cast<T*>(b1);
            for (int e = tid; e < tot; e += blockDim.x) {
                const int s = e / TX, c = e - s * TX;
                const int d = pack_index(kind, n, s);
                r1[((d >> 1) * TX + c) * 2 + (d & 1)] = nat[e] * pack_sign<T>(kind, s);
            }
            __syncthreads();
            Z = b1;
        }
        ob = reinterpret_cast<T*>(Z == b0 ? b1 : b0);
        const int npost = half * TX;
        for (int idx = tid; idx < npost; idx += blockDim.x) {
            const int m = idx / TX, c = idx - m * TX;
            post_forward_pair<T, LS, KS>(Z + c, TX, ob + c, TX, t, pst, mkt, m);
        }
    } else {
        const int npre = half * TX;
        for (int idx = tid; idx < npre; idx += blockDim.x) {
            const int m = idx / TX, c = idx - m * TX;
            pre_inverse_pair<T, LS, KS>(nat + c, TX, b1 + c, TX, t, pst, mkt, m);
        }
        __syncthreads();
        if (nrad > 0) {
            T* natout = reinterpret_cast<T*>((nrad & 1) ? b0 : b1);
            const NatIO<T> natio{nullptr, natout, 1, TX};
            fft_lines<T, true, TX, false, true, LS, KS>(b1, b0, t, TX, 1, TX, tw_s, natio);
            ob = natout;
        } else {
            const T* zr = reinterpret_cast<const T*>(b1);
            ob = reinterpret_cast<T*>(b0);
            for (int e = tid; e < tot; e += blockDim.x) {
                const int s = e / TX, c = e - s * TX;
                const int d = pack_index(kind, n, s);
                ob[e] = zr[((d >> 1) * TX + c) * 2 + (d & 1)] * pack_sign<T>(kind, s);
            }
        }
    }
    __syncthreads();
    if (a.bulk) {
        for (int e = tid; e < n * CPR; e += blockDim.x) {
            const int s = e / CPR, c0 = (e - s * CPR) * EPC;
            if (c0 < wx)
                *reinterpret_cast<float4*>(base + (long)s * nx + c0) = *reinterpret_cast<const float4*>(ob + s * TX + c0);
        }
    } else {
        for (int e = tid; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            if (c < wx) base[(long)s * nx + c] = ob[e];
        }
    }
}

template <typename T, int TX, bool INV, int LS = 0, int KS = -1>
__global__ void __launch_bounds__(256) k_cols(const __grid_constant__ ColArgs<T> a) {
    cols_body<T, TX, INV, LS, KS>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// y direction, one buffer: for L = 16 x LS2 (two passes, the second of radix
// LS2 <= 16) with TX = 16 columns and 256 threads, every pass has at most one
// butterfly per thread, so both passes run in place (read, barrier, write) in
// a single shared-memory buffer.  The natural-order column data never enters
// shared memory: the first forward pass packs it straight from global memory
// (rows prefetched into L2 at the start) and the post-processing writes the
// result rows to global memory; the inverse reads its input rows in the
// pre-processing and its last pass unpacks straight to global memory.
// Shared memory: [buffer L x 16 complex | tables] ~ 38 KB for L = 256.
// ---------------------------------------------------------------------------
template <int LS, int KS, bool INV>
__global__ void __launch_bounds__(256) k_cols_g(ColArgs<float> a) {
    constexpr int TX = 16, R1 = 16, R2 = LS / 16, NB1 = LS / R1, NB2 = LS / R2, n = 2 * LS;
    static_assert(sf_nrad(LS) == 2 && sf_radix(LS, 0) == 16 && NB1 * TX <= 256 && NB2 * TX <= 256, "shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<float>& t = a.t;
    const int nx = a.nx;
    const int tiles_x = (nx + TX - 1) / TX;
    const int plane = blockIdx.x / tiles_x;
    const int x0 = (blockIdx.x - plane * tiles_x) * TX;
    const int wx = min(TX, nx - x0);
    const int tid = threadIdx.x;
    float* __restrict__ base = reinterpret_cast<float*>(a.data) + (long)plane * n * nx + x0;
    cpx<float>* buf = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* tw_s = buf + LS * TX;
    const cpx<float>* pst = tw_s + t.twlen;
    const cpx<float>* mkt = tw_s + t.twlen + LS + 1;
    const int c = tid & (TX - 1);
    const bool live = c < wx;
    for (int s = tid; s < n; s += blockDim.x) prefetch_l2(base + (long)s * nx);
    stage_twiddles(tw_s, t);
    __syncthreads();
    const cpx<float>* tp2 = tw_s + t.twoff[1];
    if (!INV) {
        // pass 1 (radix 16, Ns = 1): pack the natural rows from global memory
        {
            const int j = tid / TX;
            cpx<float> v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int q = j + r * NB1;
                const int s0 = unpack_src(KS, n, 2 * q), s1 = unpack_src(KS, n, 2 * q + 1);
                v[r] = live ? mk(base[(long)s0 * nx + c] * pack_sign<float>(KS, s0),
                                 base[(long)s1 * nx + c] * pack_sign<float>(KS, s1))
                            : mk(0.f, 0.f);
            }
            Bfly<float, R1, false>::run(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) buf[(j * R1 + r) * TX + c] = v[r];
        }
        __syncthreads();
        // pass 2 (radix LS/16, Ns = 16) in place
        {
            const int j = tid / TX, k = j & 15;
            const bool act = j < NB2;
            cpx<float> v[R2];
            if (act) {
#pragma unroll
                for (int r = 0; r < R2; ++r) v[r] = buf[(j + r * NB2) * TX + c];
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], tp2[(r - 1) * 16 + k]);
                Bfly<float, R2, false>::run(v);
                const int b0 = (j - k) * R2 + k;
#pragma unroll
                for (int r = 0; r < R2; ++r) buf[(b0 + r * 16) * TX + c] = v[r];
            }
        }
        __syncthreads();
        // post-processing of the mode pairs straight to the global rows
        const int half = LS / 2 + 1;
        for (int idx = tid; idx < half * TX; idx += blockDim.x) {
            const int m = idx / TX, cc = idx - m * TX;
            if (cc < wx) post_forward_pair<float, LS, KS>(buf + cc, TX, base + cc, nx, t, pst, mkt, m);
        }
    } else {
        // pre-processing from the global rows
        const int half = LS / 2 + 1;
        for (int idx = tid; idx < half * TX; idx += blockDim.x) {
            const int m = idx / TX, cc = idx - m * TX;
            if (cc < wx) {
                pre_inverse_pair<float, LS, KS>(base + cc, nx, buf + cc, TX, t, pst, mkt, m);
            } else {
                buf[m * TX + cc] = mk(0.f, 0.f);
                if (LS - m != m && LS - m < LS) buf[(LS - m) * TX + cc] = mk(0.f, 0.f);
            }
        }
        __syncthreads();
        // pass 1 (radix 16, Ns = 1) in place
        {
            const int j = tid / TX;
            cpx<float> v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = buf[(j + r * NB1) * TX + c];
            __syncthreads();
            Bfly<float, R1, true>::run(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) buf[(j * R1 + r) * TX + c] = v[r];
        }
        __syncthreads();
        // pass 2 (radix LS/16, Ns = 16): unpack straight to the global rows
        {
            const int j = tid / TX, k = j & 15;
            if (j < NB2) {
                cpx<float> v[R2];
#pragma unroll
                for (int r = 0; r < R2; ++r) v[r] = buf[(j + r * NB2) * TX + c];
#pragma unroll
                for (int r = 1; r < R2; ++r) v[r] = cmulc(v[r], tp2[(r - 1) * 16 + k]);
                Bfly<float, R2, true>::run(v);
                const int b0 = (j - k) * R2 + k;
                if (live) {
#pragma unroll
                    for (int r = 0; r < R2; ++r) {
                        const int q = b0 + r * 16;
                        const int s0 = unpack_src(KS, n, 2 * q), s1 = unpack_src(KS, n, 2 * q + 1);
                        base[(long)s0 * nx + c] = v[r].x * pack_sign<float>(KS, s0);
                        base[(long)s1 * nx + c] = v[r].y * pack_sign<float>(KS, s1);
                    }
                }
            }
        }
    }
}

template <int LS, int KS>
cudaError_t launch_cols_g(const ColArgs<float>& a, bool inverse, cudaStream_t st) {
    const size_t sm = (size_t)LS * 16 * sizeof(cpx<float>) + (size_t)table_len(a.t.twlen, LS, KS) * sizeof(cpx<float>);
    const unsigned grid = (unsigned)(a.nplanes * ((a.nx + 15) / 16));
    auto kern = inverse ? k_cols_g<LS, KS, true> : k_cols_g<LS, KS, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, 256, sm, st>>>(a);
    return cudaGetLastError();
}

// The compile-time-size kernels assume the plan factorised L as sf_radix does.
template <typename T> inline bool radices_match(const DirTab<T>& t, int L) {
    if (t.L != L || t.nrad != sf_nrad(L)) return false;
    for (int p = 0; p < t.nrad; ++p)
        if (t.radix[p] != sf_radix(L, p)) return false;
    return true;
}

// ---------------------------------------------------------------------------
// launchers of one variant
// ---------------------------------------------------------------------------
template <typename T, typename TIn, int LS, int KS>
cudaError_t launch_rows_forward_v(const RowArgs<T>& a, cudaStream_t st) {
    const RowLayout<T> lay(a.rpc, a.t.L > 0 ? a.t.L : 1, a.t.n, a.t.kind, a.t.twlen, 0);
    auto kern = k_rows_forward<T, TIn, LS, KS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    const unsigned grid = (unsigned)((a.nrows + a.rpc - 1) / a.rpc);
    kern<<<grid, 256, lay.total, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int MODE, int LS, int KS>
cudaError_t launch_rows_inverse_v(const RowArgs<T>& a, cudaStream_t st) {
    const RowLayout<T> lay(a.rpc, a.t.L > 0 ? a.t.L : 1, a.t.n, a.t.kind, a.t.twlen, 0);
    auto kern = k_rows_inverse<T, MODE, LS, KS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    const unsigned grid = (unsigned)((a.nrows + a.rpc - 1) / a.rpc);
    kern<<<grid, 256, lay.total, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int TX, int LS, int KS>
cudaError_t launch_cols_v(const ColArgs<T>& a, bool inverse, cudaStream_t st) {
    const size_t sm = col_smem<T>(TX, a.t.L, a.t.kind, a.t.twlen);
    const unsigned grid = (unsigned)(a.nplanes * ((a.nx + TX - 1) / TX));
    auto kern = inverse ? k_cols<T, TX, true, LS, KS> : k_cols<T, TX, false, LS, KS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, 256, sm, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Grouped launches: one launch covers the same stage of many solves.  CTA b
// takes work[b] = (item, block of that item) and runs the item's kernel body
// on its argument block, copied into shared memory first.  Dynamic shared
// memory is the largest any item needs.
// ---------------------------------------------------------------------------
template <typename A>
__device__ __forceinline__ int load_item_args(A& dst, const A* __restrict__ items, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    const int* src = reinterpret_cast<const int*>(items + w.x);
    int* d = reinterpret_cast<int*>(&dst);
    static_assert(sizeof(A) % 4 == 0, "argument block of whole words");
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = src[i];
    __syncthreads();
    return w.y;
}

template <typename T, typename TIn>
__global__ void __launch_bounds__(256) k_rows_forward_grp(const RowArgs<T>* __restrict__ items, const int2* __restrict__ work) {
    __shared__ __align__(16) RowArgs<T> sa;
    const int bx = load_item_args(sa, items, work);
    rows_forward_body<T, TIn, 0, -1>(sa, bx);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_rows_inverse_grp(const RowArgs<T>* __restrict__ items, const int2* __restrict__ work) {
    __shared__ __align__(16) RowArgs<T> sa;
    const int bx = load_item_args(sa, items, work);
    rows_inverse_body<T, MODE, 0, -1>(sa, bx);
}

template <typename T, int TX, bool INV>
__global__ void __launch_bounds__(256) k_cols_grp(const ColArgs<T>* __restrict__ items, const int2* __restrict__ work) {
    __shared__ __align__(16) ColArgs<T> sa;
    const int bx = load_item_args(sa, items, work);
    cols_body<T, TX, INV, 0, -1>(sa, bx);
}

}  // namespace cales

// Transforms of the two uniform directions (eigenfunction expansion, Sec. 2.2).
//
// Row kernels (x): a CTA loads `rpc` consecutive rows (contiguous in memory,
// coalesced), packs them into complex pairs in shared memory, runs the
// Stockham passes and post-processing, and writes the rows back.  The paper's
// pencil transposes (Sec. 3.1) are not needed: the column kernels (y) stage a
// tile of TX consecutive columns x all ny rows of one z-plane through shared
// memory, so every global access is a contiguous run of TX elements while the
// FFT runs along y inside shared memory.
#include "kernels.cuh"

namespace cales {

// ---------------------------------------------------------------------------
// x direction
// ---------------------------------------------------------------------------
template <typename T, typename TIn>
__global__ void __launch_bounds__(256) k_rows_forward(RowArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = t.n, L = t.L;
    const long row0 = (long)blockIdx.x * a.rpc;
    const int nr = (int)min((long)a.rpc, a.nrows - row0);
    const TIn* __restrict__ in = reinterpret_cast<const TIn*>(a.in) + row0 * n;
    T* __restrict__ out = reinterpret_cast<T*>(a.out) + row0 * n;
    const T sc = T(a.in_scale);
    if (n == 1) {
        for (int e = threadIdx.x; e < nr; e += blockDim.x) out[e] = T(in[e]) * sc;
        return;
    }
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* b1 = b0 + a.rpc * L;
    T* r0 = reinterpret_cast<T*>(b0);
    const int tot = nr * n;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = e / n, s = e - r * n;
        const T v = T(in[e]) * sc * pack_sign<T>(t.kind, s);
        r0[r * n + pack_index(t.kind, n, s)] = v;   // pair (v[2j], v[2j+1]) = complex j
    }
    __syncthreads();
    cpx<T>* Z = fft_lines<T, false, false>(b0, b1, t, nr, L, 1);
    T* ob = reinterpret_cast<T*>(Z == b0 ? b1 : b0);
    const int npost = nr * (L + 1);
    for (int idx = threadIdx.x; idx < npost; idx += blockDim.x) {
        const int r = idx / (L + 1), m = idx - r * (L + 1);
        post_forward<T>(Z + r * L, 1, ob + r * n, 1, t, m);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tot; e += blockDim.x) out[e] = ob[e];
}

// Store of one inverse-x result according to the output mode.
template <typename T, int MODE>
__device__ __forceinline__ void store_out(void* outp, long e, T v, ff shift) {
    if (MODE == OUT_T) {
        reinterpret_cast<T*>(outp)[e] = v;
    } else if (MODE == OUT_F64) {
        reinterpret_cast<double*>(outp)[e] = double(v);
    } else if (MODE == OUT_FF_INIT) {
        reinterpret_cast<float2*>(outp)[e] = make_float2(float(v), 0.f);
    } else {
        const float2 pr = reinterpret_cast<const float2*>(outp)[e];
        ff x = ff_add(ff{pr.x, pr.y}, ff_sub(ff{float(v), 0.f}, shift));
        if (MODE == OUT_FF_ACC) reinterpret_cast<float2*>(outp)[e] = make_float2(x.hi, x.lo);
        else reinterpret_cast<double*>(outp)[e] = ff_to_double(x);
    }
}

// Inverse along x; the output mode decides how the result is stored.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_rows_inverse(RowArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = t.n, L = t.L;
    const long row0 = (long)blockIdx.x * a.rpc;
    const int nr = (int)min((long)a.rpc, a.nrows - row0);
    const T* __restrict__ in = reinterpret_cast<const T*>(a.in) + row0 * n;
    void* outp = reinterpret_cast<unsigned char*>(a.out) + row0 * n * (MODE == OUT_T ? sizeof(T) : 8);
    ff shift{0.f, 0.f};
    if (MODE >= OUT_FF_ACC && a.shift_acc) shift = ff_from_double(a.shift_acc[0] * a.shift_scale);
    const int tot = nr * n;
    if (n == 1) {
        for (int e = threadIdx.x; e < tot; e += blockDim.x) store_out<T, MODE>(outp, e, in[e], shift);
        return;
    }
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* b1 = b0 + a.rpc * L;
    T* x0 = reinterpret_cast<T*>(b0);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) x0[e] = in[e];
    __syncthreads();
    const int npre = nr * L;
    for (int idx = threadIdx.x; idx < npre; idx += blockDim.x) {
        const int r = idx / L, m = idx - r * L;
        b1[r * L + m] = pre_inverse<T>(x0 + r * n, 1, t, m);
    }
    __syncthreads();
    cpx<T>* z = fft_lines<T, true, false>(b1, b0, t, nr, L, 1);
    const T* zr = reinterpret_cast<const T*>(z);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = e / n, s = e - r * n;
        const T v = zr[r * n + pack_index(t.kind, n, s)] * pack_sign<T>(t.kind, s);
        store_out<T, MODE>(outp, e, v, shift);
    }
}

// ---------------------------------------------------------------------------
// y direction: tiles of TX columns of one z-plane, in place.
// ---------------------------------------------------------------------------
template <typename T, int TX, bool INV>
__global__ void __launch_bounds__(256) k_cols(ColArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DirTab<T>& t = a.t;
    const int n = t.n, L = t.L;     // n = ny
    const int nx = a.nx;
    const int tiles_x = (nx + TX - 1) / TX;
    const int plane = blockIdx.x / tiles_x;
    const int x0 = (blockIdx.x - plane * tiles_x) * TX;
    const int wx = min(TX, nx - x0);
    T* __restrict__ base = reinterpret_cast<T*>(a.data) + (long)plane * n * nx + x0;
    cpx<T>* b0 = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* b1 = b0 + TX * L;
    const int tot = n * TX;
    if (!INV) {
        T* r0 = reinterpret_cast<T*>(b0);
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            T v = (c < wx) ? base[(long)s * nx + c] : T(0);
            v *= pack_sign<T>(t.kind, s);
            const int d = pack_index(t.kind, n, s);
            r0[((d >> 1) * TX + c) * 2 + (d & 1)] = v;
        }
        __syncthreads();
        cpx<T>* Z = fft_lines<T, false, true>(b0, b1, t, TX, 1, TX);
        T* ob = reinterpret_cast<T*>(Z == b0 ? b1 : b0);
        const int npost = (L + 1) * TX;
        for (int idx = threadIdx.x; idx < npost; idx += blockDim.x) {
            const int m = idx / TX, c = idx - m * TX;
            post_forward<T>(Z + c, TX, ob + c, TX, t, m);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            if (c < wx) base[(long)s * nx + c] = ob[e];
        }
    } else {
        T* x0r = reinterpret_cast<T*>(b0);
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            x0r[e] = (c < wx) ? base[(long)s * nx + c] : T(0);
        }
        __syncthreads();
        const int npre = L * TX;
        for (int idx = threadIdx.x; idx < npre; idx += blockDim.x) {
            const int m = idx / TX, c = idx - m * TX;
            b1[m * TX + c] = pre_inverse<T>(x0r + c, TX, t, m);
        }
        __syncthreads();
        cpx<T>* z = fft_lines<T, true, true>(b1, b0, t, TX, 1, TX);
        const T* zr = reinterpret_cast<const T*>(z);
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int s = e / TX, c = e - s * TX;
            if (c < wx) {
                const int d = pack_index(t.kind, n, s);
                base[(long)s * nx + c] = zr[((d >> 1) * TX + c) * 2 + (d & 1)] * pack_sign<T>(t.kind, s);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T> static size_t row_smem(const DirTab<T>& t, int rpc) {
    return (size_t)2 * rpc * (t.L > 0 ? t.L : 1) * sizeof(cpx<T>);
}

template <typename T, typename TIn>
cudaError_t launch_rows_forward(const RowArgs<T>& a, cudaStream_t st) {
    const size_t sm = row_smem(a.t, a.rpc);
    auto kern = k_rows_forward<T, TIn>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned grid = (unsigned)((a.nrows + a.rpc - 1) / a.rpc);
    kern<<<grid, 256, sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_rows_inverse(const RowArgs<T>& a, cudaStream_t st) {
    const size_t sm = row_smem(a.t, a.rpc);
    auto kern = k_rows_inverse<T, MODE>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned grid = (unsigned)((a.nrows + a.rpc - 1) / a.rpc);
    kern<<<grid, 256, sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int TX>
static cudaError_t launch_cols_tx(const ColArgs<T>& a, bool inverse, cudaStream_t st) {
    const size_t sm = (size_t)2 * TX * a.t.L * sizeof(cpx<T>);
    const unsigned grid = (unsigned)(a.nplanes * ((a.nx + TX - 1) / TX));
    if (inverse) {
        auto kern = k_cols<T, TX, true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<grid, 256, sm, st>>>(a);
    } else {
        auto kern = k_cols<T, TX, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<grid, 256, sm, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cols(const ColArgs<T>& a, bool inverse, cudaStream_t st) {
    switch (a.tx) {
        case 32: return launch_cols_tx<T, 32>(a, inverse, st);
        case 16: return launch_cols_tx<T, 16>(a, inverse, st);
        case 8: return launch_cols_tx<T, 8>(a, inverse, st);
        default: return launch_cols_tx<T, 4>(a, inverse, st);
    }
}

template cudaError_t launch_rows_forward<double, double>(const RowArgs<double>&, cudaStream_t);
template cudaError_t launch_rows_forward<float, float>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_forward<float, double>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<double, OUT_T>(const RowArgs<double>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_T>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_F64>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_INIT>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_ACC>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_rows_inverse<float, OUT_FF_FINAL>(const RowArgs<float>&, cudaStream_t);
template cudaError_t launch_cols<double>(const ColArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_cols<float>(const ColArgs<float>&, bool, cudaStream_t);

}  // namespace cales

// Shared device definitions of the CaLES-style fast direct solver on sm_103a.
//
// Fields are [nz][ny][nx] with x fastest.  Every uniform direction is
// transformed by a real-to-real transform of length n:
//   P (periodic)  : real DFT in halfcomplex order (Re of mode m at m, Im at n-m)
//   N (Neumann)   : DCT-II        X_m = sum_i x_i cos(pi m (i+1/2)/n)
//   D (Dirichlet) : DST-II        X_m = sum_i x_i sin(pi m (i+1/2)/n), m = 1..n
// each computed from one complex FFT of length L = n/2 (real-input packing,
// Makhoul's even/odd reordering for the cosine/sine transforms).  This keeps
// the mode-space field real with exactly nx*ny*nz values, so the z tridiagonal
// systems of the eigenfunction expansion (Sec. 2.2) are real too.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cales {

// Transform kinds of a uniform direction: the kind of both sides (P, N, D;
// DF = node-centred unknowns between two zero boundary nodes), or mixed cell
// sides: ND = Neumann below, Dirichlet above; DN the reverse.
enum { KIND_P = 0, KIND_N = 1, KIND_D = 2, KIND_DF = 3, KIND_ND = 4, KIND_DN = 5 };
enum { ZBC_N = 1, ZBC_D = 2, ZBC_DF = 3 };
constexpr int MAX_RADICES = 16;

template <typename T> struct cpx { T x, y; };

template <typename T> __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
// Products with explicit rounding (no compiler contraction): every kernel
// variant that runs the same transform steps gets bit-identical results.
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return mk(fma_(a.x, b.x, -mul_(a.y, b.y)), fma_(a.x, b.y, mul_(a.y, b.x)));
}
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {   // a * conj(b)
    return mk(fma_(a.x, b.x, mul_(a.y, b.y)), fma_(a.y, b.x, -mul_(a.x, b.y)));
}
template <typename T> __device__ __forceinline__ cpx<T> conj_(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(mul_(a.x, s), mul_(a.y, s)); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> rot90(cpx<T> a) {
    return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Tables of one uniform direction (device pointers, built by the plan on the
// host in FP64 and rounded once for the FP32 copies).
// ---------------------------------------------------------------------------
template <typename T> struct DirTab {
    int n, kind, L, nrad;
    int radix[MAX_RADICES];
    int nsv[MAX_RADICES];          // sub-transform size Ns before pass p
    int tstep[MAX_RADICES];        // twiddle index step L / (Ns R) of pass p
    unsigned nbmag[MAX_RADICES];   // fast-division magic of L / R_p
    unsigned nsmag[MAX_RADICES];   // fast-division magic of Ns_p
    unsigned nmag, l1mag, lmag, hmag;   // magics of n, L + 1, L and L/2 + 1
    int twoff[MAX_RADICES];        // offset of pass p's twiddle block in tw
    int twlen;                     // total twiddle entries
    // Per-pass twiddles: pass p (Ns > 1) holds W_L^(r k tstep) at
    // tw[twoff[p] + (r - 1) Ns + k], r = 1..R-1, k = 0..Ns-1, so the threads
    // of a pass read consecutive entries (no shared-memory bank conflicts).
    const cpx<T>* tw;
    const cpx<T>* post;   // W_n^m = exp(-2 pi i m / n), m in [0, L]
    const cpx<T>* mak;    // exp(-i pi m / (2n)),        m in [0, L]
};

// q = n / d for the small operands of the transforms (n * d < 2^32): the
// magic is ceil(2^32 / d), 0 encoding d = 1 (Granlund-Montgomery style
// multiply-high; exact since the rounding error n * (magic*d - 2^32) / 2^32
// stays below 1/d).
__host__ __device__ __forceinline__ unsigned div_magic(unsigned d) {
    return d <= 1 ? 0u : (unsigned)((0x100000000ull + d - 1) / d);
}
__device__ __forceinline__ unsigned fdivu(unsigned n, unsigned mag) { return mag ? __umulhi(n, mag) : n; }

// ---------------------------------------------------------------------------
// Radix butterflies (forward: exp(-2 pi i / R); inverse: conjugate)
// ---------------------------------------------------------------------------
template <typename T, int R, bool INV> struct Bfly;

template <typename T, bool INV> struct Bfly<T, 2, INV> {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        cpx<T> a = v[0], b = v[1];
        v[0] = a + b; v[1] = a - b;
    }
};

template <typename T, bool INV> struct Bfly<T, 4, INV> {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        cpx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
        cpx<T> s13 = v[1] + v[3], d13 = rot90<T, INV>(v[1] - v[3]);
        v[0] = s02 + s13; v[2] = s02 - s13;
        v[1] = d02 + d13; v[3] = d02 - d13;
    }
};

template <typename T, bool INV> struct Bfly<T, 3, INV> {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        const T h = T(0.5), s3 = T(0.86602540378443864676372317075294);
        cpx<T> t = v[1] + v[2];
        cpx<T> d = scale(rot90<T, INV>(v[1] - v[2]), s3);
        cpx<T> m = v[0] - scale(t, h);
        v[0] = v[0] + t; v[1] = m + d; v[2] = m - d;
    }
};

template <typename T, bool INV> struct Bfly<T, 5, INV> {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi / 5)
        const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
        const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi / 5)
        const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi / 5)
        cpx<T> t1 = v[1] + v[4], t2 = v[2] + v[3];
        cpx<T> d1 = v[1] - v[4], d2 = v[2] - v[3];
        cpx<T> a = v[0] + scale(t1, c1) + scale(t2, c2);
        cpx<T> b = v[0] + scale(t1, c2) + scale(t2, c1);
        cpx<T> e = rot90<T, INV>(scale(d1, s1) + scale(d2, s2));
        cpx<T> f = rot90<T, INV>(scale(d1, s2) - scale(d2, s1));
        v[0] = v[0] + t1 + t2;
        v[1] = a + e; v[4] = a - e;
        v[2] = b + f; v[3] = b - f;
    }
};

// multiply by W16^e = exp(-2 pi i e / 16) (forward) or its conjugate (inverse)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> w16(cpx<T> a, T wr, T wi) {
    const T w2 = INV ? -wi : wi;
    return cmul(a, mk(wr, w2));
}

template <typename T, bool INV> struct Bfly<T, 16, INV> {
    // 16 = 4 x 4: radix-4 DFTs over n1 (input 4 n1 + n2), twiddles W16^(n2 k1),
    // radix-4 DFTs over n2 (output k1 + 4 k2)
    static __device__ __forceinline__ void run(cpx<T>* v) {
        const T c = T(0.92387953251128675612818318939679);    // cos(pi / 8)
        const T s = T(0.38268343236508977172845998403040);    // sin(pi / 8)
        const T r2 = T(0.70710678118654752440084436210485);
        cpx<T> a[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            cpx<T> t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
            Bfly<T, 4, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
        }
        a[1][1] = w16<T, INV>(a[1][1], c, -s);
        a[1][2] = w16<T, INV>(a[1][2], r2, -r2);
        a[1][3] = w16<T, INV>(a[1][3], s, -c);
        a[2][1] = w16<T, INV>(a[2][1], r2, -r2);
        a[2][2] = rot90<T, INV>(a[2][2]);
        a[2][3] = w16<T, INV>(a[2][3], -r2, -r2);
        a[3][1] = w16<T, INV>(a[3][1], s, -c);
        a[3][2] = w16<T, INV>(a[3][2], -r2, -r2);
        a[3][3] = w16<T, INV>(a[3][3], -c, s);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cpx<T> t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            Bfly<T, 4, INV>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
};

template <typename T, bool INV> struct Bfly<T, 8, INV> {
    static __device__ __forceinline__ void run(cpx<T>* v) {
        const T r2 = T(0.70710678118654752440084436210485);
        cpx<T> a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) { a[r] = v[r] + v[r + 4]; b[r] = v[r] - v[r + 4]; }
        // b[r] *= W8^r
        b[1] = INV ? mk(mul_(r2, b[1].x - b[1].y), mul_(r2, b[1].x + b[1].y))
                   : mk(mul_(r2, b[1].x + b[1].y), mul_(r2, b[1].y - b[1].x));
        b[2] = rot90<T, INV>(b[2]);
        b[3] = INV ? mk(mul_(-r2, b[3].x + b[3].y), mul_(r2, b[3].x - b[3].y))
                   : mk(mul_(r2, b[3].y - b[3].x), mul_(-r2, b[3].x + b[3].y));
        Bfly<T, 4, INV>::run(a);
        Bfly<T, 4, INV>::run(b);
        v[0] = a[0]; v[2] = a[1]; v[4] = a[2]; v[6] = a[3];
        v[1] = b[0]; v[3] = b[1]; v[5] = b[2]; v[7] = b[3];
    }
};

// Ghost multipliers of the low and high side of a direction (R2): the value
// beyond the boundary is mult * (the first / last unknown); periodic
// directions wrap instead (not used).
__host__ __device__ __forceinline__ float ghost_lo(int kind) {
    return (kind == KIND_N || kind == KIND_ND) ? 1.f : (kind == KIND_DF ? 0.f : -1.f);
}
__host__ __device__ __forceinline__ float ghost_hi(int kind) {
    return (kind == KIND_N || kind == KIND_DN) ? 1.f : (kind == KIND_DF ? 0.f : -1.f);
}

// ---------------------------------------------------------------------------
// Transforms of the kinds DF, ND and DN (explicit packing and post-processing
// around a forward complex FFT of length L; the same steps with a scale give
// the inverse, since each of these transforms is its own inverse up to a
// constant):
//   ND (DCT-IV, n even, L = n/2):
//     z_j = (x_{2j} + i x_{n-1-2j}) exp(-i pi (4j+1)/(4n)),  V = FFT_L(z),
//     w_k = V_k exp(-i pi k/n),  X_{2k} = Re w_k,  X_{n-1-2k} = -Im w_k.
//   DN (DST-IV): the same on the reversed input, output signs alternating:
//     X_{2k} = Re w_k, X_{n-1-2k} = Im w_k.
//   DF (DST-I, L = n+1): the real DFT of length 2(n+1) of the odd extension
//     y = (0, x_0 .. x_{n-1}, 0, -x_{n-1} .. -x_0), Y_k = -2i X_{k-1},
//     computed from the FFT of the pairs z_j = y_{2j} + i y_{2j+1}.
// Tables: `mak` holds the ND/DN pre-twiddles exp(-i pi (4j+1)/(4n)), `post`
// the post-twiddles exp(-i pi k/n) (ND/DN) or exp(-i pi k/(n+1)) (DF).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T df_ext(const T* x, int xes, int n, int t) {
    if (t == 0 || t == n + 1) return T(0);
    return t <= n ? x[(t - 1) * xes] : -x[(2 * n + 1 - t) * xes];
}

// Packed element j (of L) of one line x (element s at x[s * xes]), times sc.
template <typename T>
__device__ __forceinline__ cpx<T> pack_new(int kind, int n, const T* x, int xes, const cpx<T>* pre, int j, T sc) {
    if (kind == KIND_DF) return mk(df_ext(x, xes, n, 2 * j) * sc, df_ext(x, xes, n, 2 * j + 1) * sc);
    const T a = x[2 * j * xes], b = x[(n - 1 - 2 * j) * xes];
    const cpx<T> z = kind == KIND_ND ? mk(a, b) : mk(b, a);
    return scale(cmul(z, pre[j]), sc);
}

// Outputs of post-processing step k of one line: k in [0, L) for ND / DN
// (two outputs), k in [1, n] for DF (one output X_{k-1}).
template <typename T>
__device__ __forceinline__ void post_new(int kind, int n, int L, const cpx<T>* Z, int zes, T* out, int oes,
                                         const cpx<T>* pst, int k) {
    if (kind == KIND_DF) {
        const cpx<T> A = Z[k * zes], B = conj_(Z[(L - k) * zes]);
        const cpx<T> d = A - B;
        const cpx<T> W = pst[k];
        // Im Y_k = Im E + Im(W O), E = (A + B)/2, O = (A - B)/(2i)
        const T imy = T(0.5) * (A.y + B.y) + T(0.5) * (fma_(W.x, -d.x, mul_(W.y, d.y)));
        out[(k - 1) * oes] = T(-0.5) * imy;
        return;
    }
    const cpx<T> w = cmul(Z[k * zes], pst[k]);
    out[2 * k * oes] = w.x;
    out[(n - 1 - 2 * k) * oes] = kind == KIND_ND ? -w.y : w.y;
}

// Position of input sample s in the packed sequence v (Makhoul reordering for
// N and D; identity for P) and its sign (-1)^s for D.
__device__ __forceinline__ int pack_index(int kind, int n, int s) {
    if (kind == KIND_P) return s;
    return (s & 1) ? (n - 1 - (s >> 1)) : (s >> 1);
}

template <typename T> __device__ __forceinline__ T pack_sign(int kind, int s) {
    return (kind == KIND_D && (s & 1)) ? T(-1) : T(1);
}

// Natural sample behind element d of the packed sequence v (inverse of
// pack_index; n even): identity for P, Makhoul's even/odd split for N and D.
__device__ __forceinline__ int unpack_src(int kind, int n, int d) {
    if (kind == KIND_P) return d;
    return d < (n >> 1) ? 2 * d : 2 * (n - 1 - d) + 1;
}

// Real natural-order lines: element s of line l at base[l * nls + s * nes].
// in64: FP64 input lines read from global memory and truncated to T (IO bit
// 16 of a first pass), for the FP32 solve of an FP64 right-hand side.
template <typename T> struct NatIO {
    const T* in;
    T* out;
    int nls, nes;
    const double* in64;
};

__device__ __forceinline__ float trunc_double_int(double d);

// ---------------------------------------------------------------------------
// One Stockham autosort pass of radix R over a set of lines in shared memory
// (Govindaraju et al., SC'08 formulation): reads element j + r*L/R, applies
// the twiddles of sub-transform position k = j mod Ns, writes to
// (j - k)*R + k + r*Ns.  Lines: element e of line l at l*ls + e*es.
// TXC > 0: TXC lines (tile columns), consecutive threads -> consecutive lines;
// TXC == 0: consecutive threads -> consecutive butterflies of one line.
// IO bit 0: the pass reads the real natural-order input directly, applying
// the packing (real pairs, Makhoul order, DST signs) on the fly; bit 1: the
// pass writes the real natural-order output directly (the inverse unpacking).
// Divisions by run-time sizes use precomputed multiply-high magics.
// ---------------------------------------------------------------------------
// Row work buffers (FP32 complex, lines contiguous) are XOR-swizzled within
// blocks of 16 elements: element i lives at i ^ sw(i >> 4) with
// sw(b) = (b & 7) | ((parity(b & 7) ^ bit 3 of b) << 3), a bijection of the
// low four bits of b.  Aligned runs of 16 stay one conflict-free wavefront,
// and the strided writes of the early Stockham passes (R = 16 with Ns = 1,
// R = 8 with Ns = 1, 2, 4, 8, R = 4 with Ns = 1) land in 16 distinct 8-byte
// bank pairs per half-warp instead of piling into R-way conflicts.  Buffers
// hold a multiple of 16 elements so the map stays inside them.
// FAST: when the first pass is radix 16 (the only pass with Ns < 16), the
// plain map sw(b) = b & 15 already separates its stride-16 writes, for two
// integer operations instead of six.
template <bool ON, bool FAST = false> __device__ __forceinline__ int swz(int i) {
    if (!ON) return i;
    if (FAST) return i ^ ((i >> 4) & 15);
    const int b = i >> 4;
    const int lo = b & 7;
    return i ^ (lo | (((__popc(lo) ^ (b >> 3)) & 1) << 3));
}

// IO bits: 1 = first pass packs the real natural input, 2 = last pass unpacks
// into the real natural output, 4 = source swizzled, 8 = destination swizzled,
// 16 = the natural input is FP64 in global memory (NatIO::in64), 32 = the
// swizzle is the radix-16-first one (swz FAST).
// LS > 0: the line length L = LS is a compile-time constant (n = 2 LS), and
// so are the pass sizes (NSS = Ns of this pass); KS >= 0: compile-time kind.
// Then every index division folds to constants and shifts.
template <typename T, int R, bool INV, int TXC, int IO, int LS = 0, int NSS = 0, int KS = -1, int TWO = 0>
__device__ __forceinline__ void stockham_pass(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                              const DirTab<T>& t, int p, int nlines, int ls, int es,
                                              const cpx<T>* __restrict__ tw, const NatIO<T>& nat) {
    const int n = LS ? 2 * LS : t.n;
    const int kind = KS >= 0 ? KS : t.kind;
    constexpr int nbS = LS ? LS / R : 1;
    const int nb = LS ? nbS : t.L / R;
    const int Ns = LS ? NSS : t.nsv[p];
    const cpx<T>* __restrict__ tp = tw + (LS ? TWO : t.twoff[p]);
    const int total = nb * (TXC > 0 ? TXC : nlines);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int line, j, k;
        if (TXC > 0) {
            j = (int)((unsigned)idx / (unsigned)(TXC > 0 ? TXC : 1));
            line = idx - j * TXC;
        } else if (LS) {
            line = (int)((unsigned)idx / (unsigned)nbS);
            j = idx - line * nbS;
        } else {
            line = (int)fdivu((unsigned)idx, t.nbmag[p]);
            j = idx - line * nb;
        }
        if (LS) k = (int)((unsigned)j % (unsigned)(NSS > 0 ? NSS : 1));
        else k = j - (int)fdivu((unsigned)j, t.nsmag[p]) * Ns;
        cpx<T> v[R];
        if ((IO & 16) && (IO & 1)) {
            const double* xin = nat.in64 + line * nat.nls;
            if (kind == KIND_P && nat.nes == 1) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double2 d = *reinterpret_cast<const double2*>(xin + 2 * (j + r * nb));
                    v[r] = mk(T(trunc_double_int(d.x)), T(trunc_double_int(d.y)));
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = j + r * nb;
                    const int s0 = unpack_src(kind, n, 2 * q), s1 = unpack_src(kind, n, 2 * q + 1);
                    v[r] = mk(T(trunc_double_int(xin[s0 * nat.nes])) * pack_sign<T>(kind, s0),
                              T(trunc_double_int(xin[s1 * nat.nes])) * pack_sign<T>(kind, s1));
                }
            }
        } else if (IO & 1) {
            const T* xin = nat.in + line * nat.nls;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = j + r * nb;
                const int s0 = unpack_src(kind, n, 2 * q), s1 = unpack_src(kind, n, 2 * q + 1);
                v[r] = mk(xin[s0 * nat.nes] * pack_sign<T>(kind, s0), xin[s1 * nat.nes] * pack_sign<T>(kind, s1));
            }
        } else {
            const int s0 = line * ls + j * es, sst = nb * es;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = src[swz<(IO & 4) != 0, (IO & 32) != 0>(s0 + r * sst)];
        }
        if (LS ? (NSS > 1) : (Ns > 1)) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const cpx<T> w = tp[(r - 1) * Ns + k];
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        Bfly<T, R, INV>::run(v);
        const int base = (j - k) * R + k;
        if (IO & 2) {
            T* xo = nat.out + line * nat.nls;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = base + r * Ns;
                const int s0 = unpack_src(kind, n, 2 * q), s1 = unpack_src(kind, n, 2 * q + 1);
                xo[s0 * nat.nes] = v[r].x * pack_sign<T>(kind, s0);
                xo[s1 * nat.nes] = v[r].y * pack_sign<T>(kind, s1);
            }
        } else {
            const int d0 = line * ls + base * es, dstp = Ns * es;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[swz<(IO & 8) != 0, (IO & 32) != 0>(d0 + r * dstp)] = v[r];
        }
    }
}

template <typename T, bool INV, int TXC, int IO>
__device__ __forceinline__ void pass_dispatch(int R, const cpx<T>* src, cpx<T>* dst, const DirTab<T>& t, int p,
                                              int nlines, int ls, int es, const cpx<T>* tw, const NatIO<T>& nat) {
    switch (R) {
        case 16: stockham_pass<T, 16, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
        case 8: stockham_pass<T, 8, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
        case 4: stockham_pass<T, 4, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
        case 2: stockham_pass<T, 2, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
        case 3: stockham_pass<T, 3, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
        default: stockham_pass<T, 5, INV, TXC, IO>(src, dst, t, p, nlines, ls, es, tw, nat); break;
    }
}

// Compile-time factorisation of a line length (the plan's order: radix 16
// first, then one 8, 4 or 2, then 5s, then 3s); 0 past the last pass.
constexpr int sf_radix(int L, int p) {
    int m = L, twos = 0, fives = 0, threes = 0;
    while (m > 1 && m % 2 == 0) { m /= 2; ++twos; }
    while (m > 1 && m % 5 == 0) { m /= 5; ++fives; }
    while (m > 1 && m % 3 == 0) { m /= 3; ++threes; }
    int i = 0;
    for (int c = 0; c < twos / 4; ++c, ++i) if (i == p) return 16;
    if (twos % 4 == 3) { if (i == p) return 8; ++i; }
    if (twos % 4 == 2) { if (i == p) return 4; ++i; }
    if (twos % 4 == 1) { if (i == p) return 2; ++i; }
    for (int c = 0; c < fives; ++c, ++i) if (i == p) return 5;
    for (int c = 0; c < threes; ++c, ++i) if (i == p) return 3;
    return 0;
}
constexpr int sf_nrad(int L) {
    int p = 0;
    while (sf_radix(L, p) != 0) ++p;
    return p;
}
// offset of pass P's twiddle block (passes with Ns > 1 hold (R - 1) Ns entries)
constexpr int sf_twoff(int L, int P) {
    int off = 0, ns = 1;
    for (int q = 0; q < P; ++q) {
        if (ns > 1) off += (sf_radix(L, q) - 1) * ns;
        ns *= sf_radix(L, q);
    }
    return off;
}

// The passes of a compile-time length LS (pass P, sub-transform size NS).
template <typename T, bool INV, int TXC, int LN, int SN, int LS, int KS, int P, int NS>
struct StaticPasses {
    static __device__ __forceinline__ cpx<T>* run(cpx<T>* src, cpx<T>* dst, const DirTab<T>& t, int nlines, int ls,
                                                  int es, const cpx<T>* tw, const NatIO<T>& nat) {
        constexpr int NR = sf_nrad(LS);
        constexpr int R = sf_radix(LS, P);
        constexpr bool first = P == 0, last = P == NR - 1;
        constexpr int SW = (TXC == 0 && sizeof(T) == 4) ? 1 : 0;
        constexpr int FAST = (SW && sf_radix(LS, 0) == 16) ? 32 : 0;
        constexpr int IO = (first ? LN : 0) | (last ? SN : 0) | (first ? 0 : 4 * SW) | (last ? 0 : 8 * SW) |
                           ((first && last) ? 0 : FAST);
        stockham_pass<T, R, INV, TXC, IO, LS, NS, KS, sf_twoff(LS, P)>(src, dst, t, P, nlines, ls, es, tw, nat);
        __syncthreads();
        if constexpr (last) return dst;
        else return StaticPasses<T, INV, TXC, LN, SN, LS, KS, P + 1, NS * R>::run(dst, src, t, nlines, ls, es, tw, nat);
    }
};

// All passes of a length-L FFT (t.nrad >= 1, or LS with sf_nrad(LS) >= 1);
// returns the buffer holding the result (for STORE_NAT the result is in
// nat.out and the return is unused).  LOAD_NAT: the first pass packs the real
// natural input itself (b0 unused as input); STORE_NAT: the last pass unpacks
// into the real natural output.  `tw` is the twiddle table W_L^t staged in
// shared memory by the caller (per-pass layout of DirTab::tw).
template <typename T, bool INV, int TXC, bool LOAD_NAT, bool STORE_NAT, int LS = 0, int KS = -1, bool IN64 = false>
__device__ cpx<T>* fft_lines(cpx<T>* b0, cpx<T>* b1, const DirTab<T>& t, int nlines, int ls, int es,
                             const cpx<T>* tw, const NatIO<T>& nat) {
    constexpr int LN = LOAD_NAT ? (IN64 ? 17 : 1) : 0, SN = STORE_NAT ? 2 : 0;
    if constexpr (LS > 0) {
        return StaticPasses<T, INV, TXC, LN, SN, LS, KS, 0, 1>::run(b0, b1, t, nlines, ls, es, tw, nat);
    } else {
        // row buffers between passes are swizzled (FP32 only: 8-byte elements);
        // the input of the first and the output of the last pass are not
        constexpr int SW = (TXC == 0 && sizeof(T) == 4) ? 1 : 0;
        cpx<T>* src = b0;
        cpx<T>* dst = b1;
        for (int p = 0; p < t.nrad; ++p) {
            const bool first = p == 0, last = p == t.nrad - 1;
            const int R = t.radix[p];
            if (first && last) pass_dispatch<T, INV, TXC, LN | SN>(R, src, dst, t, p, nlines, ls, es, tw, nat);
            else if (first) pass_dispatch<T, INV, TXC, LN | 8 * SW>(R, src, dst, t, p, nlines, ls, es, tw, nat);
            else if (last) pass_dispatch<T, INV, TXC, SN | 4 * SW>(R, src, dst, t, p, nlines, ls, es, tw, nat);
            else pass_dispatch<T, INV, TXC, 12 * SW>(R, src, dst, t, p, nlines, ls, es, tw, nat);
            __syncthreads();
            cpx<T>* tmp = src; src = dst; dst = tmp;
        }
        return src;
    }
}

// Forward post-processing of the mode pair (m, L - m), m in [0, L/2], of one
// line: Z is the length-L FFT of the packed pairs, the real outputs go to
// `out` (element q of the line at out[q*oes]).  pst, mk: W_n^m and
// exp(-i pi m / (2n)) tables (m in [0, L]).  For V_{L-m} the even and odd
// parts are the conjugates of those of V_m.
template <typename T>
__device__ __forceinline__ void post_store(T* out, int oes, int kind, int n, int L, int m, cpx<T> v, cpx<T> mkm) {
    if (kind == KIND_P) {
        out[m * oes] = v.x;
        if (m > 0 && m < L) out[(n - m) * oes] = v.y;
    } else {
        const cpx<T> u = cmul(mkm, v);
        if (kind == KIND_N) {
            out[m * oes] = u.x;
            if (m > 0 && m < L) out[(n - m) * oes] = -u.y;
        } else {
            out[(n - 1 - m) * oes] = u.x;
            if (m > 0 && m < L) out[(m - 1) * oes] = -u.y;
        }
    }
}

template <typename T, int LS = 0, int KS = -1>
__device__ __forceinline__ void post_forward_pair(const cpx<T>* Z, int zes, T* out, int oes, const DirTab<T>& t,
                                                  const cpx<T>* pst, const cpx<T>* mkt, int m) {
    const int L = LS ? LS : t.L, n = LS ? 2 * LS : t.n;
    const int kind = KS >= 0 ? KS : t.kind;
    const cpx<T> zm = Z[(m == L ? 0 : m) * zes];
    const cpx<T> zc = conj_(Z[(m == 0 ? 0 : L - m) * zes]);
    const cpx<T> e = scale(zm + zc, T(0.5));
    const cpx<T> dd = zm - zc;
    const cpx<T> o = mk(T(0.5) * dd.y, T(-0.5) * dd.x);            // (zm - zc) / (2i)
    post_store<T>(out, oes, kind, n, L, m, e + cmul(pst[m], o), kind == KIND_P ? mk(T(1), T(0)) : mkt[m]);
    const int m2 = L - m;
    if (m2 != m)
        post_store<T>(out, oes, kind, n, L, m2, conj_(e) + cmul(pst[m2], conj_(o)),
                      kind == KIND_P ? mk(T(1), T(0)) : mkt[m2]);
}

// V_m of the inverse (m in [0, L]) from the real coefficients X of one line.
template <typename T, int LS = 0, int KS = -1>
__device__ __forceinline__ cpx<T> inv_spectrum(const T* X, int xes, const DirTab<T>& t, const cpx<T>* mkt, int m) {
    const int L = LS ? LS : t.L, n = LS ? 2 * LS : t.n;
    const int kind = KS >= 0 ? KS : t.kind;
    if (kind == KIND_P) {
        const T im = (m > 0 && m < L) ? X[(n - m) * xes] : T(0);
        return mk(X[m * xes], im);
    }
    cpx<T> u;
    if (kind == KIND_N) u = mk(X[m * xes], m > 0 ? -X[(n - m) * xes] : T(0));
    else                u = mk(X[(n - 1 - m) * xes], m > 0 ? -X[(m - 1) * xes] : T(0));
    return cmulc(u, mkt[m]);   // exp(+i pi m / (2n)) * U_m
}

// Inverse pre-processing of the pair (m, L - m), m in [0, L/2]: Z_m (and
// Z_{L-m} when it differs and is < L) whose unnormalised inverse FFT gives
// n * (x[2j] + i x[2j+1]) of the packed sequence.
template <typename T, int LS = 0, int KS = -1>
__device__ __forceinline__ void pre_inverse_pair(const T* X, int xes, cpx<T>* Z, int zes, const DirTab<T>& t,
                                                 const cpx<T>* pst, const cpx<T>* mkt, int m) {
    const int L = LS ? LS : t.L;
    const cpx<T> vm = inv_spectrum<T, LS, KS>(X, xes, t, mkt, m);
    const cpx<T> vl = inv_spectrum<T, LS, KS>(X, xes, t, mkt, L - m);
    {
        const cpx<T> vc = conj_(vl);
        const cpx<T> s = vm + vc;
        const cpx<T> d = cmulc(vm - vc, pst[m]);
        Z[m * zes] = mk(s.x - d.y, s.y + d.x);
    }
    const int m2 = L - m;
    if (m2 != m && m2 < L) {
        const cpx<T> vc = conj_(vm);
        const cpx<T> s = vl + vc;
        const cpx<T> d = cmulc(vl - vc, pst[m2]);
        Z[m2 * zes] = mk(s.x - d.y, s.y + d.x);
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk) between global and shared memory with an
// mbarrier for completion.  Every wait is bounded: after MBAR_MAX_POLLS failed
// polls the caller records a timeout in the status word and gives up.
// ---------------------------------------------------------------------------
constexpr long MBAR_MAX_POLLS = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// One line of global memory into L2 (no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* g) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(g));
}

// Bring [g, g + bytes) into L2 ahead of plain loads (16-byte aligned, size a
// multiple of 16); no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* g, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    for (long i = 0; i < MBAR_MAX_POLLS; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
// global -> shared, completes `bytes` on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// shared -> global (bulk group)
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Ampere-style asynchronous 16-byte copies global -> shared (zero-filled
// when `valid` is false); completion by cp.async.wait_all.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recently committed group complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_none() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Warp 0 moves `nrows` rows of `rowb` bytes (row r: src + r*sstride -> dst +
// r*dstride, strides in elements); lane 0 posts the byte count first.
template <typename T>
__device__ __forceinline__ void bulk_load_rows(uint64_t* bar, T* dst, long dstride, const T* src, long sstride,
                                               int nrows, uint32_t rowb) {
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) mbar_expect_tx(bar, rowb * (uint32_t)nrows);
        __syncwarp();
        for (int r = threadIdx.x; r < nrows; r += 32) bulk_g2s(dst + r * dstride, src + r * sstride, rowb, bar);
    }
}
template <typename T>
__device__ __forceinline__ void bulk_store_rows(T* dst, long dstride, const T* src, long sstride, int nrows,
                                                uint32_t rowb) {
    if (threadIdx.x < 32) {
        for (int r = threadIdx.x; r < nrows; r += 32) bulk_s2g(dst + r * dstride, src + r * sstride, rowb);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 units (Dekker / Knuth error-free
// transformations): a value is hi + lo with |lo| <= ulp(hi)/2, about 48
// significant bits.  Used where FP64 would run on GB300's narrow FP64 pipe.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = __double2float_rn(v);
    return ff{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

// hi + lo (a normalised pair) as a double without FP64 instructions: hi's bit
// pattern widened to a double, then lo, scaled to units of the double's last
// place by an exact power-of-two multiply and rounded to an integer, added to
// (same signs) or subtracted from (opposite signs) that pattern as a 64-bit
// integer.  hi + lo never leaves hi's binade upward; when hi is a power of
// two and lo has the opposite sign the result lies one binade lower, where the
// last place is half as large.  Tiny, huge, zero or non-finite hi take the
// FP64 path.
__device__ __forceinline__ double ff_to_double_bits(ff x) {
    const unsigned hb = __float_as_uint(x.hi), lb = __float_as_uint(x.lo);
    const unsigned eh = (hb >> 23) & 0xffu;
    if (eh < 60u || eh > 253u) return ff_to_double(x);
    const unsigned mant = hb & 0x7fffffu;
    const unsigned long long bits = ((unsigned long long)((hb & 0x80000000u) | ((eh + 896u) << 20) | (mant >> 3)) << 32) |
                                    (unsigned long long)(mant << 29);
    const bool opp = ((lb ^ hb) & 0x80000000u) && x.lo != 0.f;
    const unsigned down = (mant == 0u && opp) ? 1u : 0u;
    const float sc = __uint_as_float((306u + down - eh) << 23);        // 2^(179 - eh (+1))
    const unsigned long long l = __float2uint_rn(fabsf(x.lo) * sc);
    return __longlong_as_double((long long)(opp ? bits - l : bits + l));
}

// 2^k as a float for k in [-126, 127] (bit construction, no FP64 / MUFU).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Double -> float by truncating the significand to 24 bits, with integer
// operations only (GB300's FP64 pipe is ~1/64 of the FP32 rate, and
// conversions run on it).  |d| below 2^-126 flushes to zero.
__device__ __forceinline__ float trunc_double_int(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hw = (unsigned)(b >> 32);
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7ff);
    const int ef = e - 1023 + 127;
    if (ef <= 0) return __int_as_float(sign);
    if (ef >= 255) return __int_as_float(sign | 0x7f800000u | (e == 0x7ff && (b << 12) ? 0x400000u : 0u));
    const unsigned mh = (unsigned)((b >> 29) & 0x7fffffu);
    return __int_as_float(sign | ((unsigned)ef << 23) | mh);
}

// Double -> double-float pair (hi = 24-bit truncation, lo = the remaining 29
// significand bits rounded to a float), integer and FP32 operations only;
// hi + lo carries about 48 bits of d.
__device__ __forceinline__ ff split_double_int(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const float hi = trunc_double_int(d);
    const int e = (int)((b >> 52) & 0x7ff);
    const int ef = e - 1023 + 127;
    if (ef <= 0 || ef >= 255) return ff{hi, 0.f};
    const unsigned rem = (unsigned)(b & 0x1fffffffu);            // low 29 bits of the significand
    float lo = __uint2float_rn(rem);                             // exact to 24 bits
    const int k = e - 1075;                                      // weight of bit 0
    lo = lo * pow2f(max(k + 50, -126)) * pow2f(-50);
    return ff{hi, (b >> 63) ? -lo : lo};
}

}  // namespace cales

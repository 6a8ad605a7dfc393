// FP64 residual of the staggered 7-point operator (Eq. 16 on the MAC grid):
//   r = (f - fshift) - (c0 u + c1 L u)
// with Poisson (c0, c1) = (0, 1) and Helmholtz (1, -alpha).  Boundary ghosts
// are applied in-kernel (periodic wrap, Neumann mirror, Dirichlet
// antisymmetric mirror, zero at a Dirichlet node).  Neighbour reuse in x, y
// and z is left to L1/L2: each thread reads its point and six neighbours.
#include "kernels.cuh"

namespace cales {


__global__ void __launch_bounds__(256) k_residual(ResidArgs a) {
    const long nx = a.nx, ny = a.ny, nz = a.nz;
    const long plane = nx * ny;
    const long N = plane * nz;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
        const long k = idx / plane;
        const long rem = idx - k * plane;
        const long j = rem / nx;
        const long i = rem - j * nx;
        const double* __restrict__ u = a.u;
        const double uc = u[idx];
        double uw, ue, us, un, ud, uu;
        // ghosts (R2): N mirror, D antisymmetric mirror, DF zero boundary node,
        // per side for the mixed kinds
        if (i > 0) uw = u[idx - 1];
        else uw = (a.bcx == KIND_P) ? u[idx + nx - 1] : (double)ghost_lo(a.bcx) * uc;
        if (i < nx - 1) ue = u[idx + 1];
        else ue = (a.bcx == KIND_P) ? u[idx - (nx - 1)] : (double)ghost_hi(a.bcx) * uc;
        if (j > 0) us = u[idx - nx];
        else us = (a.bcy == KIND_P) ? u[idx + (ny - 1) * nx] : (double)ghost_lo(a.bcy) * uc;
        if (j < ny - 1) un = u[idx + nx];
        else un = (a.bcy == KIND_P) ? u[idx - (ny - 1) * nx] : (double)ghost_hi(a.bcy) * uc;
        // z: periodic (kind 0) wraps through the period, else the R2 ghosts
        if (k > 0) ud = u[idx - plane];
        else ud = a.zlo == 0 ? u[idx + (nz - 1) * plane] : (a.zlo == ZBC_N ? uc : (a.zlo == ZBC_D ? -uc : 0.0));
        if (k < nz - 1) uu = u[idx + plane];
        else uu = a.zhi == 0 ? u[idx - (nz - 1) * plane] : (a.zhi == ZBC_N ? uc : (a.zhi == ZBC_D ? -uc : 0.0));
        const double lu = (ue + uw - 2.0 * uc) * a.idx2 + (un + us - 2.0 * uc) * a.idy2
                        + a.zc[k] * (uu - uc) - a.za[k] * (uc - ud);
        const double r = (a.f[idx] - a.fshift) - (a.c0 * uc + a.c1 * lu);
        if (a.r_is_double) reinterpret_cast<double*>(a.r)[idx] = r;
        else reinterpret_cast<float*>(a.r)[idx] = float(r);
    }
}

// FP32 residual update of the fast refinement mode: r <- r - M d - dshift,
// M = c0 I + c1 L with the R2 ghosts (per side) and a periodic z wrap.  A CTA
// covers whole rows of one plane (blockIdx.y); each thread takes VW
// consecutive points of a row (VW = 4 with 16-byte vector loads when the
// rows allow it, else 1), the threads running over (row, group) together.
template <int VW>
__global__ void __launch_bounds__(256) k_residual_update(const __grid_constant__ ResidUpdArgs a, const int rows) {
    const int nx = a.nx, ny = a.ny;
    const int k = blockIdx.y;
    const long plane = (long)nx * ny;
    const float dshift = a.acc ? (float)(a.acc[0] - a.acc[2]) : 0.f;
    const RUPlane pk = ru_plane(a, k);
    const int j0 = blockIdx.x * rows, j1 = min(j0 + rows, ny);
    const int ng = nx / VW;
    const unsigned gmag = div_magic((unsigned)ng);
    const int tot = (j1 - j0) * ng;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int jj = (int)fdivu((unsigned)t, gmag);
        const int j = j0 + jj, i = (t - jj * ng) * VW;
        float r[VW];
        resupd_group<VW>(a, pk, i, j, k, dshift, r);
        float* o = a.r + (long)k * plane + (long)j * nx + i;
        if (VW == 4) *reinterpret_cast<float4*>(o) = make_float4(r[0], r[1], r[2], r[3]);
        else o[0] = r[0];
    }
}

cudaError_t launch_residual_update(const ResidUpdArgs& a, cudaStream_t st) {
    const int rows = residual_rows_per_cta(a.nx, a.ny);
    const dim3 grid((unsigned)((a.ny + rows - 1) / rows), (unsigned)a.nz);
    const bool vec = a.nx % 4 == 0 && ((uintptr_t)a.r % 16) == 0 && ((uintptr_t)a.d % 16) == 0;
    if (vec) k_residual_update<4><<<grid, 256, 0, st>>>(a, rows);
    else k_residual_update<1><<<grid, 256, 0, st>>>(a, rows);
    return cudaGetLastError();
}

cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st) {
    const long N = (long)a.nx * a.ny * a.nz;
    long blocks = (N + 255) / 256;
    if (blocks > 152L * 64) blocks = 152L * 64;
    k_residual<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Double-float residual (FP32 pipes).  u is stored as (hi, lo) float pairs;
// each difference and product is carried in double-float, and f is split
// into a pair with integer operations, so no FP64 instruction runs per point.  One CTA row of
// the grid per z-plane, so the dzf weight of the gauge sum is uniform in it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff ldu(const float2* __restrict__ u, long i) {
    const float2 v = u[i];
    return ff{v.x, v.y};
}

__device__ __forceinline__ ff ghost_ff(int kind, ff c) { return kind == KIND_N ? c : ff_neg(c); }

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

// r = f - cshift - (c0 u + c1 L u) with u = (hi, lo) pairs, written with the
// neighbour differences first,
//   f - cshift - c0 uc - [cx ((ue-uc) + (uw-uc)) + cy ((un-uc) + (us-uc))
//                         + zc (uu-uc) + za (ud-uc)],
// so rounding errors scale with the (small) differences of a smooth u, not
// with u times the large 1/dz^2 couplings.  Differences of the hi parts are
// exact (TwoSum), products of the leading parts exact (TwoProd by FMA), the
// accumulation is TwoSum with every rounding error gathered in one FP32
// compensation term, and the lo parts (2^-24 smaller) and the low halves of
// the coefficients enter that term in plain FP32: about double-float accuracy
// with fewer instructions.
__global__ void __launch_bounds__(256) k_residual_ff(ResidFFArgs a) {
    const int nx = a.nx, ny = a.ny;
    const long plane = (long)nx * ny;
    const int k = blockIdx.y;
    const long kbase = (long)k * plane;
    const float2* __restrict__ u = a.u;
    // plane coefficients (FP64 once per CTA, then split)
    const double zad = a.c1 * a.za[k], zcd = a.c1 * a.zc[k];
    const double cxd = (double)a.cxh + (double)a.cxl, cyd = (double)a.cyh + (double)a.cyl;
    const ff za = ff_from_double(zad), zc = ff_from_double(zcd);
    const ff cx{a.cxh, a.cxl}, cy{a.cyh, a.cyl};
    const float c0 = a.c0h;     // 0 (Poisson) or 1 (Helmholtz): c0 u is exact
    (void)cxd; (void)cyd;
    const ff csh = a.cshift ? ff_from_double(a.cshift[0]) : ff{0.f, 0.f};
    const bool kd = k > 0, ku = k < a.nz - 1;
    const float gd = a.zlo == ZBC_N ? 1.f : (a.zlo == ZBC_D ? -1.f : 0.f);
    const float gu = a.zhi == ZBC_N ? 1.f : (a.zhi == ZBC_D ? -1.f : 0.f);
    const float gxl = ghost_lo(a.bcx), gxh = ghost_hi(a.bcx), gyl = ghost_lo(a.bcy), gyh = ghost_hi(a.bcy);
    ff gsum{0.f, 0.f};                       // gauge sum of u (double-float)
    const int rows = a.rows_per_cta;
    const int j0 = blockIdx.x * rows, j1 = min(j0 + rows, ny);
    for (int j = j0; j < j1; ++j) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const long idx = kbase + (long)j * nx + i;
            const float2 c = u[idx];
            float2 w, e, s, n, d, up;
            if (i > 0) w = u[idx - 1];
            else w = a.bcx == KIND_P ? u[idx + nx - 1] : make_float2(gxl * c.x, gxl * c.y);
            if (i < nx - 1) e = u[idx + 1];
            else e = a.bcx == KIND_P ? u[idx - (nx - 1)] : make_float2(gxh * c.x, gxh * c.y);
            if (j > 0) s = u[idx - nx];
            else s = a.bcy == KIND_P ? u[idx + (long)(ny - 1) * nx] : make_float2(gyl * c.x, gyl * c.y);
            if (j < ny - 1) n = u[idx + nx];
            else n = a.bcy == KIND_P ? u[idx - (long)(ny - 1) * nx] : make_float2(gyh * c.x, gyh * c.y);
            if (kd || a.zlo == 0) d = u[idx + (kd ? -plane : (long)(a.nz - 1) * plane)];
            else d = make_float2(gd * c.x, gd * c.y);
            if (ku || a.zhi == 0) up = u[idx + (ku ? plane : -(long)(a.nz - 1) * plane)];
            else up = make_float2(gu * c.x, gu * c.y);
            // exact differences of the hi parts (TwoSum), lo parts in FP32:
            // errors scale with the small neighbour differences of a smooth u
            const ff de = two_sum(e.x, -c.x), dw = two_sum(w.x, -c.x);
            const ff dn = two_sum(n.x, -c.x), ds = two_sum(s.x, -c.x);
            const ff du = two_sum(up.x, -c.x), dd = two_sum(d.x, -c.x);
            const ff sx = two_sum(de.hi, dw.hi), sy = two_sum(dn.hi, ds.hi);
            const float sxl = sx.lo + de.lo + dw.lo + ((e.y - c.y) + (w.y - c.y));
            const float syl = sy.lo + dn.lo + ds.lo + ((n.y - c.y) + (s.y - c.y));
            const float dul = du.lo + (up.y - c.y), ddl = dd.lo + (d.y - c.y);
            // exact products of the leading parts, first-order corrections in comp
            const ff px = two_prod(cx.hi, sx.hi);
            float comp = __fmaf_rn(cx.hi, sxl, __fmaf_rn(cx.lo, sx.hi, px.lo));
            const ff py = two_prod(cy.hi, sy.hi);
            comp += __fmaf_rn(cy.hi, syl, __fmaf_rn(cy.lo, sy.hi, py.lo));
            const ff pz = two_prod(zc.hi, du.hi);
            comp += __fmaf_rn(zc.hi, dul, __fmaf_rn(zc.lo, du.hi, pz.lo));
            const ff pd = two_prod(za.hi, dd.hi);
            comp += __fmaf_rn(za.hi, ddl, __fmaf_rn(za.lo, dd.hi, pd.lo));
            // accumulate f - cshift - c0 u - t
            const ff fs = split_double_int(a.f[idx]);
            ff acc = two_sum(fs.hi, -csh.hi);
            float err = acc.lo + fs.lo - csh.lo - comp - c0 * c.y;
            acc = two_sum(acc.hi, -c0 * c.x); err += acc.lo;
            acc = two_sum(acc.hi, -px.hi); err += acc.lo;
            acc = two_sum(acc.hi, -py.hi); err += acc.lo;
            acc = two_sum(acc.hi, -pz.hi); err += acc.lo;
            acc = two_sum(acc.hi, -pd.hi); err += acc.lo;
            a.r[idx] = __fadd_rn(acc.hi, err);
            if (a.gacc) gsum = ff_add(gsum, ff{c.x, c.y});
        }
    }
    if (a.gacc) {
        double v = ff_to_double(gsum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double red[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += red[w2];
            atomicAdd(a.gacc, t * a.dzf[k]);
        }
    }
}

// Double -> (hi, lo) pair as split_double_int, with fewer integer operations
// for |d| in [2^-74, 2^128) (both parts normal floats); other values (zero,
// tiny, huge, non-finite) take the general path.
__device__ __forceinline__ ff split_double_fast(double d) {
    const unsigned lw = (unsigned)__double2loint(d), hw = (unsigned)__double2hiint(d);
    const unsigned e = (hw >> 20) & 0x7ffu;
    if (e - 949u > 201u) return split_double_int(d);
    const unsigned sg = hw & 0x80000000u;
    const float hi = __uint_as_float(sg | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const float lo = __uint2float_rn(lw & 0x1fffffffu) * __uint_as_float(sg | ((e - 948u) << 23));
    return ff{hi, lo};
}

// Second difference a + b - 2c of three hi parts as an exact pair: TwoSum of
// the neighbours, then TwoSum with -2c (exact scaling); the two rounding
// errors are gathered in one float.  About half the operations of two
// one-sided differences and their TwoSum.
__device__ __forceinline__ ff second_diff(float a, float b, float c) {
    const ff t = two_sum(a, b);
    const ff v = two_sum(t.hi, -2.f * c);
    return ff{v.hi, t.lo + v.lo};
}

// One point of the double-float residual
//   r = (f - cshift) - (c0 u + cx Sx + cy Sy + zc (u_up - u) + za (u_dn - u)),
// Sx = u_e + u_w - 2u, Sy = u_n + u_s - 2u, with u = (hi, lo) pairs: second
// differences and one-sided z differences of the hi parts exact (TwoSum),
// leading products exact (TwoProd by FMA), every rounding error and the
// first-order terms of the lo parts and of the coefficients' low halves
// gathered in one FP32 compensation, the accumulation a TwoSum chain.  LO =
// false: every lo part is zero (the first sweep after an FP32 solve).
// SING: singular Poisson (consistency shift subtracted); HELM: the c0 u term
// of Eq. 18; GAUGE: the gauge sum of u as an unnormalised (hi, lo) pair.
template <bool SING, bool HELM, bool GAUGE, bool LO>
__device__ __forceinline__ float resid_point(float2 c, float2 w, float2 e, float2 s, float2 n, float2 d, float2 up,
                                             double fv, ff cx, ff cy, ff zc, ff za, ff csh, float& ghi,
                                             float& glo) {
    const ff sx = second_diff(e.x, w.x, c.x), sy = second_diff(n.x, s.x, c.x);
    const ff du = two_sum(up.x, -c.x), dd = two_sum(d.x, -c.x);
    float sxl = sx.lo, syl = sy.lo, dul = du.lo, ddl = dd.lo;
    if (LO) {
        sxl += __fmaf_rn(-2.f, c.y, e.y + w.y);
        syl += __fmaf_rn(-2.f, c.y, n.y + s.y);
        dul += up.y - c.y;
        ddl += d.y - c.y;
    }
    const ff px = two_prod(cx.hi, sx.hi);
    float comp = __fmaf_rn(cx.hi, sxl, __fmaf_rn(cx.lo, sx.hi, px.lo));
    const ff py = two_prod(cy.hi, sy.hi);
    comp += __fmaf_rn(cy.hi, syl, __fmaf_rn(cy.lo, sy.hi, py.lo));
    const ff pz = two_prod(zc.hi, du.hi);
    comp += __fmaf_rn(zc.hi, dul, __fmaf_rn(zc.lo, du.hi, pz.lo));
    const ff pd = two_prod(za.hi, dd.hi);
    comp += __fmaf_rn(za.hi, ddl, __fmaf_rn(za.lo, dd.hi, pd.lo));
    const ff fs = split_double_fast(fv);
    ff acc;
    float err;
    if (SING) {
        acc = two_sum(fs.hi, -csh.hi);
        err = acc.lo + fs.lo - csh.lo - comp;
    } else {
        acc = ff{fs.hi, 0.f};
        err = fs.lo - comp;
    }
    if (HELM) {
        acc = two_sum(acc.hi, -c.x);
        err += acc.lo;
        if (LO) err -= c.y;
    }
    acc = two_sum(acc.hi, -px.hi); err += acc.lo;
    acc = two_sum(acc.hi, -py.hi); err += acc.lo;
    acc = two_sum(acc.hi, -pz.hi); err += acc.lo;
    acc = two_sum(acc.hi, -pd.hi); err += acc.lo;
    if (GAUGE) {
        const ff g = two_sum(ghi, c.x);
        ghi = g.hi;
        glo += LO ? g.lo + c.y : g.lo;
    }
    return __fadd_rn(acc.hi, err);
}

__device__ __forceinline__ float4 ld4(const float2* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 sc4(float g, float4 v) { return make_float4(g * v.x, g * v.y, g * v.z, g * v.w); }

// Two x-adjacent points per thread with 16-byte loads (nx even, 16-byte
// aligned u and f): the centre pair, both y and both z neighbour pairs and
// f come in one vector load each, the x neighbours of the pair in two 8-byte
// loads.  A CTA covers whole rows of one z-plane.
template <bool SING, bool HELM, bool GAUGE, bool LO, bool FLAT>
__device__ __forceinline__ void residual_df_body(const ResidFFArgs& a, const int bx, const int k) {
    const int nx = a.nx, ny = a.ny;
    const long plane = (long)nx * ny;
    const long kbase = (long)k * plane;
    const float2* __restrict__ u = a.u;
    const ff za = ff_from_double(a.c1 * a.za[k]), zc = ff_from_double(a.c1 * a.zc[k]);
    const ff cx{a.cxh, a.cxl}, cy{a.cyh, a.cyl};
    const ff csh = (SING && a.cshift) ? ff_from_double(a.cshift[0]) : ff{0.f, 0.f};
    const bool kd = k > 0, ku = k < a.nz - 1;
    const float gd = a.zlo == ZBC_N ? 1.f : (a.zlo == ZBC_D ? -1.f : 0.f);
    const float gu = a.zhi == ZBC_N ? 1.f : (a.zhi == ZBC_D ? -1.f : 0.f);
    const float gxl = ghost_lo(a.bcx), gxh = ghost_hi(a.bcx), gyl = ghost_lo(a.bcy), gyh = ghost_hi(a.bcy);
    const bool px_ = a.bcx == KIND_P, py_ = a.bcy == KIND_P;
    float ghi = 0.f, glo = 0.f;
    const int npair = nx >> 1;
    const int j0 = bx * a.rows_per_cta, j1 = min(j0 + a.rows_per_cta, ny);
    // neighbour offsets and multipliers: a ghost reads the centre (offset 0)
    // and scales it (Neumann mirror 1, Dirichlet -1, node 0); the tests on
    // the multipliers are uniform per CTA (z) or per row (y)
    // periodic z (kind 0) wraps: plane nz-1 below plane 0, plane 0 above nz-1
    const bool pz_ = a.zlo == 0;
    const long offD = kd ? -plane : (pz_ ? (long)(a.nz - 1) * plane : 0);
    const long offU = ku ? plane : (pz_ ? -(long)(a.nz - 1) * plane : 0);
    const float mD = (kd || pz_) ? 1.f : gd, mU = (ku || pz_) ? 1.f : gu;
    auto pair_at = [&](const int j, const int pi) {
        const long offS = j > 0 ? -(long)nx : (py_ ? (long)(ny - 1) * nx : 0);
        const long offN = j < ny - 1 ? (long)nx : (py_ ? -(long)(ny - 1) * nx : 0);
        const float mS = (j > 0 || py_) ? 1.f : gyl, mN = (j < ny - 1 || py_) ? 1.f : gyh;
        const long rb = kbase + (long)j * nx;
        const int i = 2 * pi;
        const float2* q = u + rb + i;
        const float4 c = ld4(q);
        float4 s = ld4(q + offS), n = ld4(q + offN), d = ld4(q + offD), up = ld4(q + offU);
        const int ow = i > 0 ? -1 : (px_ ? nx - 1 : 0);
        const int oe = i + 2 < nx ? 2 : (px_ ? -i : 1);
        float2 w = q[ow], e = q[oe];
        const double2 fv = *reinterpret_cast<const double2*>(a.f + rb + i);
        if (mS != 1.f) s = sc4(mS, s);
        if (mN != 1.f) n = sc4(mN, n);
        if (mD != 1.f) d = sc4(mD, d);
        if (mU != 1.f) up = sc4(mU, up);
        if (!px_) {
            if (i == 0) w = make_float2(gxl * w.x, gxl * w.y);
            if (i + 2 == nx) e = make_float2(gxh * e.x, gxh * e.y);
        }
        const float r0 = resid_point<SING, HELM, GAUGE, LO>(lo2(c), w, hi2(c), lo2(s), lo2(n), lo2(d), lo2(up),
                                                            fv.x, cx, cy, zc, za, csh, ghi, glo);
        const float r1 = resid_point<SING, HELM, GAUGE, LO>(hi2(c), lo2(c), e, hi2(s), hi2(n), hi2(d), hi2(up),
                                                            fv.y, cx, cy, zc, za, csh, ghi, glo);
        *reinterpret_cast<float2*>(a.r + rb + i) = make_float2(r0, r1);
    };
    if (!FLAT) {
        for (int j = j0; j < j1; ++j)
            for (int pi = threadIdx.x; pi < npair; pi += blockDim.x) pair_at(j, pi);
    } else {
        // short rows (FLAT): the threads run over (row, pair) together, so
        // none idles when a row has fewer pairs than the CTA has threads
        const int tot = (j1 - j0) * npair;
        const unsigned mag = div_magic((unsigned)npair);
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int jj = (int)fdivu((unsigned)e, mag);
            pair_at(j0 + jj, e - jj * npair);
        }
    }
    if (GAUGE && a.gacc) {
        double v = (double)ghi + (double)glo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double red[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += red[w2];
            atomicAdd(a.gacc, t * a.dzf[k]);
        }
    }
}

template <bool SING, bool HELM, bool GAUGE, bool LO, bool FLAT>
__global__ void __launch_bounds__(256) k_residual_df(const __grid_constant__ ResidFFArgs a) {
    residual_df_body<SING, HELM, GAUGE, LO, FLAT>(a, blockIdx.x, blockIdx.y);
}

// Grouped launch over many solves: CTA b takes block work[b].y (row block +
// plane, row blocks fastest) of item work[b].x.
template <bool SING, bool HELM, bool GAUGE, bool LO>
__global__ void __launch_bounds__(256, 4) k_residual_df_grp(const ResidFFArgs* __restrict__ items,
                                                         const int2* __restrict__ work) {
    __shared__ __align__(16) ResidFFArgs sa;
    const int2 w = work[blockIdx.x];
    {
        const int* src = reinterpret_cast<const int*>(items + w.x);
        int* d = reinterpret_cast<int*>(&sa);
        for (int i = threadIdx.x; i < (int)(sizeof(ResidFFArgs) / 4); i += blockDim.x) d[i] = src[i];
    }
    __syncthreads();
    const int nby = (sa.ny + sa.rows_per_cta - 1) / sa.rows_per_cta;
    const int k = w.y / nby;
    residual_df_body<SING, HELM, GAUGE, LO, true>(sa, w.y - k * nby, k);
}

// Rows per CTA of the double-float residual: about 4096 points, whole rows.
int residual_rows_per_cta(int nx, int ny) {
    int rows = (int)((4096 + nx - 1) / nx);
    if (rows < 1) rows = 1;
    if (rows > ny) rows = ny;
    return rows;
}

cudaError_t launch_residual_ff_grp(const ResidFFArgs* items, const int2* work, int nblocks, int variant,
                                   cudaStream_t st) {
    // variant bits: 1 SING, 2 HELM, 4 GAUGE, 8 LO
    const dim3 g((unsigned)nblocks), b(256);
    switch (variant) {
        case 0: k_residual_df_grp<false, false, false, false><<<g, b, 0, st>>>(items, work); break;
        case 2: k_residual_df_grp<false, true, false, false><<<g, b, 0, st>>>(items, work); break;
        case 1: k_residual_df_grp<true, false, false, false><<<g, b, 0, st>>>(items, work); break;
        case 3: k_residual_df_grp<true, true, false, false><<<g, b, 0, st>>>(items, work); break;
        case 5: k_residual_df_grp<true, false, true, false><<<g, b, 0, st>>>(items, work); break;
        case 7: k_residual_df_grp<true, true, true, false><<<g, b, 0, st>>>(items, work); break;
        case 8: k_residual_df_grp<false, false, false, true><<<g, b, 0, st>>>(items, work); break;
        case 10: k_residual_df_grp<false, true, false, true><<<g, b, 0, st>>>(items, work); break;
        case 9: k_residual_df_grp<true, false, false, true><<<g, b, 0, st>>>(items, work); break;
        case 11: k_residual_df_grp<true, true, false, true><<<g, b, 0, st>>>(items, work); break;
        case 13: k_residual_df_grp<true, false, true, true><<<g, b, 0, st>>>(items, work); break;
        case 15: k_residual_df_grp<true, true, true, true><<<g, b, 0, st>>>(items, work); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool LO, bool FLAT>
static void launch_df(const ResidFFArgs& a, dim3 grid, bool sing, bool helm, cudaStream_t st) {
    if (a.gacc && !helm) k_residual_df<true, false, true, LO, FLAT><<<grid, 256, 0, st>>>(a);
    else if (a.gacc) k_residual_df<true, true, true, LO, FLAT><<<grid, 256, 0, st>>>(a);
    else if (sing && !helm) k_residual_df<true, false, false, LO, FLAT><<<grid, 256, 0, st>>>(a);
    else if (sing) k_residual_df<true, true, false, LO, FLAT><<<grid, 256, 0, st>>>(a);
    else if (helm) k_residual_df<false, true, false, LO, FLAT><<<grid, 256, 0, st>>>(a);
    else k_residual_df<false, false, false, LO, FLAT><<<grid, 256, 0, st>>>(a);
}

cudaError_t launch_residual_ff(const ResidFFArgs& a0, cudaStream_t st) {
    ResidFFArgs a = a0;
    const int rows = residual_rows_per_cta(a.nx, a.ny);
    a.rows_per_cta = rows;
    dim3 grid((unsigned)((a.ny + rows - 1) / rows), (unsigned)a.nz);
    const bool vec = (a.nx % 2 == 0) && ((uintptr_t)a.u % 16 == 0) && ((uintptr_t)a.f % 16 == 0) &&
                     ((uintptr_t)a.r % 8 == 0);
    const bool sing = a.gacc != nullptr || a.cshift != nullptr;
    const bool helm = a.c0h != 0.f;
    if (!vec) k_residual_ff<<<grid, 256, 0, st>>>(a);
    else if (a.nx / 2 >= 256) {
        if (a.lo_zero) launch_df<false, false>(a, grid, sing, helm, st);
        else launch_df<true, false>(a, grid, sing, helm, st);
    } else {
        if (a.lo_zero) launch_df<false, true>(a, grid, sing, helm, st);
        else launch_df<true, true>(a, grid, sing, helm, st);
    }
    return cudaGetLastError();
}

}  // namespace cales

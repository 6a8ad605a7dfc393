// Plan construction and solve orchestration behind the C ABI (cales.h).
//
// A plan holds, per uniform direction, the FFT length L = n/2, its radix
// factorisation and the twiddle / post-processing / eigenvalue tables
// (computed on the host in FP64 with exact integer argument reduction, FP32
// copies rounded once), and along z the tridiagonal couplings 1/(dzc dzf).
// A solve is five launches on the caller's stream:
//   x forward -> y forward -> z tridiagonal per mode -> y inverse -> x inverse
// FP32_REFINE adds per sweep an FP64 residual and a second FP32 pass whose
// last kernel accumulates the correction into the FP64 solution.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "cales.h"
#include "kernels.cuh"
#include "plan.h"

#include <type_traits>

using namespace cales;

namespace {

void split_double(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// cos and sin of 2 pi num / den with exact integer quadrant reduction.
void cis_frac(long num, long den, double& c, double& s) {
    long r = num % den;
    if (r < 0) r += den;
    const long q = (4 * r) / den;
    const long rem = 4 * r - q * den;
    const double a = 1.5707963267948966192313216916398 * (double)rem / (double)den;
    const double ca = std::cos(a), sa = std::sin(a);
    switch (q & 3) {
        case 0: c = ca; s = sa; break;
        case 1: c = -sa; s = ca; break;
        case 2: c = -ca; s = -sa; break;
        default: c = sa; s = -ca; break;
    }
}

// Radix passes of a length-L FFT.  order 0: radix 16 first (fewest
// shared-memory passes; the compile-time-size kernels use this order, see
// sf_radix), then one 8, 4 or 2, then the 5s and 3s; order 1: the 5s and 3s
// first, then the powers of two as in order 0; order 2: radix 8 passes
// instead of 16 (more passes, fewer registers per butterfly).
bool factorize(int L, int* radix, int& nrad, int order = 0) {
    nrad = 0;
    int m = L;
    int twos = 0, fives = 0, threes = 0;
    while (m % 2 == 0) { m /= 2; ++twos; }
    while (m % 5 == 0) { m /= 5; ++fives; }
    while (m % 3 == 0) { m /= 3; ++threes; }
    if (m != 1) return false;
    auto odd = [&] {
        for (int i = 0; i < fives && nrad < MAX_RADICES; ++i) radix[nrad++] = 5;
        for (int i = 0; i < threes && nrad < MAX_RADICES; ++i) radix[nrad++] = 3;
    };
    auto pow2 = [&] {
        int t = twos;
        if (order != 2)
            while (t >= 4 && nrad < MAX_RADICES) { radix[nrad++] = 16; t -= 4; }
        while (t >= 3 && nrad < MAX_RADICES) { radix[nrad++] = 8; t -= 3; }
        if (t == 2 && nrad < MAX_RADICES) radix[nrad++] = 4;
        if (t == 1 && nrad < MAX_RADICES) radix[nrad++] = 2;
    };
    if (order == 1) { odd(); pow2(); }
    else { pow2(); odd(); }
    int prod = 1;
    for (int i = 0; i < nrad; ++i) prod *= radix[i];
    return prod == L;
}

template <typename T> T* dev_upload(const std::vector<T>& h, std::vector<void*>& owned) {
    void* p = nullptr;
    if (cudaMalloc(&p, h.size() * sizeof(T) + 16) != cudaSuccess) return nullptr;
    cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    owned.push_back(p);
    return reinterpret_cast<T*>(p);
}

// Tables of one uniform direction of n unknowns, transform kind `kind`
// (KIND_P .. KIND_DN) and spacing h.  FFT length L = n/2, or n + 1 for the
// DST-I of node-centred unknowns (the real DFT of the odd extension).
int build_dir(DirHost& d, int n, int kind, double h, std::vector<void*>& owned, int order = 0) {
    d.n = n;
    d.kind = kind;
    if (kind == KIND_DF) {
        d.L = n + 1;
    } else {
        if (n > 1 && (n % 2)) return CALES_EUNSUPPORTED;
        d.L = n >= 2 ? n / 2 : 1;
    }
    if (!factorize(d.L, d.radix, d.nrad, order)) return CALES_EUNSUPPORTED;
    const int L = d.L;
    // per-pass twiddles W_L^(r k tstep) at twoff[p] + (r - 1) Ns + k
    std::vector<double2> tw, post(L + 1), mak(L + 1);
    std::vector<float2> twf, postf(L + 1), makf(L + 1);
    {
        int ns = 1;
        for (int p = 0; p < d.nrad; ++p) {
            const int R = d.radix[p], tstep = L / (ns * R);
            d.twoff[p] = (int)tw.size();
            if (ns > 1)
                for (int r = 1; r < R; ++r)
                    for (int k = 0; k < ns; ++k) {
                        double c, s;
                        cis_frac((int)(((long long)r * k * tstep) % L), L, c, s);
                        tw.push_back(make_double2(c, -s));
                    }
            ns *= R;
        }
        d.twlen = (int)tw.size();
        if (tw.empty()) tw.push_back(make_double2(1.0, 0.0));
        twf.resize(tw.size());
    }
    for (int m = 0; m <= L; ++m) {
        double c, s;
        if (kind == KIND_ND || kind == KIND_DN) {
            cis_frac(m, 2L * n, c, s);                 // exp(-i pi m / n)
            post[m] = make_double2(c, -s);
            cis_frac(4L * m + 1, 8L * n, c, s);        // exp(-i pi (4m + 1) / (4n))
            mak[m] = make_double2(c, -s);
        } else if (kind == KIND_DF) {
            cis_frac(m, 2L * (n + 1), c, s);           // exp(-i pi m / (n + 1))
            post[m] = make_double2(c, -s);
            mak[m] = post[m];
        } else {
            cis_frac(m, n >= 2 ? n : 1, c, s);
            post[m] = make_double2(c, -s);
            cis_frac(m, 4L * (n >= 1 ? n : 1), c, s);
            mak[m] = make_double2(c, -s);
        }
    }
    std::vector<double> lam(n);
    std::vector<float> lamf(n);
    const double pi = 3.14159265358979323846;
    for (int q = 0; q < n; ++q) {
        double sv;
        if (kind == KIND_P) {
            const int m = q <= n / 2 ? q : n - q;
            sv = std::sin(pi * m / n);
        } else if (kind == KIND_N) {
            sv = std::sin(pi * q / (2.0 * n));
        } else if (kind == KIND_D) {
            sv = std::sin(pi * (q + 1) / (2.0 * n));
        } else if (kind == KIND_DF) {
            sv = std::sin(pi * (q + 1) / (2.0 * (n + 1)));
        } else {
            sv = std::sin(pi * (2 * q + 1) / (4.0 * n));
        }
        lam[q] = -(4.0 / (h * h)) * sv * sv;
        lamf[q] = (float)lam[q];
    }
    for (size_t i = 0; i < tw.size(); ++i) twf[i] = make_float2((float)tw[i].x, (float)tw[i].y);
    for (int i = 0; i <= L; ++i) {
        postf[i] = make_float2((float)post[i].x, (float)post[i].y);
        makf[i] = make_float2((float)mak[i].x, (float)mak[i].y);
    }
    d.tw_d = dev_upload(tw, owned);
    d.post_d = dev_upload(post, owned);
    d.mak_d = dev_upload(mak, owned);
    d.lam_d = dev_upload(lam, owned);
    d.tw_f = dev_upload(twf, owned);
    d.post_f = dev_upload(postf, owned);
    d.mak_f = dev_upload(makf, owned);
    d.lam_f = dev_upload(lamf, owned);
    if (!d.tw_d || !d.post_d || !d.mak_d || !d.lam_d || !d.tw_f || !d.post_f || !d.mak_f || !d.lam_f)
        return CALES_ENOMEM;
    return CALES_OK;
}

}  // namespace

// Rebuild the x and y tables with FFT radix order `order` (see factorize);
// the old tables are released.  CALES_EUNSUPPORTED leaves the plan as it was.
int plan_set_radix_order(cales_plan_s* P, int order) {
    if (order == P->radix_order) return CALES_OK;
    if (order < 0 || order > 2) return CALES_EINVAL;
    DirHost nx_, ny_;
    std::vector<void*> fresh;
    int rc = build_dir(nx_, P->nx, P->X.kind, P->dx, fresh, order);
    if (rc == CALES_OK) rc = build_dir(ny_, P->ny, P->Y.kind, P->dy, fresh, order);
    if (rc != CALES_OK) {
        for (void* q : fresh) cudaFree(q);
        return rc;
    }
    for (DirHost* d : {&P->X, &P->Y}) {
        const void* old[8] = {d->tw_d, d->post_d, d->mak_d, d->lam_d, d->tw_f, d->post_f, d->mak_f, d->lam_f};
        for (const void* q : old) {
            for (size_t i = 0; i < P->owned.size(); ++i)
                if (P->owned[i] == q) {
                    cudaFree(P->owned[i]);
                    P->owned.erase(P->owned.begin() + (long)i);
                    break;
                }
        }
    }
    P->X = nx_;
    P->Y = ny_;
    P->owned.insert(P->owned.end(), fresh.begin(), fresh.end());
    P->radix_order = order;
    return CALES_OK;
}

template <> DirTab<double> DirHost::tab<double>() const {
    DirTab<double> t;
    t.n = n; t.kind = kind; t.L = L; t.nrad = nrad;
    int ns = 1;
    for (int i = 0; i < MAX_RADICES; ++i) {
        t.radix[i] = i < nrad ? radix[i] : 1;
        t.nsv[i] = ns;
        t.tstep[i] = i < nrad ? L / (ns * radix[i]) : 1;
        t.nbmag[i] = i < nrad ? div_magic((unsigned)(L / radix[i])) : 0u;
        t.nsmag[i] = div_magic((unsigned)ns);
        t.twoff[i] = twoff[i];
        if (i < nrad) ns *= radix[i];
    }
    t.twlen = twlen;
    t.nmag = div_magic((unsigned)n);
    t.l1mag = div_magic((unsigned)(L + 1));
    t.lmag = div_magic((unsigned)L);
    t.hmag = div_magic((unsigned)(L / 2 + 1));
    t.tw = reinterpret_cast<const cpx<double>*>(tw_d);
    t.post = reinterpret_cast<const cpx<double>*>(post_d);
    t.mak = reinterpret_cast<const cpx<double>*>(mak_d);
    return t;
}

template <> DirTab<float> DirHost::tab<float>() const {
    DirTab<float> t;
    t.n = n; t.kind = kind; t.L = L; t.nrad = nrad;
    int ns = 1;
    for (int i = 0; i < MAX_RADICES; ++i) {
        t.radix[i] = i < nrad ? radix[i] : 1;
        t.nsv[i] = ns;
        t.tstep[i] = i < nrad ? L / (ns * radix[i]) : 1;
        t.nbmag[i] = i < nrad ? div_magic((unsigned)(L / radix[i])) : 0u;
        t.nsmag[i] = div_magic((unsigned)ns);
        t.twoff[i] = twoff[i];
        if (i < nrad) ns *= radix[i];
    }
    t.twlen = twlen;
    t.nmag = div_magic((unsigned)n);
    t.l1mag = div_magic((unsigned)(L + 1));
    t.lmag = div_magic((unsigned)L);
    t.hmag = div_magic((unsigned)(L / 2 + 1));
    t.tw = reinterpret_cast<const cpx<float>*>(tw_f);
    t.post = reinterpret_cast<const cpx<float>*>(post_f);
    t.mak = reinterpret_cast<const cpx<float>*>(mak_f);
    return t;
}

namespace cales {

// Rows per CTA of the x kernels: about 64 KB of shared memory per CTA
// (two transform buffers plus the FP64 / pair staging row when used).
template <typename T> int rows_per_cta(int n, size_t extra_per_elem, int budget_kb = 64) {
    const size_t per_row = (2 * sizeof(T) + extra_per_elem) * (size_t)(n >= 2 ? n : 2);
    int rpc = (int)(((size_t)(budget_kb > 0 ? budget_kb : 64) * 1024) / per_row);
    if (rpc < 1) rpc = 1;
    if (rpc > 16) rpc = 16;
    return rpc;
}

// z tiles: P threads per mode (segments of the z line), tm modes per CTA and
// the register bound maxm on the rows of a segment (register-pivot kernel);
// at most 256 threads and about 100 KB of shared memory per CTA.
template <typename T> bool choose_zt(int nz, int& tm, int& P, int& maxm, int& warp_mode, int fw = 0, int fm = 0) {
    // default: warp-per-segment kernel, P = ceil(nz / maxm) warps of 32 modes
    warp_mode = 0;
    {
        // measured on GB300: 16-row segments up to nz = 256, then 32 (P <= 16 warps)
        int mm = nz <= 256 ? 16 : (nz <= 512 ? 32 : 64);
        int pw = (nz + mm - 1) / mm;
        if ((fm == 16 || fm == 32 || fm == 64) && fw >= 1 && fw <= 16 && (nz + fw - 1) / fw <= fm) {
            pw = fw;
            mm = fm;
        }
        const char* ov = getenv("CALES_ZTILE");
        int a = 0, b = 0, c = 0;
        if (ov && sscanf(ov, "w,%d,%d", &b, &c) == 2 && (c == 16 || c == 32 || c == 64) && b >= 1 && b <= 16) {
            pw = b; mm = c;
        } else if (ov && sscanf(ov, "%d,%d,%d", &a, &b, &c) >= 2) {
            pw = 0;
        }
        if (pw >= 1 && pw <= 16 && (nz + pw - 1) / pw <= mm && zsolve_w_smem<T>(nz, pw) <= 200 * 1024) {
            warp_mode = 1; P = pw; maxm = mm; tm = 32;
            return true;
        }
    }
    if (nz <= 16) { P = 1; maxm = 16; }
    else if (nz <= 32) { P = 2; maxm = 16; }
    else if (nz <= 64) { P = 4; maxm = 16; }
    else if (nz <= 128) { P = 8; maxm = 16; }
    else if (nz <= 256) { P = 8; maxm = 32; }
    else if (nz <= 512) { P = 8; maxm = 64; }
    else if (nz <= 1024) { P = 16; maxm = 64; }
    else { P = 16; maxm = 0; }
    if (sizeof(T) == 8 && maxm == 64) { P = 16; maxm = 32; if (nz > 512) maxm = 64; }
    tm = 128 / P;
    if (const char* ov = getenv("CALES_ZTILE")) {       // "tm,P,maxm" (tuning sweeps)
        int a = 0, b = 0, c = 0;
        const int n = sscanf(ov, "%d,%d,%d", &a, &b, &c);
        if (n >= 2 && a >= 1 && (b == 1 || b == 2 || b == 4 || b == 8 || b == 16) && a * b <= 256) {
            tm = a; P = b;
            maxm = n == 3 ? c : 0;
        }
    }
    const int m = (nz + P - 1) / P;
    if (maxm > 0 && m > maxm) maxm = 0;
    auto smem = [&](int t) { return maxm > 0 ? zsolve_reg_smem<T>(nz, t, P) : zsolve_smem<T>(nz, t, P); };
    const int tm_min = (int)(16 / sizeof(T));
    while (tm > tm_min && smem(tm) > 100 * 1024) tm /= 2;
    while (tm > 1 && smem(tm) > 200 * 1024) tm /= 2;
    return smem(tm) <= 200 * 1024;
}

// y tiles: the widest tile (<= 32 columns, 128-byte rows) whose two buffers
// fit in ~72 KB.  Short FP32 columns (L x 32 < 2048 complex elements, i.e.
// ny < 128) take up to 128 columns so that the first radix pass keeps most
// of the 256 threads busy, but no more columns than the row (rounded up to
// 32); ny = 128 and longer keep 32 (the compile-time-size kernels).
// ny: real elements of one FFT line (2L); nx: row length (0: unknown).
template <typename T> int choose_tx(int ny, int forced = 0, int nx = 0) {
    const int cands[6] = {128, 64, 32, 16, 8, 4};
    const size_t per_col = 2 * (size_t)(ny >= 2 ? ny : 2) * sizeof(T);
    for (int c : cands)
        if (forced == c && per_col * c <= 200 * 1024 && c * sizeof(T) >= 16) return forced;
    int widest = 32;
    if (sizeof(T) == 4) {
        const long L = ny / 2 > 0 ? ny / 2 : 1;
        const int rowcap = nx > 0 ? ((nx + 31) / 32) * 32 : 128;
        while (widest < 128 && L * widest < 2048 && widest * 2 <= rowcap) widest *= 2;
    }
    for (int c : cands)
        if (c <= widest && per_col * c <= 72 * 1024 && (c * sizeof(T) <= 128 || sizeof(T) == 4)) return c;
    for (int i = 2; i < 6; ++i)
        if (per_col * cands[i] <= 200 * 1024) return cands[i];
    return 0;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// The persistent double-buffered z kernel replaces the one-tile-per-CTA
// kernel only with CALES_ZPERSIST=1: measured on GB300 at 1536 x 512 x 512
// (FP32, 16 segments of 32 rows) it took 1.55 ms per launch against 0.87 ms,
// since one resident CTA per SM leaves the serial segment chains and the
// tile copies unhidden.
static bool zpersist_enabled() {
    static const bool on = [] {
        const char* e = getenv("CALES_ZPERSIST");
        return e && e[0] == '1';
    }();
    return on;
}

// Argument blocks of the stages of one pass: in (TIn) -> work (T, mode
// space) -> out (MODE).  Shared by the single-solve pipeline and the grouped
// batch executor.
template <typename T, typename TIn>
RowArgs<T> fwd_row_args(cales_plan_s* P, const void* in, T* work) {
    RowArgs<T> ra;
    ra.t = P->X.tab<T>();
    ra.in = in;
    ra.out = work;
    ra.nrows = (long)P->ny * P->nz;
    ra.rpc = rows_per_cta<T>(2 * P->X.L, 0, P->sched[0]);
    ra.in_scale = 1.0;
    ra.shift_acc = nullptr;
    ra.shift_scale = 0.0;
    ra.status = P->status;
    const size_t in_size = std::is_same<TIn, RUIn>::value ? sizeof(T) : sizeof(TIn);
    ra.bulk = (aligned16(in) && aligned16(work) && ((size_t)P->nx * in_size) % 16 == 0 &&
               ((size_t)P->nx * sizeof(T)) % 16 == 0) ? 1 : 0;
    ra.dout = nullptr;
    ra.gacc = nullptr;
    ra.gw = P->dzf_d;
    ra.ny = P->ny;
    ra.nymag = div_magic((unsigned)P->ny);
    return ra;
}

template <typename T>
ColArgs<T> col_args(cales_plan_s* P, T* work) {
    ColArgs<T> ca;
    ca.t = P->Y.tab<T>();
    ca.data = work;
    ca.nx = P->nx;
    ca.nplanes = P->nz;
    ca.tx = choose_tx<T>(2 * P->Y.L, P->sched[1], P->nx);
    ca.bulk = (aligned16(work) && ((size_t)P->nx * sizeof(T)) % 16 == 0 && ca.tx * sizeof(T) >= 16) ? 1 : 0;
    ca.status = P->status;
    return ca;
}

// z stage; the pivot-cache mode is chosen from the plan's cache key, which
// z_args_done updates once the launch is enqueued.
template <typename T>
ZArgs<T> z_args(cales_plan_s* P, T* work, const PassOpt& o) {
    ZArgs<T> za;
    za.data = work;
    za.src = nullptr;
    za.lamx = sizeof(T) == 8 ? (const T*)P->X.lam_d : (const T*)P->X.lam_f;
    za.lamy = sizeof(T) == 8 ? (const T*)P->Y.lam_d : (const T*)P->Y.lam_f;
    za.za = sizeof(T) == 8 ? (const T*)P->za_d : (const T*)P->za_f;
    za.zc = sizeof(T) == 8 ? (const T*)P->zc_d : (const T*)P->zc_f;
    za.dzf = P->dzf_d;
    za.nx = P->nx; za.ny = P->ny; za.nz = P->nz;
    za.zlo = P->bc[4]; za.zhi = P->bc[5];
    za.singular = o.singular ? 1 : 0;
    za.adjoint = o.adjoint ? 1 : 0;
    choose_zt<T>(P->nz, za.tm, za.P, za.maxm, za.warp_mode, P->sched[2], P->sched[3]);
    za.bulk = (aligned16(work) && ((size_t)P->nx * P->ny * sizeof(T)) % 16 == 0 && (za.tm * sizeof(T)) % 16 == 0) ? 1 : 0;
    za.sigma = T(o.sigma); za.alpha = T(o.alpha); za.scale = T(o.scale);
    za.status = P->status;
    za.cacc = o.cacc;
    za.cacc_scale = 1.0 / (o.scale * (double)P->nx * (double)P->ny);
    za.ecache = nullptr;
    za.ecache_mode = 0;
    const int zi = sizeof(T) == 8 ? 1 : 0;
    cales_plan_s::ZCacheKey& zk = P->zkey[zi];
    if (za.warp_mode && za.P <= 16 && P->zcache[zi] && P->bc[4] != CALES_BC_P) {
        za.ecache = reinterpret_cast<T*>(P->zcache[zi]);
        za.ecache_mode = (zk.valid && zk.P == za.P && zk.maxm == za.maxm && zk.sigma == o.sigma &&
                          zk.alpha == o.alpha) ? 2 : 1;
    }
    za.ecache_stride = (long)P->nx * P->ny;
    za.persist = (zpersist_enabled() || P->sched[5] == 1) ? 1 : 0;
    // the gauge shift of the last refinement sweep is applied to the mode
    // (0, 0) line here: a constant in mode space (0, 0) is the same constant
    // at every point after the unnormalised inverse transforms
    za.shift_acc = o.shift_acc;
    za.shift_scale = o.shift_scale;
    return za;
}

template <typename T>
void z_args_done(cales_plan_s* P, const ZArgs<T>& za, const PassOpt& o) {
    if (za.ecache_mode == 1) {
        cales_plan_s::ZCacheKey& zk = P->zkey[sizeof(T) == 8 ? 1 : 0];
        zk.valid = 1; zk.P = za.P; zk.maxm = za.maxm; zk.sigma = o.sigma; zk.alpha = o.alpha;
    }
}

template <typename T, int MODE>
RowArgs<T> inv_row_args(cales_plan_s* P, T* work, void* out, const PassOpt& o) {
    RowArgs<T> ri = fwd_row_args<T, T>(P, work, work);
    ri.in = work;
    ri.out = out;
    ri.bulk = (aligned16(work) && aligned16(out) && ((size_t)P->nx * sizeof(T)) % 16 == 0 &&
               ((size_t)P->nx * 8) % 16 == 0) ? 1 : 0;
    ri.shift_acc = nullptr;          // applied by the z solve (z_args)
    ri.shift_scale = 0.0;
    return ri;
}

// One pass of the solver: in (TIn) -> work (T, mode space) -> out (MODE).
// OUT_FF_ACC_D: the inverse x pass also stores the correction into work
// (its own input rows) and adds the gauge sum of the updated pairs to gacc.
// TIn = RUIn: the forward x pass forms its rows as the residual update *ru
// (the fused fast-mode update; `in` unused).
template <typename T, typename TIn, int MODE>
int pipeline(cales_plan_s* P, const void* in, void* out, T* work, const PassOpt& o, cudaStream_t st,
             double* gacc = nullptr, const ResidUpdArgs* ru = nullptr) {
    RowArgs<T> ra = fwd_row_args<T, TIn>(P, in, work);
    if constexpr (std::is_same<TIn, RUIn>::value) ra.ru = *ru;
    P->prof_begin(st, std::is_same<TIn, RUIn>::value ? "x_fwd_ru" : "x_fwd");
    if (launch_rows_forward<T, TIn>(ra, st) != cudaSuccess) return CALES_ECUDA;
    P->prof_end(st);

    const ColArgs<T> ca = col_args<T>(P, work);
    if (P->ny > 1) {
        P->prof_begin(st, "y_fwd");
        if (launch_cols<T>(ca, false, st) != cudaSuccess) return CALES_ECUDA;
        P->prof_end(st);
    }

    ZArgs<T> za = z_args<T>(P, work, o);
    P->prof_begin(st, "z_solve");
    if (P->bc[4] == CALES_BC_P) {
        T* ework = reinterpret_cast<T*>(P->zcyc);
        if (launch_zsolve_cyclic<T>(za, ework, ework + (size_t)P->nx * P->ny * P->nz, st) != cudaSuccess)
            return CALES_ECUDA;
    } else if (launch_zsolve<T>(za, st) != cudaSuccess) {
        return CALES_ECUDA;
    }
    z_args_done<T>(P, za, o);
    P->prof_end(st);

    if (P->ny > 1) {
        P->prof_begin(st, "y_inv");
        if (launch_cols<T>(ca, true, st) != cudaSuccess) return CALES_ECUDA;
        P->prof_end(st);
    }

    RowArgs<T> ri = inv_row_args<T, MODE>(P, work, out, o);
    if (MODE == OUT_FF_ACC_D) {
        ri.dout = work;
        ri.gacc = gacc;
    }
    P->prof_begin(st, MODE >= OUT_FF_ACC ? "x_inv_acc" : "x_inv");
    if (launch_rows_inverse<T, MODE>(ri, st) != cudaSuccess) return CALES_ECUDA;
    P->prof_end(st);
    return CALES_OK;
}

}  // namespace cales

// ---------------------------------------------------------------------------
// profiling hooks (CUDA events around each launch when enabled)
// ---------------------------------------------------------------------------
void cales_plan_s::prof_begin(cudaStream_t st, const char* name) {
    if (!prof_on || prof_n >= PROF_MAX) return;
    ProfRec& r = prof[prof_n];
    if (!r.a) { cudaEventCreate(&r.a); cudaEventCreate(&r.b); }
    r.name = name;
    cudaEventRecord(r.a, st);
}

void cales_plan_s::prof_end(cudaStream_t st) {
    if (!prof_on || prof_n >= PROF_MAX) return;
    cudaEventRecord(prof[prof_n].b, st);
    ++prof_n;
}

namespace cales {

PassOpt solve_opts(const cales_plan_s* P, bool helm, double alpha, bool adjoint) {
    const double nxy = (double)P->nx * (double)P->ny;
    PassOpt o;
    o.sigma = helm ? 1.0 : 0.0;
    o.alpha = helm ? alpha : 1.0;
    o.scale = (helm ? 1.0 : -1.0) / nxy;
    o.singular = !helm && P->singular_poisson;
    o.adjoint = adjoint;
    o.cacc = nullptr;
    o.shift_acc = nullptr;
    o.shift_scale = 0.0;
    return o;
}

// Residual of sweep s (of ns) of the refinement: r = f - cacc - M p with p
// held as pairs; the gauge sum into gacc on the last sweep of a singular
// problem (the operator annihilates constants, so earlier iterates may
// carry any mean).
ResidFFArgs resid_args(const cales_plan_s* P, bool helm, double alpha, const void* f, void* p, float* work,
                       double* cacc, double* gacc, int s, int ns) {
    const bool sing = !helm && P->singular_poisson;
    const double c1 = helm ? -alpha : 1.0;
    ResidFFArgs ra;
    ra.f = (const double*)f;
    ra.u = (const float2*)p;
    ra.r = work;
    ra.nx = P->nx; ra.ny = P->ny; ra.nz = P->nz;
    ra.bcx = P->X.kind; ra.bcy = P->Y.kind; ra.zlo = P->bc[4]; ra.zhi = P->bc[5];
    split_double(c1 / (P->dx * P->dx), ra.cxh, ra.cxl);
    split_double(c1 / (P->dy * P->dy), ra.cyh, ra.cyl);
    ra.c0h = helm ? 1.0f : 0.0f;
    ra.za = P->za_d;
    ra.zc = P->zc_d;
    ra.c1 = c1;
    ra.cshift = sing ? cacc : nullptr;
    ra.gacc = (sing && s == ns - 1) ? gacc : nullptr;
    ra.dzf = P->dzf_d;
    ra.lo_zero = s == 0 ? 1 : 0;       // the FP32 solve wrote (v, 0) pairs
    ra.rows_per_cta = residual_rows_per_cta(P->nx, P->ny);
    return ra;
}

template RowArgs<float> fwd_row_args<float, double>(cales_plan_s*, const void*, float*);
template RowArgs<float> fwd_row_args<float, float>(cales_plan_s*, const void*, float*);
template ColArgs<float> col_args<float>(cales_plan_s*, float*);
template ZArgs<float> z_args<float>(cales_plan_s*, float*, const PassOpt&);
template void z_args_done<float>(cales_plan_s*, const ZArgs<float>&, const PassOpt&);
template RowArgs<float> inv_row_args<float, OUT_F64>(cales_plan_s*, float*, void*, const PassOpt&);
template RowArgs<float> inv_row_args<float, OUT_FF_INIT>(cales_plan_s*, float*, void*, const PassOpt&);
template RowArgs<float> inv_row_args<float, OUT_FF_ACC>(cales_plan_s*, float*, void*, const PassOpt&);
template RowArgs<float> inv_row_args<float, OUT_FF_FINAL>(cales_plan_s*, float*, void*, const PassOpt&);

}  // namespace cales

// FP32 solves with double-float refinement.  While sweeping, the caller's
// FP64 output buffer holds the solution as (hi, lo) float pairs; the last
// sweep writes it back as doubles.  For a singular Poisson problem the
// consistency constant of f is estimated from the first mode-space solve and
// refined by every sweep (acc[0]); the dzf-weighted mean of the solution is
// measured by each residual pass (acc[1]) and removed by the same sweep.
// work: one FP32 field (mode space and residual); acc: two FP64 accumulators.
static int refine_solve(cales_plan_t P, bool helm, double alpha, const void* f, void* p, PassOpt o, float* work,
                        double* acc, cudaStream_t st) {
    const int ns = P->sweeps;
    const bool sing = o.singular;
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(double), st) != cudaSuccess) return CALES_ECUDA;
    o.cacc = sing ? acc : nullptr;
    int rc = ns == 0 ? pipeline<float, double, OUT_F64>(P, f, p, work, o, st)
                     : pipeline<float, double, OUT_FF_INIT>(P, f, p, work, o, st);
    if (rc) return rc;
    for (int s = 0; s < ns; ++s) {
        if (sing && cudaMemsetAsync(acc + 1, 0, sizeof(double), st) != cudaSuccess) return CALES_ECUDA;
        const ResidFFArgs ra = resid_args(P, helm, alpha, f, p, work, acc, acc + 1, s, ns);
        P->prof_begin(st, "residual");
        if (launch_residual_ff(ra, st) != cudaSuccess) return CALES_ECUDA;
        P->prof_end(st);
        o.shift_acc = (sing && s == ns - 1) ? acc + 1 : nullptr;
        o.shift_scale = 1.0 / ((double)P->nx * (double)P->ny * P->dzf_sum);
        rc = (s == ns - 1) ? pipeline<float, float, OUT_FF_FINAL>(P, work, p, work, o, st)
                           : pipeline<float, float, OUT_FF_ACC>(P, work, p, work, o, st);
        if (rc) return rc;
    }
    return CALES_OK;
}

// The last residual update of the fast refinement fused into the forward x
// transform of the last solve: only with CALES_FUSE_RU=1.  It saves the 8
// bytes per point of writing and re-reading the updated residual, but on
// GB300 at 1536 x 512 x 512 the fused pass took 1.66 ms against 1.42 ms for
// the update (0.73 ms, 96 % of the copy bandwidth at 64 warps per SM) and the
// transform (0.69 ms) apart: inside the transform's CTAs (73 KB of shared
// memory, 24 warps per SM) the update's neighbour loads are not hidden, and
// fewer rows per CTA did not help (1.69 ms with 2 rows, 2.26 ms with 1).
// Needs rows of a multiple of 4 points and 16-byte aligned fields.
static bool fuse_residual_update(cales_plan_t P, const ResidUpdArgs& ua) {
    static const bool on = [] {
        const char* e = getenv("CALES_FUSE_RU");
        return e && e[0] == '1';
    }();
    if (!on) return false;
    RowArgs<float> ra = fwd_row_args<float, RUIn>(P, nullptr, ua.r);
    ra.ru = ua;
    return rows_forward_ru_ok(ra);
}

// Fast refinement: the residual is formed in double-float once, after the
// first FP32 solve; every later sweep updates it in FP32 from the correction
// of the sweep before, r_{s+1} = r_s - M d_s (the inverse x pass stores d_s
// beside the pair update), and subtracts the change of the consistency
// constant (acc[0] - acc[2]) for a singular problem.  The gauge of the
// solution is measured by the pair update of the last-but-one sweep (acc[1])
// and removed by the last one.  work: mode space and corrections; res: the
// residual field.
static int refine_solve_fast(cales_plan_t P, bool helm, double alpha, const void* f, void* p, PassOpt o,
                             float* work, float* res, double* acc, cudaStream_t st) {
    const int ns = P->sweeps;
    const bool sing = o.singular;
    if (ns <= 1) return CALES_EINVAL;
    if (cudaMemsetAsync(acc, 0, 4 * sizeof(double), st) != cudaSuccess) return CALES_ECUDA;
    o.cacc = sing ? acc : nullptr;
    int rc = pipeline<float, double, OUT_FF_INIT>(P, f, p, work, o, st);
    if (rc) return rc;
    if (sing && cudaMemcpyAsync(acc + 2, acc, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return CALES_ECUDA;
    const ResidFFArgs ra = resid_args(P, helm, alpha, f, p, res, acc, nullptr, 0, ns);
    P->prof_begin(st, "residual");
    if (launch_residual_ff(ra, st) != cudaSuccess) return CALES_ECUDA;
    P->prof_end(st);
    ResidUpdArgs ua;
    ua.r = res;
    ua.d = work;
    ua.nx = P->nx; ua.ny = P->ny; ua.nz = P->nz;
    ua.bcx = P->X.kind; ua.bcy = P->Y.kind; ua.zlo = P->bc[4]; ua.zhi = P->bc[5];
    const double c1 = helm ? -alpha : 1.0;
    ua.cx = (float)(c1 / (P->dx * P->dx));
    ua.cy = (float)(c1 / (P->dy * P->dy));
    ua.c0 = helm ? 1.f : 0.f;
    ua.c1 = (float)c1;
    ua.za = P->za_f;
    ua.zc = P->zc_f;
    ua.acc = sing ? acc : nullptr;
    for (int s = 0; s < ns; ++s) {
        const bool last = s == ns - 1;
        if (last && fuse_residual_update(P, ua)) {
            // the last update fused into the forward x pass: the update of
            // each row is formed in shared memory and transformed there, the
            // transformed rows overwrite the residual (this pass reads only
            // its own rows of it), which then serves as the solve's workspace
            o.shift_acc = sing ? acc + 1 : nullptr;
            o.shift_scale = 1.0 / ((double)P->nx * (double)P->ny * P->dzf_sum);
            rc = pipeline<float, RUIn, OUT_FF_FINAL>(P, nullptr, p, res, o, st, nullptr, &ua);
            if (rc) return rc;
            continue;
        }
        if (s > 0) {
            P->prof_begin(st, "residual_update");
            if (launch_residual_update(ua, st) != cudaSuccess) return CALES_ECUDA;
            P->prof_end(st);
            if (sing && cudaMemcpyAsync(acc + 2, acc, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return CALES_ECUDA;
        }
        if (last) {
            o.shift_acc = sing ? acc + 1 : nullptr;
            o.shift_scale = 1.0 / ((double)P->nx * (double)P->ny * P->dzf_sum);
            rc = pipeline<float, float, OUT_FF_FINAL>(P, res, p, work, o, st);
        } else {
            // the gauge of the solution that the last correction updates
            if (sing && s == ns - 2 && cudaMemsetAsync(acc + 1, 0, sizeof(double), st) != cudaSuccess)
                return CALES_ECUDA;
            PassOpt od = o;
            od.shift_acc = nullptr;
            rc = pipeline<float, float, OUT_FF_ACC_D>(P, res, p, work, od, st, (sing && s == ns - 2) ? acc + 1 : nullptr);
        }
        if (rc) return rc;
    }
    return CALES_OK;
}

static int solve_common(cales_plan_t P, bool helm, double alpha, bool adjoint, const void* f, void* p, void* stream);

int cales_internal_solve(cales_plan_s* P, bool helm, double alpha, bool adjoint, const void* f, void* p,
                         void* stream) {
    return solve_common(P, helm, alpha, adjoint, f, p, stream);
}

static int solve_common(cales_plan_t P, bool helm, double alpha, bool adjoint, const void* f, void* p, void* stream) {
    if (!P || !f || !p) return CALES_EINVAL;
    if (helm && !(alpha > 0.0)) return CALES_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const PassOpt o = solve_opts(P, helm, alpha, adjoint);
    switch (P->precision) {
        case CALES_FP64:
            return pipeline<double, double, OUT_T>(P, f, p, (double*)p, o, st);
        case CALES_FP32:
            return pipeline<float, float, OUT_T>(P, f, p, (float*)p, o, st);
        case CALES_FP32_REFINE:
            if (adjoint) return CALES_EUNSUPPORTED;
            if (f == p || !P->work) return CALES_EINVAL;
            return refine_solve(P, helm, alpha, f, p, o, P->work, P->acc, st);
        case CALES_FP32_REFINE_FAST:
            if (adjoint) return CALES_EUNSUPPORTED;
            if (f == p || !P->work || !P->work2) return CALES_EINVAL;
            if (P->sweeps <= 1) return refine_solve(P, helm, alpha, f, p, o, P->work, P->acc, st);
            return refine_solve_fast(P, helm, alpha, f, p, o, P->work, P->work2, P->acc, st);
        default:
            return CALES_EINVAL;
    }
}

void cales_plan_s::fill_resid(cales::ResidArgs& ra, const double* u, const double* f, void* r, bool r_double,
                              double c0, double c1) const {
    ra.u = u;
    ra.f = f;
    ra.r = r;
    ra.r_is_double = r_double ? 1 : 0;
    ra.nx = nx; ra.ny = ny; ra.nz = nz;
    ra.bcx = X.kind; ra.bcy = Y.kind; ra.zlo = bc[4]; ra.zhi = bc[5];
    ra.idx2 = 1.0 / (dx * dx);
    ra.idy2 = 1.0 / (dy * dy);
    ra.za = za_d;
    ra.zc = zc_d;
    ra.c0 = c0;
    ra.c1 = c1;
    ra.fshift = 0.0;
}

// Line solves of the wall-normal implicit step (Eq. 21): the z kernel on the
// physical field with every eigenvalue zero and no transform scaling.
template <typename T>
static int z_lines(cales_plan_t P, double alpha, const T* f, T* u, cudaStream_t st) {
    ZArgs<T> za;
    za.data = u;
    za.src = f;
    za.lamx = sizeof(T) == 8 ? (const T*)P->zero_d : (const T*)P->zero_f;
    za.lamy = za.lamx;
    za.za = sizeof(T) == 8 ? (const T*)P->za_d : (const T*)P->za_f;
    za.zc = sizeof(T) == 8 ? (const T*)P->zc_d : (const T*)P->zc_f;
    za.dzf = P->dzf_d;
    za.nx = P->nx; za.ny = P->ny; za.nz = P->nz;
    za.zlo = P->bc[4]; za.zhi = P->bc[5];
    za.singular = 0;
    za.adjoint = 0;
    choose_zt<T>(P->nz, za.tm, za.P, za.maxm, za.warp_mode, P->sched[2], P->sched[3]);
    za.bulk = (aligned16(u) && aligned16(f) && ((size_t)P->nx * P->ny * sizeof(T)) % 16 == 0 &&
               (za.tm * sizeof(T)) % 16 == 0) ? 1 : 0;
    za.sigma = T(1); za.alpha = T(alpha); za.scale = T(1);
    za.status = P->status;
    za.cacc = nullptr;
    za.cacc_scale = 0.0;
    za.ecache = nullptr;
    za.ecache_mode = 0;
    za.ecache_stride = 0;
    za.persist = (zpersist_enabled() || P->sched[5] == 1) ? 1 : 0;
    za.shift_acc = nullptr;
    za.shift_scale = 0.0;
    const int zi = sizeof(T) == 8 ? 1 : 0;
    cales_plan_s::ZCacheKey& lk = P->lkey[zi];
    if (za.warp_mode && za.P <= 16 && P->lcache[zi]) {
        za.ecache = reinterpret_cast<T*>(P->lcache[zi]);
        za.ecache_mode = (lk.valid && lk.P == za.P && lk.maxm == za.maxm && lk.alpha == alpha) ? 2 : 1;
    }
    if (P->bc[4] == CALES_BC_P) {
        // periodic z: one cyclic system per line (no eigenvalues, sigma 1),
        // in place on u
        if (f != u && cudaMemcpyAsync(u, f, (size_t)P->nx * P->ny * P->nz * sizeof(T), cudaMemcpyDeviceToDevice,
                                      st) != cudaSuccess)
            return CALES_ECUDA;
        za.src = nullptr;
        T* ework = reinterpret_cast<T*>(P->zcyc);
        P->prof_begin(st, "z_lines");
        if (launch_zsolve_cyclic<T>(za, ework, ework + (size_t)P->nx * P->ny * P->nz, st) != cudaSuccess)
            return CALES_ECUDA;
        P->prof_end(st);
        return CALES_OK;
    }
    if (!za.warp_mode) {
        // the other z kernels work in place
        if (f != u && cudaMemcpyAsync(u, f, (size_t)P->nx * P->ny * P->nz * sizeof(T), cudaMemcpyDeviceToDevice,
                                      st) != cudaSuccess)
            return CALES_ECUDA;
        za.src = nullptr;
    }
    P->prof_begin(st, "z_lines");
    if (launch_zsolve<T>(za, st) != cudaSuccess) return CALES_ECUDA;
    P->prof_end(st);
    if (za.ecache_mode == 1) {
        lk.valid = 1; lk.P = za.P; lk.maxm = za.maxm; lk.sigma = 1.0; lk.alpha = alpha;
    }
    return CALES_OK;
}

// Segment-entry pivot cache of one precision: 16 slots per mode (the largest
// segment count of the z kernel).  Left out when the allocation fails.
static void alloc_zcache(cales_plan_s* P, int zi) {
    if (P->zcache[zi]) return;
    const size_t bytes = (size_t)P->nx * P->ny * 16 * (zi ? sizeof(double) : sizeof(float));
    void* m = nullptr;
    if (cudaMalloc(&m, bytes) == cudaSuccess) P->zcache[zi] = m;
    else cudaGetLastError();
    P->zkey[zi].valid = 0;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int cales_plan(cales_plan_t* out, int nx, int ny, int nz, const int bc[6], double dx, double dy,
               const double* dzc, const double* dzf) {
    if (!out || !bc || !dzc || !dzf) return CALES_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0)) return CALES_EINVAL;
    if ((long)nx * ny * nz > (1L << 34)) return CALES_EINVAL;
    for (int i = 0; i < 6; ++i)
        if (bc[i] < 0 || bc[i] > 3) return CALES_EINVAL;
    // transform kind of each uniform direction: both sides alike, or mixed
    // Neumann / Dirichlet cell sides (DCT-IV / DST-IV); periodic pairs only
    // with periodic
    int dkind[2];
    for (int d = 0; d < 2; ++d) {
        const int lo = bc[2 * d], hi = bc[2 * d + 1];
        if ((lo == CALES_BC_P) != (hi == CALES_BC_P)) return CALES_EINVAL;
        if (lo == hi) dkind[d] = lo;
        else if (lo == CALES_BC_N && hi == CALES_BC_D) dkind[d] = KIND_ND;
        else if (lo == CALES_BC_D && hi == CALES_BC_N) dkind[d] = KIND_DN;
        else return CALES_EUNSUPPORTED;
    }
    if ((bc[4] == CALES_BC_P) != (bc[5] == CALES_BC_P)) return CALES_EINVAL;
    if (bc[4] == CALES_BC_P && nz < 3) return CALES_EUNSUPPORTED;
    for (int k = 0; k <= nz; ++k)
        if (!(dzc[k] > 0) || !std::isfinite(dzc[k])) return CALES_EINVAL;
    for (int k = 0; k < nz; ++k)
        if (!(dzf[k] > 0) || !std::isfinite(dzf[k])) return CALES_EINVAL;
    // periodic z: dzc[0] and dzc[nz] are the same wrap-around distance; the
    // operator only telescopes under dzf weighting when they agree
    if (bc[4] == CALES_BC_P && std::fabs(dzc[0] - dzc[nz]) > 1e-12 * dzc[0]) return CALES_EINVAL;

    cales_plan_s* P = new (std::nothrow) cales_plan_s();
    if (!P) return CALES_ENOMEM;
    P->nx = nx; P->ny = ny; P->nz = nz;
    for (int i = 0; i < 6; ++i) P->bc[i] = bc[i];
    P->dx = dx; P->dy = dy;
    // singular: no Dirichlet condition anywhere (x, y sides periodic or Neumann)
    P->singular_poisson = ((dkind[0] == KIND_P || dkind[0] == KIND_N) && (dkind[1] == KIND_P || dkind[1] == KIND_N) &&
                           (bc[4] == CALES_BC_N || bc[4] == CALES_BC_P) && (bc[5] == CALES_BC_N || bc[5] == CALES_BC_P))
                              ? 1 : 0;
    int rc = build_dir(P->X, nx, dkind[0], dx, P->owned);
    if (rc == CALES_OK) rc = build_dir(P->Y, ny, dkind[1], dy, P->owned);
    if (rc == CALES_OK) {
        int tm_, p_, mm_, wm_;
        const int ex = 2 * P->X.L, ey = 2 * P->Y.L;       // real elements of one FFT buffer line
        if (rows_per_cta<double>(ex, 0) < 1 || 2.0 * ex * sizeof(double) > 200.0 * 1024 ||
            !choose_zt<double>(nz, tm_, p_, mm_, wm_) || choose_tx<double>(ey) == 0)
            rc = CALES_EUNSUPPORTED;
    }
    if (rc == CALES_OK) {
        std::vector<double> za(nz), zc(nz), df(dzf, dzf + nz);
        std::vector<float> zaf(nz), zcf(nz);
        for (int k = 0; k < nz; ++k) {
            za[k] = 1.0 / (dzc[k] * dzf[k]);
            zc[k] = 1.0 / (dzc[k + 1] * dzf[k]);
            zaf[k] = (float)za[k];
            zcf[k] = (float)zc[k];
        }
        P->za_d = dev_upload(za, P->owned);
        P->zc_d = dev_upload(zc, P->owned);
        P->dzf_d = dev_upload(df, P->owned);
        P->za_f = dev_upload(zaf, P->owned);
        P->zc_f = dev_upload(zcf, P->owned);
        std::vector<int> st(4, 0);
        P->status = dev_upload(st, P->owned);
        std::vector<double> idzf(nz), idzc(nz + 1);
        std::vector<float> idzff(nz), idzcf(nz + 1);
        for (int k = 0; k < nz; ++k) { idzf[k] = 1.0 / dzf[k]; idzff[k] = (float)idzf[k]; }
        for (int k = 0; k <= nz; ++k) { idzc[k] = 1.0 / dzc[k]; idzcf[k] = (float)idzc[k]; }
        P->idzf_d = dev_upload(idzf, P->owned);
        P->idzc_d = dev_upload(idzc, P->owned);
        P->idzf_f = dev_upload(idzff, P->owned);
        P->idzc_f = dev_upload(idzcf, P->owned);
        std::vector<double> acc(4, 0.0);
        P->acc = dev_upload(acc, P->owned);
        std::vector<double> zcen(nz);
        double zacc = 0.0;
        for (int k = 0; k < nz; ++k) { zcen[k] = zacc + 0.5 * dzf[k]; zacc += dzf[k]; }
        P->zcen_d = dev_upload(zcen, P->owned);
        P->sgs_coef = dev_upload(std::vector<double>(nz, 0.0), P->owned);
        if (bc[4] == CALES_BC_P) {
            if (cudaMalloc(&P->zcyc, 2 * (size_t)nx * ny * nz * sizeof(double)) == cudaSuccess) P->owned.push_back(P->zcyc);
            else P->zcyc = nullptr;
            if (!P->zcyc) rc = CALES_ENOMEM;
        }
        const int nzero = nx > ny ? nx : ny;
        P->zero_d = dev_upload(std::vector<double>(nzero, 0.0), P->owned);
        P->zero_f = dev_upload(std::vector<float>(nzero, 0.0f), P->owned);
        P->lcache[1] = dev_upload(std::vector<double>(16, 0.0), P->owned);
        P->lcache[0] = dev_upload(std::vector<float>(16, 0.0f), P->owned);
        P->dzf_sum = 0.0;
        for (int k = 0; k < nz; ++k) P->dzf_sum += dzf[k];
        if (!P->za_d || !P->zc_d || !P->dzf_d || !P->za_f || !P->zc_f || !P->status || !P->acc || !P->idzf_d ||
            !P->idzc_d || !P->idzf_f || !P->idzc_f || !P->zero_d || !P->zero_f || !P->zcen_d ||
            !P->sgs_coef)
            rc = CALES_ENOMEM;
    }
    if (rc == CALES_OK && cudaDeviceSynchronize() != cudaSuccess) rc = CALES_ECUDA;
    if (rc != CALES_OK) {
        cales_destroy(P);
        return rc;
    }
    P->precision = CALES_FP64;
    P->sweeps = 2;
    alloc_zcache(P, 1);
    const char* pe = getenv("CALES_PROFILE");
    P->prof_on = pe && pe[0] == '1';
    *out = P;
    return CALES_OK;
}

int cales_set_precision(cales_plan_t P, int mode, int sweeps) {
    if (!P || mode < 0 || mode > 3 || sweeps < 0 || sweeps > 8) return CALES_EINVAL;
    const size_t bytes = (size_t)P->nx * P->ny * P->nz * sizeof(float);
    if ((mode == CALES_FP32_REFINE || mode == CALES_FP32_REFINE_FAST) && !P->work) {
        void* w = nullptr;
        if (cudaMalloc(&w, bytes) != cudaSuccess) return CALES_ENOMEM;
        P->work = reinterpret_cast<float*>(w);
    }
    if (mode == CALES_FP32_REFINE_FAST && !P->work2) {
        void* w = nullptr;
        if (cudaMalloc(&w, bytes) != cudaSuccess) return CALES_ENOMEM;
        P->work2 = reinterpret_cast<float*>(w);
    }
    P->precision = mode;
    P->sweeps = sweeps;
    alloc_zcache(P, mode == CALES_FP64 ? 1 : 0);
    return CALES_OK;
}

int cales_poisson_solve(cales_plan_t P, const void* f, void* p, void* stream) {
    return solve_common(P, false, 0.0, false, f, p, stream);
}

int cales_helmholtz_solve(cales_plan_t P, double alpha, const void* f, void* u, void* stream) {
    return solve_common(P, true, alpha, false, f, u, stream);
}

int cales_helmholtz_z_solve(cales_plan_t P, double alpha, const void* f, void* u, void* stream) {
    if (!P || !f || !u || !(alpha >= 0.0) || !std::isfinite(alpha)) return CALES_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (P->precision == CALES_FP32) return z_lines<float>(P, alpha, (const float*)f, (float*)u, st);
    return z_lines<double>(P, alpha, (const double*)f, (double*)u, st);
}

int cales_poisson_solve_adjoint(cales_plan_t P, const void* w, void* g, void* stream) {
    return solve_common(P, false, 0.0, true, w, g, stream);
}

int cales_helmholtz_solve_adjoint(cales_plan_t P, double alpha, const void* w, void* g, void* stream) {
    return solve_common(P, true, alpha, true, w, g, stream);
}

int cales_residual(cales_plan_t P, double alpha, const double* u, const double* f, double* r, void* stream) {
    if (!P || !u || !f || !r) return CALES_EINVAL;
    ResidArgs ra;
    const bool helm = alpha >= 0.0;
    P->fill_resid(ra, u, f, r, true, helm ? 1.0 : 0.0, helm ? -alpha : 1.0);
    if (launch_residual(ra, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return CALES_ECUDA;
    return CALES_OK;
}

int cales_get_status(cales_plan_t P, int* device_status) {
    if (!P || !device_status) return CALES_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return CALES_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, P->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CALES_ECUDA;
    cudaMemset(P->status, 0, sizeof(int));
    *device_status = v;
    return CALES_OK;
}

const char* cales_strerror(int code) {
    switch (code) {
        case CALES_OK: return "ok";
        case CALES_EINVAL: return "invalid argument";
        case CALES_EUNSUPPORTED: return "unsupported size or boundary combination";
        case CALES_ENOMEM: return "device allocation failed";
        case CALES_ECUDA: return "CUDA runtime error";
        case CALES_ETOOBIG: return "grid exceeds the 8388608-point static scratch of cales_poisson_solve_noalloc";
        default: return "unknown error";
    }
}

void cales_destroy(cales_plan_t P) {
    if (!P) return;
    for (void* p : P->owned) cudaFree(p);
    for (void* z : P->zcache)
        if (z) cudaFree(z);
    if (P->work) cudaFree(P->work);
    if (P->work2) cudaFree(P->work2);
    for (int i = 0; i < cales_plan_s::PROF_MAX; ++i) {
        if (P->prof[i].a) { cudaEventDestroy(P->prof[i].a); cudaEventDestroy(P->prof[i].b); }
    }
    delete P;
}

// Per-kernel timings of the last solve when profiling is on (CALES_PROFILE=1
// or cales_profile_enable).  Synchronises.  Returns the number of records.
int cales_profile_enable(cales_plan_t P, int on) {
    if (!P) return CALES_EINVAL;
    P->prof_on = on != 0;
    P->prof_n = 0;
    return CALES_OK;
}

int cales_profile_read(cales_plan_t P, int max, const char** names, float* ms) {
    if (!P) return CALES_EINVAL;
    cudaDeviceSynchronize();
    const int n = P->prof_n < max ? P->prof_n : max;
    for (int i = 0; i < n; ++i) {
        names[i] = P->prof[i].name;
        float t = 0.f;
        cudaEventElapsedTime(&t, P->prof[i].a, P->prof[i].b);
        ms[i] = t;
    }
    return n;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Poisson solve (FP32 + double-float refinement) that allocates nothing.
//
// Some callers cannot allocate device memory at solve time: code that runs
// while a CUDA stream is being captured into a graph (cudaMalloc is not
// allowed there), hosts that hand the library a fixed memory budget and fail
// any further allocation, and real-time loops that must not stall in the
// allocator.  This entry point takes its scratch (the FP32 mode-space field
// and two FP64 accumulators) from one file-scope device array instead of the
// plan's workspace, so a plan never needs cales_set_precision(FP32_REFINE).
// The array is CALES_STATIC_SCRATCH_POINTS floats plus 256 bytes; every GPU
// that loads this library holds it until the process exits.
// ---------------------------------------------------------------------------
#define CALES_STATIC_SCRATCH_POINTS (8L * 1024 * 1024)
static __device__ __align__(256) unsigned char g_static_scratch[256 + CALES_STATIC_SCRATCH_POINTS * sizeof(float)];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device (looked up once
// per device with that device current; the host symbol is not an address).
int static_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CALES_ECUDA;
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return CALES_ECUDA;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return CALES_OK;
}
}  // namespace

extern "C" int cales_poisson_solve_noalloc(cales_plan_t P, const void* f, void* p, void* stream) {
    if (!P || !f || !p || f == p) return CALES_EINVAL;
    if (P->bc[4] == CALES_BC_P) return CALES_EUNSUPPORTED;
    if ((long)P->nx * P->ny * P->nz > CALES_STATIC_SCRATCH_POINTS) return CALES_ETOOBIG;
    void* base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    double* acc = reinterpret_cast<double*>(base);
    float* work = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(base) + 256);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PassOpt o;
    o.sigma = 0.0;
    o.alpha = 1.0;
    o.scale = -1.0 / ((double)P->nx * (double)P->ny);
    o.singular = P->singular_poisson != 0;
    o.adjoint = false;
    o.cacc = nullptr;
    o.shift_acc = nullptr;
    o.shift_scale = 0.0;
    // the same refinement as cales_poisson_solve on an FP32_REFINE plan, with
    // the scratch taken from the static array (it keeps the previous call's
    // contents: refine_solve clears the accumulators itself)
    return refine_solve(P, false, 0.0, f, p, o, work, acc, st);
}

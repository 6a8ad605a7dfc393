// Kernel argument blocks and launcher declarations (internal to the library).
#pragma once
#include "common.cuh"

namespace cales {

// FP32 update of a refinement residual from the last correction d (the fast
// refinement mode): r <- r - (c0 d + c1 L d) - (acc[0] - acc[2]).
struct ResidUpdArgs {
    float* r;            // in/out [nz][ny][nx]
    const float* d;      // correction [nz][ny][nx]
    int nx, ny, nz;
    int bcx, bcy, zlo, zhi;   // KIND_* for x/y, ZBC_* (0 periodic) for z
    float cx, cy, c0, c1;     // c1/dx^2, c1/dy^2, c0 (0 or 1), c1 (1 or -alpha)
    const float* za;     // [nz] couplings 1/(dzc dzf), unscaled
    const float* zc;
    const double* acc;   // singular problems: acc[0] (current) and acc[2] (in r), else null
};

// Input tag of the forward x transform whose rows are the residual update
// above, formed in shared memory (the update fused into the transform).
struct RUIn {};

// Plane constants of the residual update (plane k): the scaled z couplings,
// the offsets of the z neighbours (periodic wrap, or the point itself at a
// wall) and their ghost multipliers.
struct RUPlane {
    float zc, za, mD, mU;
    long offD, offU;
};
__device__ __forceinline__ RUPlane ru_plane(const ResidUpdArgs& a, int k) {
    const long plane = (long)a.nx * a.ny;
    const bool pz = a.zlo == 0;
    const float gd = a.zlo == ZBC_N ? 1.f : (a.zlo == ZBC_D ? -1.f : 0.f);
    const float gu = a.zhi == ZBC_N ? 1.f : (a.zhi == ZBC_D ? -1.f : 0.f);
    RUPlane c;
    c.zc = mul_(a.c1, a.zc[k]);
    c.za = mul_(a.c1, a.za[k]);
    c.offD = k > 0 ? -plane : (pz ? (long)(a.nz - 1) * plane : 0);
    c.offU = k < a.nz - 1 ? plane : (pz ? -(long)(a.nz - 1) * plane : 0);
    c.mD = (k > 0 || pz) ? 1.f : gd;
    c.mU = (k < a.nz - 1 || pz) ? 1.f : gu;
    return c;
}

// The residual update at VW consecutive points i .. i+VW-1 of row j of plane
// k (plane constants pk): returns r - (c0 d + c1 L d) - dshift there, with the
// R2 ghosts per side and the periodic wraps.  Every product that feeds a sum
// is rounded explicitly, so the standalone update and the one fused into the
// forward x transform give the same bits.  VW = 4 needs 16-byte aligned rows.
template <int VW>
__device__ __forceinline__ void resupd_group(const ResidUpdArgs& a, const RUPlane& pk, int i, int j, int k, float dshift,
                                             float* out) {
    const int nx = a.nx, ny = a.ny;
    const bool px = a.bcx == KIND_P, py = a.bcy == KIND_P;
    const long rb = (long)k * nx * ny + (long)j * nx;
    const long offS = j > 0 ? -(long)nx : (py ? (long)(ny - 1) * nx : 0);
    const long offN = j < ny - 1 ? (long)nx : (py ? -(long)(ny - 1) * nx : 0);
    const float mS = (j > 0 || py) ? 1.f : ghost_lo(a.bcy), mN = (j < ny - 1 || py) ? 1.f : ghost_hi(a.bcy);
    const float* q = a.d + rb + i;
    float c[VW], sv[VW], nv[VW], dn[VW], up[VW], r[VW];
    if (VW == 4) {
        const float4 c4 = *reinterpret_cast<const float4*>(q), s4 = *reinterpret_cast<const float4*>(q + offS);
        const float4 n4 = *reinterpret_cast<const float4*>(q + offN), d4 = *reinterpret_cast<const float4*>(q + pk.offD);
        const float4 u4 = *reinterpret_cast<const float4*>(q + pk.offU);
        const float4 r4 = *reinterpret_cast<const float4*>(a.r + rb + i);
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        sv[0] = s4.x; sv[1] = s4.y; sv[2] = s4.z; sv[3] = s4.w;
        nv[0] = n4.x; nv[1] = n4.y; nv[2] = n4.z; nv[3] = n4.w;
        dn[0] = d4.x; dn[1] = d4.y; dn[2] = d4.z; dn[3] = d4.w;
        up[0] = u4.x; up[1] = u4.y; up[2] = u4.z; up[3] = u4.w;
        r[0] = r4.x; r[1] = r4.y; r[2] = r4.z; r[3] = r4.w;
    } else {
        c[0] = q[0]; sv[0] = q[offS]; nv[0] = q[offN]; dn[0] = q[pk.offD]; up[0] = q[pk.offU]; r[0] = a.r[rb + i];
    }
    const float w = i > 0 ? q[-1] : (px ? q[nx - 1] : mul_(ghost_lo(a.bcx), c[0]));
    const float e = i + VW < nx ? q[VW] : (px ? q[VW - nx] : mul_(ghost_hi(a.bcx), c[VW - 1]));
#pragma unroll
    for (int v = 0; v < VW; ++v) {
        const float xl = v > 0 ? c[v - 1] : w, xr = v < VW - 1 ? c[v + 1] : e;
        const float tx = (xr - c[v]) + (xl - c[v]);
        const float ty = (mul_(mN, nv[v]) - c[v]) + (mul_(mS, sv[v]) - c[v]);
        const float tu = mul_(pk.mU, up[v]) - c[v], td = mul_(pk.mD, dn[v]) - c[v];
        const float ld = fma_(pk.za, td, fma_(pk.zc, tu, fma_(a.cy, ty, mul_(a.cx, tx))));
        out[v] = (r[v] - fma_(a.c0, c[v], ld)) - dshift;
    }
}

template <typename T> struct RowArgs {
    DirTab<T> t;
    const void* in;
    void* out;
    long nrows;          // nz * ny rows of length nx
    int rpc;             // rows per CTA
    double in_scale;     // forward: multiply the input (1 normally)
    const double* shift_acc;   // inverse accumulation: subtract shift_acc[0] * shift_scale
    double shift_scale;
    int bulk;            // rows move with TMA bulk copies (alignment checked on the host)
    int* status;
    // OUT_FF_ACC_D only: the FP32 correction is also stored to dout (same
    // rows as the input), and with gacc non-null the dzf-weighted sum of the
    // updated pairs is added to gacc[0] (plane k = row / ny, weight gw[k])
    void* dout;
    double* gacc;
    const double* gw;
    int ny;
    unsigned nymag;
    // forward transform with input RUIn: the rows are the residual update
    // (ru.r rows of this CTA, ru.d with its neighbours), computed in shared
    // memory; `in` is unused
    ResidUpdArgs ru;
};

// Output modes of the inverse x kernel.
enum OutMode {
    OUT_T = 0,          // write the compute type
    OUT_F64 = 1,        // write double
    OUT_FF_INIT = 2,    // write a double-float pair (v, 0) into the 8-byte slot
    OUT_FF_ACC = 3,     // pair += v - shift
    OUT_FF_FINAL = 4,   // double = pair + v - shift
    OUT_FF_ACC_D = 5    // pair += v, v also stored as FP32 (the correction), optional gauge sum
};

template <typename T> struct ColArgs {
    DirTab<T> t;         // y tables (n = ny)
    void* data;          // in place, [nplanes][ny][nx]
    int nx;
    long nplanes;
    int tx;              // columns per tile (4 .. 32)
    int bulk;            // rows may be moved with TMA bulk copies (alignment checked on the host)
    int* status;
};

// z tridiagonal solve per mode: (sigma - alpha L) u = scale * g in mode space,
// L = L_z + lambda_x(mx) + lambda_y(my).
template <typename T> struct ZArgs {
    T* data;             // [nz][nmodes] in place (nmodes = nx * ny)
    const T* src;        // warp-per-segment kernel: input read from here (null: data)
    const T* lamx;       // [nx]
    const T* lamy;       // [ny]
    const T* za;         // [nz] coupling to k-1 (1 / (dzc[k] dzf[k]))
    const T* zc;         // [nz] coupling to k+1 (1 / (dzc[k+1] dzf[k]))
    const double* dzf;   // [nz] (FP64; projection, gauge and adjoint scaling)
    int nx, ny, nz;
    int zlo, zhi;        // ZBC_*
    int singular;        // Poisson with only P/N sides: project, pin, gauge mode 0
    int adjoint;         // apply D S D^-1 (D = diag(dzf))
    int tm;              // modes per CTA
    int P;               // threads per mode (segments of the z line)
    int maxm;            // > 0: register-pivot kernel for segments of at most maxm rows
    int warp_mode;       // warp-per-segment kernel (32 modes per CTA, P warps)
    int bulk;            // tile rows may be moved with TMA bulk copies
    T sigma, alpha, scale;
    int* status;         // device status word (bit flags)
    double* cacc;        // singular mode 0: cacc[0] += (weighted mean of the rhs line) * cacc_scale
    double cacc_scale;
    // Warp-per-segment kernel: the pivot entering segment s of mode q (it
    // depends on sigma, alpha and the mode only, not on the right-hand side)
    // at ecache[s * nmodes + q].  ecache_mode 0: computed, not kept; 1:
    // computed and stored; 2: loaded (the composite-map phase is skipped).
    T* ecache;
    int ecache_mode;
    long ecache_stride;  // nmodes; 0 when every line has the same pivots (line solves)
    int persist;         // warp-per-segment kernel: 0 = one tile per CTA; else the persistent
                         // double-buffered variant where it applies
    // singular mode 0: shift_acc[0] * shift_scale subtracted from the whole
    // line after the gauge (a constant of the solution in physical space; the
    // last refinement sweep removes the measured mean of its iterate this way)
    const double* shift_acc;
    double shift_scale;
};

// FP64 residual r = f - (c0 u + c1 L u) of the 7-point staggered Laplacian.
struct ResidArgs {
    const double* u;
    const double* f;
    void* r;             // float or double output
    int r_is_double;
    int nx, ny, nz;
    int bcx, bcy, zlo, zhi;   // KIND_* for x/y, ZBC_* for z
    double idx2, idy2;
    const double* za;
    const double* zc;
    double c0, c1;
    double fshift;       // subtracted from f (consistency constant)
};

// Double-float residual r = (f - cshift) - (c0 u + c1 L u) with u held as
// double-float pairs; optional dzf-weighted sum of u into gacc[0].
struct ResidFFArgs {
    const double* f;
    const float2* u;     // (hi, lo) pairs
    float* r;
    int nx, ny, nz;
    int bcx, bcy, zlo, zhi;
    float cxh, cxl, cyh, cyl, c0h;   // c1/dx^2, c1/dy^2 (split), c0 (0 or 1)
    const double* za;    // [nz] FP64 couplings, scaled by c1 per CTA
    const double* zc;
    double c1;
    const double* cshift;
    double* gacc;
    const double* dzf;
    int lo_zero;         // every lo part of u is zero (first sweep after an FP32 solve)
    int rows_per_cta;    // set by the launcher
};

// Smagorinsky / van Driest eddy viscosity at the cell centres of a channel.
template <typename T> struct SgsArgs {
    const T* u;          // x-faces [nz][ny][nx]
    const T* v;          // y-faces [nz][ny][nx]
    const T* w;          // z-faces [nz+1][ny][nx], w[0] = w[nz] = 0
    T* nut;              // centres [nz][ny][nx]
    int nx, ny, nz;
    T idx, idy;
    const T* idzf;       // 1/dzf [nz]
    const T* idzc;       // 1/dzc [nz+1]
    const double* zcen;  // cell-centre heights [nz] (bottom wall at 0)
    const double* dzf;   // [nz]
    double* coef;        // [nz] scratch: (C_s Delta D)^2 per plane
    double lz, dx, dy, cs, nu, utau;
};

// Explicit RK3 predictor of the pressure-correction substep (Eq. 7) on a channel.
template <typename T> struct MomArgs {
    const T* u;          // x-faces [nz][ny][nx]
    const T* v;          // y-faces [nz][ny][nx]
    const T* w;          // z-faces [nz+1][ny][nx], w[0] = w[nz] = 0
    const T* nut;        // eddy viscosity, centres [nz][ny][nx]
    const T* p;          // pressure p^{k-1/2}, centres
    T* us;               // predicted velocity u* (same layouts as u, v, w)
    T* vs;
    T* ws;
    T* ru;               // in: R^{k-1} (read only when beta != 0); out: R^k = H^k + nu L u^k
    T* rv;
    T* rw;
    int nx, ny, nz;
    T idx, idy;
    const T* idzf;       // 1/dzf [nz]
    const T* idzc;       // 1/dzc [nz+1]
    T nu, dt, alpha, beta, gamma;
    int implicit;        // 0: explicit viscous terms (Eq. 11); 1: Crank-Nicolson in all directions
                         // (Eqs. 17-18); 2: Crank-Nicolson in z only (Eqs. 20-21)
};

enum StatusBits { ST_NONFINITE = 1, ST_BADPIVOT = 2, ST_TIMEOUT = 4 };

template <typename T, typename TIn> cudaError_t launch_rows_forward(const RowArgs<T>& a, cudaStream_t st);
// RUIn input: needs nx % 4 == 0 and 16-byte aligned ru.r, ru.d
bool rows_forward_ru_ok(const RowArgs<float>& a);
template <typename T, int MODE> cudaError_t launch_rows_inverse(const RowArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t launch_cols(const ColArgs<T>& a, bool inverse, cudaStream_t st);
// Compile-time-size FP32 variants of the transforms (periodic rows with
// L = 128, 256, 768; column tiles (L, TX) = (64, 32), (128, 32), (256, 16)
// of every kind): launch and return true when the sizes have one.
// CALES_STATIC_FFT=0 in the environment turns them off.
// in_kind: 0 FP32 rows, 1 FP64 rows, 2 the fused residual update (RUIn)
bool launch_rows_forward_static(const RowArgs<float>& a, int in_kind, cudaStream_t st, cudaError_t* err);
bool launch_rows_inverse_static(const RowArgs<float>& a, int mode, cudaStream_t st, cudaError_t* err);
bool launch_cols_static(const ColArgs<float>& a, bool inverse, cudaStream_t st, cudaError_t* err);
bool static_fft_enabled();
template <typename T> cudaError_t launch_zsolve(const ZArgs<T>& a, cudaStream_t st);
template <typename T> size_t zsolve_smem(int nz, int tm, int P);
template <typename T> size_t zsolve_reg_smem(int nz, int tm, int P);
template <typename T> size_t zsolve_w_smem(int nz, int P);
cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st);
template <typename T> cudaError_t launch_eddy_viscosity(const SgsArgs<T>& a, cudaStream_t st);
cudaError_t launch_residual_ff(const ResidFFArgs& a, cudaStream_t st);
int residual_rows_per_cta(int nx, int ny);
cudaError_t launch_residual_update(const ResidUpdArgs& a, cudaStream_t st);

// Grouped launches: the same stage of many solves in one launch; CTA b runs
// block work[b].y of item work[b].x (argument blocks in device memory).
template <typename T> size_t rows_smem_bytes(const RowArgs<T>& a);
template <typename T> size_t cols_smem_bytes(const ColArgs<T>& a);
template <typename T> size_t zsolve_w_smem_pb(int nz, int P, int Pb);
template <typename T, typename TIn>
cudaError_t launch_rows_forward_grp(const RowArgs<T>* items, const int2* work, int nblocks, size_t smem, cudaStream_t);
template <typename T, int MODE>
cudaError_t launch_rows_inverse_grp(const RowArgs<T>* items, const int2* work, int nblocks, size_t smem, cudaStream_t);
template <typename T>
cudaError_t launch_cols_grp(const ColArgs<T>* items, const int2* work, int nblocks, int tx, bool inverse, size_t smem,
                            cudaStream_t);
template <typename T>
cudaError_t launch_zsolve_grp(const ZArgs<T>* items, const int2* work, int nblocks, int maxm, bool adjoint,
                              int threads, size_t smem, cudaStream_t);
// variant bits: 1 singular (consistency shift), 2 Helmholtz, 4 gauge sum, 8 lo parts present
cudaError_t launch_residual_ff_grp(const ResidFFArgs* items, const int2* work, int nblocks, int variant,
                                   cudaStream_t st);

// ---- projection operators and learned-closure kernels ----
template <typename T> struct GridArgs {
    int nx, ny, nz;
    T idx, idy;
    const T* idzf;
    const T* idzc;
};
struct StencilArgs {
    int nx, ny, nz;
    const float* theta;
    const float* in[3];
    float* out[3];
    float a, beta;
};
struct WGradArgs {
    int nx, ny, nz;
    const float* g[3];
    const float* in[3];
    double* gtheta;
};
struct SqErrArgs {
    long n[3];
    const float* pred[3];
    const float* target[3];
    float* grad[3];
    double* loss;
    float scale;
};
template <typename T> cudaError_t launch_divergence(const GridArgs<T>&, const T*, const T*, const T*, T*, cudaStream_t);
template <typename T>
cudaError_t launch_gradient(const GridArgs<T>&, const T*, const T*, const T*, const T*, T*, T*, T*, int, cudaStream_t);
template <typename T>
cudaError_t launch_divergence_T(const GridArgs<T>&, const T*, const T*, const T*, const T*, T*, T*, T*, cudaStream_t);
template <typename T> cudaError_t launch_gradient_T(const GridArgs<T>&, const T*, const T*, const T*, T*, cudaStream_t);
// periodic z: cyclic tridiagonal per mode (row 0 eliminated last), two scratch fields [nz][nmodes]
template <typename T> cudaError_t launch_zsolve_cyclic(const ZArgs<T>&, T* ework, T* zwork, cudaStream_t);
template <typename T> cudaError_t launch_mom_predict(const MomArgs<T>&, cudaStream_t);
template <typename T> cudaError_t launch_pressure_update(T* p, const T* phi, T scale, long n, cudaStream_t);
// u, v, w -= grad phi' in place; p += (phi' - a L phi') * scale with L the full
// (implicit 1) or z-only (implicit 2) Laplacian, Neumann z walls (Eqs. 13, 19, 22)
template <typename T>
cudaError_t launch_correct_cn(const GridArgs<T>& g, T* u, T* v, T* w, T* p, const T* phi, T a, T scale, int implicit,
                              cudaStream_t);
cudaError_t launch_stencil27(const StencilArgs&, cudaStream_t);
cudaError_t launch_stencil27_wgrad(const WGradArgs&, cudaStream_t);
cudaError_t launch_sqerr(const SqErrArgs&, cudaStream_t);
cudaError_t launch_adam(float*, const double*, float*, float*, int, float, float, float, float, int, float, cudaStream_t);

}  // namespace cales

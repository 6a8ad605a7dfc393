// Kernel argument blocks and launcher declarations (internal to the library).
#pragma once
#include "common.cuh"

namespace cales {

template <typename T> struct RowArgs {
    DirTab<T> t;
    const void* in;
    void* out;
    long nrows;          // nz * ny rows of length nx
    int rpc;             // rows per CTA
    double in_scale;     // forward: multiply the input (1 normally)
    const double* shift_acc;   // inverse accumulation: subtract shift_acc[0] * shift_scale
    double shift_scale;
};

// Output modes of the inverse x kernel.
enum OutMode {
    OUT_T = 0,          // write the compute type
    OUT_F64 = 1,        // write double
    OUT_FF_INIT = 2,    // write a double-float pair (v, 0) into the 8-byte slot
    OUT_FF_ACC = 3,     // pair += v - shift
    OUT_FF_FINAL = 4    // double = pair + v - shift
};

template <typename T> struct ColArgs {
    DirTab<T> t;         // y tables (n = ny)
    void* data;          // in place, [nplanes][ny][nx]
    int nx;
    long nplanes;
    int tx;              // columns per tile (8, 16 or 32)
};

// z tridiagonal solve per mode: (sigma - alpha L) u = scale * g in mode space,
// L = L_z + lambda_x(mx) + lambda_y(my).
template <typename T> struct ZArgs {
    T* data;             // [nz][nmodes] in place (nmodes = nx * ny)
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
    T sigma, alpha, scale;
    int* status;         // device status word (bit flags)
    double* cacc;        // singular mode 0: cacc[0] += (weighted mean of the rhs line) * cacc_scale
    double cacc_scale;
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
};

enum StatusBits { ST_NONFINITE = 1, ST_BADPIVOT = 2 };

template <typename T, typename TIn> cudaError_t launch_rows_forward(const RowArgs<T>& a, cudaStream_t st);
template <typename T, int MODE> cudaError_t launch_rows_inverse(const RowArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t launch_cols(const ColArgs<T>& a, bool inverse, cudaStream_t st);
template <typename T> cudaError_t launch_zsolve(const ZArgs<T>& a, cudaStream_t st);
cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st);
cudaError_t launch_residual_ff(const ResidFFArgs& a, cudaStream_t st);

}  // namespace cales

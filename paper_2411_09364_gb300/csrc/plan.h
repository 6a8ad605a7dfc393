// Host-side plan object behind the opaque cales_plan_t handle.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.cuh"

struct DirHost {
    int n = 1, kind = 0, L = 1, nrad = 0;
    int radix[cales::MAX_RADICES] = {0};
    int twoff[cales::MAX_RADICES] = {0};
    int twlen = 0;
    double2* tw_d = nullptr;
    double2* post_d = nullptr;
    double2* mak_d = nullptr;
    double* lam_d = nullptr;
    float2* tw_f = nullptr;
    float2* post_f = nullptr;
    float2* mak_f = nullptr;
    float* lam_f = nullptr;
    template <typename T> cales::DirTab<T> tab() const;
};

struct ProfRec {
    const char* name = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
};

struct cales_plan_s;

namespace cales {
// Per-solve options of one pass of the solver.
struct PassOpt {
    double sigma, alpha, scale;
    bool singular, adjoint;
    double* cacc;              // consistency-constant accumulator (singular mode 0)
    const double* shift_acc;   // gauge accumulator subtracted by the inverse-x kernel
    double shift_scale;
};
// Argument blocks of the stages of one pass (plan.cu), shared by the
// single-solve pipeline and the grouped batch executor.
template <typename T, typename TIn> RowArgs<T> fwd_row_args(cales_plan_s* P, const void* in, T* work);
template <typename T> ColArgs<T> col_args(cales_plan_s* P, T* work);
template <typename T> ZArgs<T> z_args(cales_plan_s* P, T* work, const PassOpt& o);
template <typename T> void z_args_done(cales_plan_s* P, const ZArgs<T>& za, const PassOpt& o);
template <typename T, int MODE> RowArgs<T> inv_row_args(cales_plan_s* P, T* work, void* out, const PassOpt& o);
// Options of a Poisson (helm false) or Helmholtz solve on plan P.
PassOpt solve_opts(const cales_plan_s* P, bool helm, double alpha, bool adjoint);
// Double-float residual arguments of refinement sweep s of ns.
ResidFFArgs resid_args(const cales_plan_s* P, bool helm, double alpha, const void* f, void* p, float* work,
                       double* cacc, double* gacc, int s, int ns);
}  // namespace cales

// Rebuild the x / y FFT tables with another radix order (plan.cu).
int plan_set_radix_order(cales_plan_s* P, int order);

// Internal entry shared by the C ABI, the batch executor and the autotuner.
int cales_internal_solve(cales_plan_s* P, bool helm, double alpha, bool adjoint, const void* f, void* p,
                         void* stream);

struct cales_plan_s {
    int nx = 0, ny = 0, nz = 0;
    int bc[6] = {0};
    double dx = 0, dy = 0;
    int singular_poisson = 0;
    DirHost X, Y;
    double* za_d = nullptr;
    double* zc_d = nullptr;
    double* dzf_d = nullptr;
    float* za_f = nullptr;
    double* zcen_d = nullptr;    // cell-centre heights [nz], bottom face at 0
    double* sgs_coef = nullptr;  // [nz] eddy-viscosity plane coefficients (C_s Delta D)^2
    void* zcyc = nullptr;        // periodic z: two [nz][nx*ny] scratch fields (FP64 size)
    double* zero_d = nullptr;    // max(nx, ny) zeros: the eigenvalues of the line solves
    float* zero_f = nullptr;
    float* zc_f = nullptr;
    int* status = nullptr;
    double* acc = nullptr;       // [0] consistency constant, [1] gauge sum (refinement)
    double* idzf_d = nullptr;    // 1/dzf [nz]
    double* idzc_d = nullptr;    // 1/dzc [nz+1]
    float* idzf_f = nullptr;
    float* idzc_f = nullptr;
    double dzf_sum = 0.0;
    int precision = 0, sweeps = 2;
    // launch schedule (0 = built-in heuristic): x shared-memory budget in KB,
    // y tile width, z warps per CTA, z rows per segment bound, radix order of
    // the x and y FFTs (0 radix 16 first, 1 radices 5 and 3 first, 2 radix 8
    // instead of 16), z kernel variant (0 one tile per CTA, 1 persistent)
    static constexpr int NSCHED = 6;
    int sched[NSCHED] = {0, 0, 0, 0, 0, 0};
    int radix_order = 0;         // order the X and Y tables were built with
    float* work = nullptr;
    float* work2 = nullptr;      // fast refinement: the residual field kept between sweeps
    // Segment-entry pivots of the z sweeps (FP32 and FP64 copies, 16 segment
    // slots per mode) and the (sigma, alpha, P, maxm) they were computed for.
    struct ZCacheKey { int valid = 0, P = 0, maxm = 0; double sigma = 0.0, alpha = 0.0; };
    void* zcache[2] = {nullptr, nullptr};
    ZCacheKey zkey[2];
    // the same for the line solves (all eigenvalues zero: 16 values per precision)
    void* lcache[2] = {nullptr, nullptr};
    ZCacheKey lkey[2];
    std::vector<void*> owned;
    static constexpr int PROF_MAX = 4096;
    bool prof_on = false;
    int prof_n = 0;
    ProfRec prof[PROF_MAX];
    void prof_begin(cudaStream_t st, const char* name);
    void prof_end(cudaStream_t st);
    void fill_resid(cales::ResidArgs& ra, const double* u, const double* f, void* r, bool r_double, double c0,
                    double c1) const;
};

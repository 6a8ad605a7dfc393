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
    // y tile width, z warps per CTA, z rows per segment bound
    int sched[4] = {0, 0, 0, 0};
    float* work = nullptr;
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

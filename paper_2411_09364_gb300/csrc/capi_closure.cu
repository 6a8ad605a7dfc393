// C ABI of the projection operators and learned-closure kernels (cales.h).
#include "cales.h"
#include "kernels.cuh"
#include "plan.h"

#include <cmath>



using namespace cales;

static bool channel_layout(cales_plan_t P) {
    return P && P->bc[0] == CALES_BC_P && P->bc[2] == CALES_BC_P && P->bc[4] == CALES_BC_N && P->bc[5] == CALES_BC_N;
}

template <typename T> static GridArgs<T> gargs(cales_plan_t P) {
    GridArgs<T> g;
    g.nx = P->nx; g.ny = P->ny; g.nz = P->nz;
    g.idx = T(1.0 / P->dx);
    g.idy = T(1.0 / P->dy);
    g.idzf = sizeof(T) == 8 ? (const T*)P->idzf_d : (const T*)P->idzf_f;
    g.idzc = sizeof(T) == 8 ? (const T*)P->idzc_d : (const T*)P->idzc_f;
    return g;
}

template <typename T>
static SgsArgs<T> sgs_args(cales_plan_t P, double cs, double nu, double utau, const void* u, const void* v,
                           const void* w, void* nut) {
    SgsArgs<T> a;
    a.u = (const T*)u; a.v = (const T*)v; a.w = (const T*)w; a.nut = (T*)nut;
    a.nx = P->nx; a.ny = P->ny; a.nz = P->nz;
    a.idx = T(1.0 / P->dx);
    a.idy = T(1.0 / P->dy);
    a.idzf = sizeof(T) == 8 ? (const T*)P->idzf_d : (const T*)P->idzf_f;
    a.idzc = sizeof(T) == 8 ? (const T*)P->idzc_d : (const T*)P->idzc_f;
    a.zcen = P->zcen_d;
    a.dzf = P->dzf_d;
    a.coef = P->sgs_coef;
    a.lz = P->dzf_sum; a.dx = P->dx; a.dy = P->dy;
    a.cs = cs; a.nu = nu; a.utau = utau;
    return a;
}

// Wray's low-storage RK3 coefficients (Sec. 2.2, below Eq. 14): alpha_k,
// beta_k, gamma_k = alpha_k + beta_k; the three gammas sum to one.
static const double kRk3Alpha[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double kRk3Beta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

// One explicit substep (Eqs. 11-14, then Eq. 4): predictor, divergence of u*,
// Poisson solve for phi' = gamma dt phi, correction u = u* - grad phi',
// p += phi' / (gamma dt), nu_t from the new velocity.  d = div u* is staged
// in the nut array, whose old values the predictor has consumed.
template <typename T>
static int rk3_substep(cales_plan_t P, int stage, double dt, double nu, double cs, double utau, T* u, T* v, T* w,
                       T* p, T* nut, T* ru, T* rv, T* rw, T* work, cudaStream_t st) {
    const size_t n = (size_t)P->nx * P->ny * P->nz, nw = (size_t)P->nx * P->ny * (P->nz + 1);
    T* us = work;
    T* vs = us + n;
    T* ws = vs + n;
    T* phi = ws + nw;
    const double al = kRk3Alpha[stage], be = kRk3Beta[stage], ga = al + be;
    const GridArgs<T> g = gargs<T>(P);
    MomArgs<T> m;
    m.u = u; m.v = v; m.w = w; m.nut = nut; m.p = p;
    m.us = us; m.vs = vs; m.ws = ws;
    m.ru = ru; m.rv = rv; m.rw = rw;
    m.nx = P->nx; m.ny = P->ny; m.nz = P->nz;
    m.idx = g.idx; m.idy = g.idy; m.idzf = g.idzf; m.idzc = g.idzc;
    m.nu = T(nu); m.dt = T(dt); m.alpha = T(al); m.beta = T(be); m.gamma = T(ga);
    m.implicit = 0;
    if (launch_mom_predict<T>(m, st) != cudaSuccess) return CALES_ECUDA;
    if (launch_divergence<T>(g, us, vs, ws, nut, st) != cudaSuccess) return CALES_ECUDA;
    const int rc = cales_internal_solve(P, false, 0.0, false, nut, phi, st);
    if (rc != CALES_OK) return rc;
    if (launch_gradient<T>(g, phi, us, vs, ws, u, v, w, 1, st) != cudaSuccess) return CALES_ECUDA;
    if (launch_pressure_update<T>(p, phi, T(1.0 / (ga * dt)), (long)n, st) != cudaSuccess) return CALES_ECUDA;
    if (launch_eddy_viscosity<T>(sgs_args<T>(P, cs, nu, utau, u, v, w, nut), st) != cudaSuccess) return CALES_ECUDA;
    return CALES_OK;
}

// Crank-Nicolson substep (Eqs. 17-19 for implicit = 1, Eqs. 20-22 for
// implicit = 2): the predictor writes the right-hand sides of the velocity
// solves into the work buffers, the solves write u* over u^k (consumed by
// then), and one kernel applies the correction and the pressure update.
template <typename T>
static int rk3_substep_cn(cales_plan_t P, cales_plan_t Puv, cales_plan_t Pw, int implicit, int stage, double dt,
                          double nu, double cs, double utau, T* u, T* v, T* w, T* p, T* nut, T* ru, T* rv, T* rw,
                          T* work, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)P->nx * P->ny, n = plane * P->nz, nw = plane * (P->nz + 1);
    T* us = work;
    T* vs = us + n;
    T* ws = vs + n;
    T* phi = ws + nw;
    const double al = kRk3Alpha[stage], be = kRk3Beta[stage], ga = al + be, ah = 0.5 * ga * nu * dt;
    const GridArgs<T> g = gargs<T>(P);
    MomArgs<T> m;
    m.u = u; m.v = v; m.w = w; m.nut = nut; m.p = p;
    m.us = us; m.vs = vs; m.ws = ws;
    m.ru = ru; m.rv = rv; m.rw = rw;
    m.nx = P->nx; m.ny = P->ny; m.nz = P->nz;
    m.idx = g.idx; m.idy = g.idy; m.idzf = g.idzf; m.idzc = g.idzc;
    m.nu = T(nu); m.dt = T(dt); m.alpha = T(al); m.beta = T(be); m.gamma = T(ga);
    m.implicit = implicit;
    if (launch_mom_predict<T>(m, st) != cudaSuccess) return CALES_ECUDA;
    int rc;
    if (implicit == 1) {
        if ((rc = cales_internal_solve(Puv, true, ah, false, us, u, stream)) != CALES_OK) return rc;
        if ((rc = cales_internal_solve(Puv, true, ah, false, vs, v, stream)) != CALES_OK) return rc;
        if ((rc = cales_internal_solve(Pw, true, ah, false, ws + plane, w + plane, stream)) != CALES_OK) return rc;
    } else {
        if ((rc = cales_helmholtz_z_solve(Puv, ah, us, u, stream)) != CALES_OK) return rc;
        if ((rc = cales_helmholtz_z_solve(Puv, ah, vs, v, stream)) != CALES_OK) return rc;
        if ((rc = cales_helmholtz_z_solve(Pw, ah, ws + plane, w + plane, stream)) != CALES_OK) return rc;
    }
    if (launch_divergence<T>(g, u, v, w, nut, st) != cudaSuccess) return CALES_ECUDA;
    if ((rc = cales_internal_solve(P, false, 0.0, false, nut, phi, stream)) != CALES_OK) return rc;
    if (launch_correct_cn<T>(g, u, v, w, p, phi, T(ah), T(1.0 / (ga * dt)), implicit, st) != cudaSuccess)
        return CALES_ECUDA;
    if (launch_eddy_viscosity<T>(sgs_args<T>(P, cs, nu, utau, u, v, w, nut), st) != cudaSuccess) return CALES_ECUDA;
    return CALES_OK;
}

// the velocity plans of a Crank-Nicolson substep match the pressure plan:
// same nx, ny, dx, dy and precision; u, v plan Dirichlet in z on nz cells, w
// plan wall nodes in z on the nz - 1 interior faces; x and y periodic
static bool cn_plans_match(cales_plan_t P, cales_plan_t Puv, cales_plan_t Pw) {
    if (!Puv || !Pw) return false;
    for (cales_plan_t Q : {Puv, Pw}) {
        if (Q->nx != P->nx || Q->ny != P->ny || Q->dx != P->dx || Q->dy != P->dy || Q->precision != P->precision ||
            Q->bc[0] != CALES_BC_P || Q->bc[2] != CALES_BC_P)
            return false;
    }
    return Puv->nz == P->nz && Puv->bc[4] == CALES_BC_D && Puv->bc[5] == CALES_BC_D && Pw->nz == P->nz - 1 &&
           Pw->bc[4] == CALES_BC_DF && Pw->bc[5] == CALES_BC_DF;
}

#define CALES_DISPATCH(P, CALL_D, CALL_F) \
    ((P)->precision == CALES_FP32 ? (CALL_F) : (CALL_D))

extern "C" {

int cales_eddy_viscosity(cales_plan_t P, double cs, double nu, double utau, const void* u, const void* v,
                         const void* w, void* nut, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!u || !v || !w || !nut || !(cs >= 0.0) || !(nu > 0.0) || !(utau >= 0.0) || !std::isfinite(cs) ||
        !std::isfinite(nu) || !std::isfinite(utau))
        return CALES_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (P->precision == CALES_FP32) e = launch_eddy_viscosity<float>(sgs_args<float>(P, cs, nu, utau, u, v, w, nut), st);
    else e = launch_eddy_viscosity<double>(sgs_args<double>(P, cs, nu, utau, u, v, w, nut), st);
    return e == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_rk3_substep(cales_plan_t P, int stage, double dt, double nu, double cs, double utau, void* u, void* v,
                      void* w, void* p, void* nut, void* ru, void* rv, void* rw, void* work, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (stage < 0 || stage > 2 || !(dt > 0.0) || !std::isfinite(dt) || !(nu > 0.0) || !std::isfinite(nu) ||
        !(cs >= 0.0) || !std::isfinite(cs) || !(utau >= 0.0) || !std::isfinite(utau))
        return CALES_EINVAL;
    if (!u || !v || !w || !p || !nut || !ru || !rv || !rw || !work) return CALES_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->precision == CALES_FP32)
        return rk3_substep<float>(P, stage, dt, nu, cs, utau, (float*)u, (float*)v, (float*)w, (float*)p,
                                  (float*)nut, (float*)ru, (float*)rv, (float*)rw, (float*)work, st);
    return rk3_substep<double>(P, stage, dt, nu, cs, utau, (double*)u, (double*)v, (double*)w, (double*)p,
                               (double*)nut, (double*)ru, (double*)rv, (double*)rw, (double*)work, st);
}

int cales_rk3_substep_cn(cales_plan_t P, cales_plan_t Puv, cales_plan_t Pw, int implicit, int stage, double dt,
                         double nu, double cs, double utau, void* u, void* v, void* w, void* p, void* nut, void* ru,
                         void* rv, void* rw, void* work, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (implicit < 1 || implicit > 2 || stage < 0 || stage > 2 || !(dt > 0.0) || !std::isfinite(dt) ||
        !(nu > 0.0) || !std::isfinite(nu) || !(cs >= 0.0) || !std::isfinite(cs) || !(utau >= 0.0) ||
        !std::isfinite(utau) || P->nz < 2)
        return CALES_EINVAL;
    if (!u || !v || !w || !p || !nut || !ru || !rv || !rw || !work) return CALES_EINVAL;
    if (!cn_plans_match(P, Puv, Pw)) return CALES_EINVAL;
    if (P->precision == CALES_FP32)
        return rk3_substep_cn<float>(P, Puv, Pw, implicit, stage, dt, nu, cs, utau, (float*)u, (float*)v, (float*)w,
                                     (float*)p, (float*)nut, (float*)ru, (float*)rv, (float*)rw, (float*)work, stream);
    return rk3_substep_cn<double>(P, Puv, Pw, implicit, stage, dt, nu, cs, utau, (double*)u, (double*)v, (double*)w,
                                  (double*)p, (double*)nut, (double*)ru, (double*)rv, (double*)rw, (double*)work,
                                  stream);
}

int cales_divergence(cales_plan_t P, const void* u, const void* v, const void* w, void* d, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!u || !v || !w || !d) return CALES_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = CALES_DISPATCH(P,
        launch_divergence<double>(gargs<double>(P), (const double*)u, (const double*)v, (const double*)w, (double*)d, st),
        launch_divergence<float>(gargs<float>(P), (const float*)u, (const float*)v, (const float*)w, (float*)d, st));
    return e == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_gradient(cales_plan_t P, const void* phi, const void* uin, const void* vin, const void* win, void* gx,
                   void* gy, void* gz, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!phi || !gx || !gy || !gz) return CALES_EINVAL;
    const int sub = (uin && vin && win) ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = CALES_DISPATCH(P,
        launch_gradient<double>(gargs<double>(P), (const double*)phi, (const double*)uin, (const double*)vin,
                                (const double*)win, (double*)gx, (double*)gy, (double*)gz, sub, st),
        launch_gradient<float>(gargs<float>(P), (const float*)phi, (const float*)uin, (const float*)vin,
                               (const float*)win, (float*)gx, (float*)gy, (float*)gz, sub, st));
    return e == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_divergence_adjoint(cales_plan_t P, const void* d, const void* uin, const void* vin, const void* win,
                             void* u, void* v, void* w, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!d || !u || !v || !w) return CALES_EINVAL;
    if (!(uin && vin && win)) uin = vin = win = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = CALES_DISPATCH(P,
        launch_divergence_T<double>(gargs<double>(P), (const double*)d, (const double*)uin, (const double*)vin,
                                    (const double*)win, (double*)u, (double*)v, (double*)w, st),
        launch_divergence_T<float>(gargs<float>(P), (const float*)d, (const float*)uin, (const float*)vin,
                                   (const float*)win, (float*)u, (float*)v, (float*)w, st));
    return e == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_gradient_adjoint(cales_plan_t P, const void* gx, const void* gy, const void* gz, void* phi, void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!gx || !gy || !gz || !phi) return CALES_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = CALES_DISPATCH(P,
        launch_gradient_T<double>(gargs<double>(P), (const double*)gx, (const double*)gy, (const double*)gz, (double*)phi, st),
        launch_gradient_T<float>(gargs<float>(P), (const float*)gx, (const float*)gy, (const float*)gz, (float*)phi, st));
    return e == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_stencil27(cales_plan_t P, const float* theta, float a, float beta, const float* const* in, float* const* out,
                    void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!theta || !in || !out) return CALES_EINVAL;
    StencilArgs s;
    s.nx = P->nx; s.ny = P->ny; s.nz = P->nz;
    s.theta = theta;
    for (int c = 0; c < 3; ++c) {
        if (!in[c] || !out[c] || in[c] == out[c]) return CALES_EINVAL;
        s.in[c] = in[c];
        s.out[c] = out[c];
    }
    s.a = a;
    s.beta = beta;
    return launch_stencil27(s, (cudaStream_t)stream) == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_stencil27_weight_grad(cales_plan_t P, const float* const* g, const float* const* in, double* gtheta,
                                void* stream) {
    if (!channel_layout(P)) return P ? CALES_EUNSUPPORTED : CALES_EINVAL;
    if (!g || !in || !gtheta) return CALES_EINVAL;
    WGradArgs s;
    s.nx = P->nx; s.ny = P->ny; s.nz = P->nz;
    for (int c = 0; c < 3; ++c) {
        if (!g[c] || !in[c]) return CALES_EINVAL;
        s.g[c] = g[c];
        s.in[c] = in[c];
    }
    s.gtheta = gtheta;
    return launch_stencil27_wgrad(s, (cudaStream_t)stream) == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_sq_error(const float* const* pred, const float* const* target, float* const* grad, const long* n,
                   float scale, double* loss, void* stream) {
    if (!pred || !target || !n || !loss) return CALES_EINVAL;
    SqErrArgs s;
    for (int c = 0; c < 3; ++c) {
        if (!pred[c] || !target[c] || n[c] < 0) return CALES_EINVAL;
        s.n[c] = n[c];
        s.pred[c] = pred[c];
        s.target[c] = target[c];
        s.grad[c] = grad ? grad[c] : nullptr;
    }
    s.loss = loss;
    s.scale = scale;
    return launch_sqerr(s, (cudaStream_t)stream) == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_adam_step(float* theta, const double* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                    float eps, int t, float grad_scale, void* stream) {
    if (!theta || !grad || !m || !v || n < 1 || t < 1) return CALES_EINVAL;
    return launch_adam(theta, grad, m, v, n, lr, beta1, beta2, eps, t, grad_scale, (cudaStream_t)stream) == cudaSuccess
               ? CALES_OK
               : CALES_ECUDA;
}

int cales_zero(void* p, unsigned long bytes, void* stream) {
    if (!p) return CALES_EINVAL;
    return cudaMemsetAsync(p, 0, bytes, (cudaStream_t)stream) == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

}  // extern "C"

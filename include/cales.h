/*
 * cales.h -- C ABI of the GB300 fast direct solver for the pressure Poisson
 * and Crank-Nicolson velocity Helmholtz equations on a staggered grid.
 *
 * Method (paper Sec. 2.2): the Poisson equation for the pressure correction,
 * Eq. (12), and the three Helmholtz equations of the implicit viscous step,
 * Eq. (18), are discretised with second-order finite differences on a
 * staggered grid and solved by an eigenfunction expansion: real FFT /
 * DCT-II / DST-II in the uniform directions x and y, one tridiagonal system
 * per wavenumber pair along the stretched direction z (Thomas algorithm),
 * then the inverse transforms.  The paper computes its FFTs with cuFFT and
 * its transposes with cuDecomp (Sec. 3.1); here every step is a hand-written
 * sm_103a kernel behind this interface.
 *
 * Conventions (all calls):
 *  - Fields are contiguous device arrays laid out [nz][ny][nx], x fastest.
 *  - Element type: double for CALES_FP64 and CALES_FP32_REFINE plans, float
 *    for CALES_FP32 plans.  The caller owns every field buffer; the plan owns
 *    its tables and workspace (allocated by cales_plan / cales_set_precision).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Solves are asynchronous, launch kernels only, perform no host
 *    synchronisation and no allocation, and may be captured in a CUDA graph.
 *  - Return value: CALES_OK (0) or a negative cales_status code.  Conditions
 *    detected on the device (non-finite values, non-positive pivots) are
 *    OR-ed into a device status word read by cales_get_status.
 *  - A plan may be used from one stream at a time (its workspace is shared
 *    by its solves).
 */
#ifndef CALES_H
#define CALES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cales_plan_s* cales_plan_t;
typedef struct cales_batch_s* cales_batch_t;

/* Boundary kinds, per side: xlo, xhi, ylo, yhi, zlo, zhi. */
enum cales_bc {
    CALES_BC_P = 0,  /* periodic (both sides of the direction)                       */
    CALES_BC_N = 1,  /* homogeneous Neumann at the boundary face, cell-centred unknown */
    CALES_BC_D = 2,  /* homogeneous Dirichlet at the boundary face, cell-centred
                        unknown: ghost = -interior at the mirror distance            */
    CALES_BC_DF = 3  /* homogeneous Dirichlet at a boundary node, node-centred unknown:
                        the boundary value is exactly zero (in x or y on both
                        sides of the direction, DST-I)                           */
};

enum cales_precision {
    CALES_FP64 = 0,        /* FP64 transforms and tridiagonal sweeps              */
    CALES_FP32 = 1,        /* FP32 throughout (float fields)                     */
    CALES_FP32_REFINE = 2, /* FP32 solves + FP64 residual and FP64 accumulation   */
    CALES_FP32_REFINE_FAST = 3 /* as CALES_FP32_REFINE, but only the first sweep
                                forms the residual in double-float; later sweeps
                                update it in FP32 from the previous correction
                                (r <- r - M d): one residual pass per solve fewer
                                per extra sweep, about ten times the final
                                error (double fields, 2 FP32 work fields)     */
};

enum cales_status {
    CALES_OK = 0,
    CALES_EINVAL = -1,       /* bad size, spacing, boundary pairing or argument  */
    CALES_EUNSUPPORTED = -2, /* x/y: a length the transforms do not take (see
                                cales_plan) or a side pairing other than P-P,
                                N-N, D-D, DF-DF, N-D, D-N; periodic z with
                                nz < 3 or in the allocation-free solve      */
    CALES_ENOMEM = -3,       /* device allocation failed                        */
    CALES_ECUDA = -4,        /* a CUDA runtime call failed                      */
    CALES_ETOOBIG = -5       /* grid larger than the static scratch of
                                cales_poisson_solve_noalloc                     */
};

enum cales_device_status_bits {
    CALES_DEV_NONFINITE = 1, /* a non-finite value was produced               */
    CALES_DEV_BADPIVOT = 2,  /* a non-positive pivot met outside the pinned mode */
    CALES_DEV_TIMEOUT = 4    /* a bounded wait for an asynchronous copy gave up;
                                the kernel skipped its tile and returned      */
};

/*
 * Create a plan for an nx x ny x nz grid (paper Sec. 2.2: uniform x, y;
 * stretched z).  bc[6] = {xlo, xhi, ylo, yhi, zlo, zhi}.  Each of x and y
 * takes, with its transform: P on both sides (real DFT), N-N (DCT-II), D-D
 * (DST-II), N-D (DCT-IV), D-N (DST-IV) for cell-centred unknowns, with an
 * even length (or 1) whose half factors into 2, 3 and 5; or DF-DF (DST-I)
 * for node-centred unknowns between two wall nodes (n = interior nodes,
 * spacing = node distance), with n + 1 factoring into 2, 3 and 5.  Periodic
 * on one side only is CALES_EINVAL, other pairings CALES_EUNSUPPORTED.
 * z takes N, D or DF independently per side, or P on both sides (nz >= 3).
 * Periodic z: each mode's z system is cyclic (row 0 couples to row nz-1
 * through dzc[0], row nz-1 to row 0 through dzc[nz]; both must hold the same
 * distance, the one between the last and the first cell centre through the
 * period, else CALES_EINVAL).  Row 0 is eliminated last: rows 1..nz-1 are a
 * tridiagonal T solved by Thomas with excess-form pivots for two right-hand
 * sides (the data, and the couplings to u[0]), u = p + u[0] (1 - q), and
 * u[0] follows from row 0 through a denominator that is a sum of positive
 * terms.  One thread per mode, 16 bytes per grid point of plan-owned
 * scratch.  It serves the Poisson and Helmholtz solves in every precision
 * mode, their adjoints, the wall-normal line solves and the residual;
 * all-periodic/Neumann Poisson problems are made consistent, their zero mode
 * pinned and the result gauged as below.
 * dx, dy: uniform spacings.  dzc[0..nz]: distance between unknowns k-1 and k
 * (dzc[0], dzc[nz]: to the ghost/boundary node; mirror value dzf[0] resp.
 * dzf[nz-1] for cell-centred unknowns).  dzf[0..nz-1]: control-volume width
 * of unknown k.  Both arrays are host memory and are copied.
 * For node-centred unknowns (e.g. w in z with walls) pass the node grid:
 * nz = number of interior nodes, dzc = distances between nodes, dzf = the
 * widths between neighbouring cell centres.
 * Default precision: CALES_FP64 with 2 refinement sweeps preset.
 */
int cales_plan(cales_plan_t* out, int nx, int ny, int nz, const int bc[6],
               double dx, double dy, const double* dzc, const double* dzf);

/* Select precision and refinement sweeps (0..8; used by CALES_FP32_REFINE and
 * CALES_FP32_REFINE_FAST, which with fewer than 2 sweeps runs as
 * CALES_FP32_REFINE).  Allocates the FP32 workspace (4 bytes per grid point,
 * 8 for the fast mode) when needed. */
int cales_set_precision(cales_plan_t plan, int mode, int refine_sweeps);

/*
 * Poisson solve, Eq. (12): L p = f with the staggered 7-point Laplacian
 * (Eq. 16).  With only periodic/Neumann sides L is singular: f is first made
 * consistent (its dzf-weighted mean removed) and p is returned with zero
 * dzf-weighted mean.  f and p are device arrays of nx*ny*nz elements; f == p
 * is allowed (in place) for CALES_FP64 and CALES_FP32 plans.
 */
int cales_poisson_solve(cales_plan_t plan, const void* f, void* p, void* stream);

/*
 * Helmholtz solve, Eq. (18): (I - alpha L) u = f, alpha > 0
 * (alpha = gamma_k nu dt / 2 of the Crank-Nicolson substep).
 */
int cales_helmholtz_solve(cales_plan_t plan, double alpha, const void* f, void* u, void* stream);

/*
 * Adjoint (transpose) solves: g = S^T w where S is the linear map f -> p of
 * cales_poisson_solve (resp. f -> u of cales_helmholtz_solve).  Computed as
 * the same transforms around the transposed tridiagonal systems
 * (S^T = D S D^-1 with D = diag(dzf) along z).  CALES_FP64 and CALES_FP32
 * plans; CALES_FP32_REFINE plans return CALES_EUNSUPPORTED.
 */
int cales_poisson_solve_adjoint(cales_plan_t plan, const void* w, void* g, void* stream);
int cales_helmholtz_solve_adjoint(cales_plan_t plan, double alpha, const void* w, void* g, void* stream);

/*
 * Wall-normal implicit step, Eq. 21 (viscous term implicit along the
 * stretched direction only): (I - alpha L_z) u = f on every (i, j) line
 * independently, one tridiagonal system per line with the plan's z grid and
 * z boundary kinds (x and y kinds play no part).  alpha >= 0.  f and u are
 * device arrays of nx*ny*nz elements, double for CALES_FP64 and
 * CALES_FP32_REFINE plans (solved in FP64: one sweep per line, no
 * refinement needed), float for CALES_FP32 plans; f == u is allowed.
 */
int cales_helmholtz_z_solve(cales_plan_t plan, double alpha, const void* f, void* u, void* stream);

/*
 * Poisson solve like cales_poisson_solve with FP32 solves and double-float
 * refinement (the plan's refine_sweeps), for callers that cannot allocate
 * device memory when they solve: hosts that hand the library a fixed
 * device-memory budget and fail any further allocation (another framework's
 * memory pool owns the rest of the GPU), and time-stepping loops that must
 * not block in cudaMalloc, which may synchronise the device.  No counterpart
 * in the paper (an interface addition).  It allocates nothing: its scratch (4 bytes per grid point plus
 * 256 bytes) is one file-scope device array of the library, sized for at most
 * 8,388,608 grid points (8 * 2^20); larger grids return CALES_ETOOBIG.  The
 * plan needs no cales_set_precision call; f, p: double device arrays, f != p.
 * The first call on each device looks the array's address up with that device
 * current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call on a device shares the one array, which keeps the last
 * call's contents (the call clears what must start at zero itself): calls
 * that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.
 */
int cales_poisson_solve_noalloc(cales_plan_t plan, const void* f, void* p, void* stream);

/*
 * FP64 residual r = f - L u (alpha < 0 selects Poisson) or r = f - (I - alpha L) u.
 * u, f, r: double device arrays.  No projection is applied to f.
 */
int cales_residual(cales_plan_t plan, double alpha, const double* u, const double* f, double* r, void* stream);

/*
 * Staggered projection operators of the fractional-step method (Sec. 2.2,
 * Eqs. 12-13) for plans periodic in x and y with Neumann (wall) z sides.
 * Layout: u on x-faces and v on y-faces, [nz][ny][nx]; w on z-faces,
 * [nz+1][ny][nx] with w[0] = w[nz] = 0 at the walls; scalars [nz][ny][nx].
 * Element type as for the solves (float for CALES_FP32 plans, else double).
 *   divergence: d = (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy + (w_{k+1} - w_k)/dzf_k
 *   gradient  : (gx, gy, gz) = grad phi, gz = 0 on the walls; with uin, vin,
 *               win non-NULL the outputs are (uin, vin, win) - grad phi, i.e.
 *               the velocity correction of Eq. (13) with gamma dt folded in phi.
 *   *_adjoint : the exact transposes (for gradients through the projection);
 *               divergence_adjoint with uin, vin, win non-NULL returns
 *               (uin, vin, win) - div^T d.
 * Other boundary kinds return CALES_EUNSUPPORTED.
 */
int cales_divergence(cales_plan_t plan, const void* u, const void* v, const void* w, void* d, void* stream);
int cales_gradient(cales_plan_t plan, const void* phi, const void* uin, const void* vin, const void* win,
                   void* gx, void* gy, void* gz, void* stream);
int cales_divergence_adjoint(cales_plan_t plan, const void* d, const void* uin, const void* vin, const void* win,
                             void* u, void* v, void* w, void* stream);
int cales_gradient_adjoint(cales_plan_t plan, const void* gx, const void* gy, const void* gz, void* phi, void* stream);

/*
 * Smagorinsky eddy viscosity with van Driest damping, Eq. 4 (Sec. 2.1; model
 * evaluated at the cell centres, Sec. 2.2): nu_t = (cs Delta D)^2 |S| with
 * |S| = sqrt(2 S_ij S_ij), D = 1 - exp(-y+/25).  Same plans and layouts as
 * the projection operators above (periodic x and y, walls in z); u, v, w
 * are the staggered velocity, nut is written at the cell centres [nz][ny][nx].
 * The diagonal strain rates are formed at the centres, the off-diagonal ones
 * on the four surrounding cell edges and averaged to the centre; u and v
 * take no-slip ghosts (minus the first interior value, at the mirror
 * distances dzc[0], dzc[nz]) and w is zero on the wall faces.  Filter width
 * Delta = (dx dy dzf_k)^(1/3); y+ = (distance of the centre to the nearer
 * wall) * utau / nu.  cs >= 0, nu > 0, utau >= 0.  FP32 plans compute in
 * FP32 (float arrays), the others in FP64 (double arrays).  The per-plane
 * coefficients (cs Delta D)^2 go through a plan-owned scratch array, so one
 * plan serves one eddy-viscosity call at a time (like its solves).  Arrays
 * 16-byte aligned with nx a multiple of 4 (FP32) / 2 (FP64) take vector
 * loads; any other alignment is served by a scalar kernel.  Returns
 * CALES_EINVAL for NULL arrays or parameters out of range, CALES_ECUDA when
 * the launch fails (nz > 65535 included).
 */
int cales_eddy_viscosity(cales_plan_t plan, double cs, double nu, double utau, const void* u, const void* v,
                         const void* w, void* nut, void* stream);

/*
 * One substep (stage 0, 1, 2) of the low-storage RK3 pressure-correction
 * scheme with explicit viscous terms, Sec. 2.2 Eqs. 11-14 and Algorithm 1:
 *   R^k       = H^k + nu L u^k,  H_i = -d(u_i u_j)/dx_j + d(2 nu_t S_ij)/dx_j (Eq. 15;
 *               signs from Eqs. 2-3)
 *   u*        = u^k + dt (alpha_k R^k + beta_k R^{k-1} - gamma_k grad p^{k-1/2})   (Eq. 11)
 *   L phi     = div u* / (gamma_k dt)                                          (Eq. 12)
 *   u^{k+1}   = u* - gamma_k dt grad phi                                       (Eq. 13)
 *   p^{k+1/2} = p^{k-1/2} + phi                                                (Eq. 14)
 *   nu_t^{k+1} from u^{k+1} as cales_eddy_viscosity (Eq. 4)
 * with Wray's alpha = (8/15, 5/12, 3/4), beta = (0, -17/60, -5/12),
 * gamma = alpha + beta.  Channel plans only (periodic x and y, Neumann z for
 * the pressure; the velocity has no-slip walls, ghosts as in
 * cales_eddy_viscosity; nu_t beyond a wall repeats the first interior value).
 * Advection is in divergence form with mean interpolation; the off-diagonal
 * stresses sit on cell edges with nu_t averaged from the four centres.
 *   u, v [nz][ny][nx], w [nz+1][ny][nx] (w[0] = w[nz] = 0): in u^k, out u^{k+1}
 *   p [nz][ny][nx]: in p^{k-1/2}, out p^{k+1/2}
 *   nut [nz][ny][nx]: in nu_t^k, out nu_t^{k+1} (also used as scratch)
 *   ru, rv [nz][ny][nx], rw [nz+1][ny][nx]: in R^{k-1} (not read at stage 0),
 *     out R^k, for the next stage
 *   work: 3 nx ny nz + nx ny (nz+1) elements (u*, v*, w*, phi), not aliased
 * Element type: float for CALES_FP32 plans, double otherwise (the Poisson
 * solve runs in the plan's precision mode).  All arrays are device memory
 * owned by the caller.  Returns CALES_EUNSUPPORTED for other boundary
 * layouts, CALES_EINVAL for a stage outside 0..2, dt or nu not positive,
 * cs or utau negative or any NULL array, CALES_ECUDA on launch failure.
 */
int cales_rk3_substep(cales_plan_t plan, int stage, double dt, double nu, double cs, double utau, void* u,
                      void* v, void* w, void* p, void* nut, void* ru, void* rv, void* rw, void* work,
                      void* stream);

/*
 * The same substep with Crank-Nicolson viscous terms, Sec. 2.2:
 *   implicit = 1 (Eqs. 17-19):
 *     u**  = u^k + dt (alpha_k H^k + beta_k H^{k-1} + gamma_k (nu L u^k - grad p^{k-1/2}))
 *     (I - a L) u* = u** - a L u^k,   a = gamma_k nu dt / 2   (modified Helmholtz, Eq. 18)
 *     Poisson and correction as above (Eqs. 12-13)
 *     p^{k+1/2} = p^{k-1/2} + phi - a L phi
 *     R^k = H^k
 *   implicit = 2 (Eqs. 20-22): L replaced by its wall-normal part L_z in the
 *     implicit terms (line solves, as cales_helmholtz_z_solve); nu (L_x + L_y) u
 *     joins H in the explicit RK3 terms, R^k = H^k + nu (L_x + L_y) u^k.
 * plan: the pressure plan (as cales_rk3_substep).  uv_plan: the u and v
 * solves, bc (P, P, P, P, D, D) on the same nx, ny, nz, dx, dy and z spacings.
 * w_plan: the w solve on the nz - 1 interior z-faces, bc (P, P, P, P, DF, DF),
 * node spacings dzc_w = dzf, control volumes dzf_w = dzc[1..nz-1] of the
 * pressure grid.  All three plans of the same precision mode; the z spacings
 * are the caller's to keep consistent (nx, ny, nz, dx, dy, kinds and precision
 * are checked: CALES_EINVAL otherwise).  Arrays, work size, ownership and the
 * other errors as cales_rk3_substep; implicit outside 1..2 is CALES_EINVAL.
 * The velocity solves use the plans' own workspaces, so the three plans serve
 * one call at a time.
 */
int cales_rk3_substep_cn(cales_plan_t plan, cales_plan_t uv_plan, cales_plan_t w_plan, int implicit, int stage,
                         double dt, double nu, double cs, double utau, void* u, void* v, void* w, void* p,
                         void* nut, void* ru, void* rv, void* rw, void* work, void* stream);

/*
 * Learned closure trained through the projection (the paper motivates
 * machine-learned closures built on the solver, Sec. 1).  FP32, plan layout
 * as above.  theta: device [3][27] taps, tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).
 *   cales_stencil27: out_c = a*in_c + sum_t theta[c][t] in_c(x + o_t) + beta*tanh(in_c)
 *     (x, y periodic; zero outside the component's planes in z; w walls held 0);
 *     in[3], out[3]: device pointers of u, v, w (out != in).
 *   cales_stencil27_weight_grad: gtheta[c][t] += sum_x g_c(x) in_c(x + o_t)
 *     (FP64 device accumulators, zeroed by the caller; g at w walls ignored).
 *   cales_sq_error: loss[0] += sum (pred - target)^2 over the three arrays of
 *     n[c] elements; grad[c] (optional) = scale * (pred - target).
 *   cales_adam_step: one Adam update of n parameters (Kingma & Ba) from the
 *     FP64 gradient times grad_scale; m, v: device moment buffers; t >= 1.
 */
int cales_stencil27(cales_plan_t plan, const float* theta, float a, float beta, const float* const* in,
                    float* const* out, void* stream);
int cales_stencil27_weight_grad(cales_plan_t plan, const float* const* g, const float* const* in, double* gtheta,
                                void* stream);
int cales_sq_error(const float* const* pred, const float* const* target, float* const* grad, const long* n,
                   float scale, double* loss, void* stream);
int cales_adam_step(float* theta, const double* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                    float eps, int t, float grad_scale, void* stream);

/*
 * Launch schedule of a plan, CALES_SCHED_LEN entries: {x shared-memory budget
 * per CTA in KB, y tile width in columns, z warps per CTA, z rows-per-segment
 * bound, FFT radix order of x and y (0: radix-16 passes first, the order of
 * the compile-time-size kernels; 1: radices 5 and 3 first; 2: radix-8 passes
 * in place of radix 16), z kernel variant (0: one 32-mode tile per CTA; 1:
 * persistent CTAs with two tile buffers)}; 0 selects the built-in heuristic
 * and infeasible sizes fall back to it.  A new radix order rebuilds the
 * plan's transform tables (synchronises the device).  CALES_EINVAL for
 * negative entries, an order > 2 or a variant > 1.
 */
#define CALES_SCHED_LEN 6
int cales_set_schedule(cales_plan_t plan, const int sched[CALES_SCHED_LEN]);
int cales_get_schedule(cales_plan_t plan, int sched[CALES_SCHED_LEN]);

/*
 * Autotuner (the analogue of the paper's runtime-tuned decomposition and
 * communication backends, Sec. 3.1): times candidate schedules of the plan's
 * Poisson solve at its current precision on the device (each knob tuned in
 * turn: FFT radix order 0/1/2 on the x + y stages, x budget 32/64/96 KB, y
 * tiles 8/16/32/64/128, z segments of 16/32/64 rows, then the persistent z
 * kernel, kept only when more than 3 % faster),
 * keeps the fastest and sets it on the plan.  With cache_path non-NULL the
 * result is looked up first and stored after tuning in a JSON object keyed by
 * "nx,ny,nz,bcx,bcy,zlo,zhi,precision,device".  Allocates two temporary fields
 * and synchronises `stream`: call it at set-up, not inside a capture.
 */
int cales_autotune(cales_plan_t plan, const char* cache_path, void* stream);

/*
 * Batched solves (a Runge-Kutta substep of Algorithm 1: per domain the three
 * Helmholtz solves of Eq. 18 and the Poisson solve of Eq. 12, over many
 * independent domains).  kinds[i]: 0 = Poisson, 1 = Helmholtz with alphas[i].
 * Grouped execution (default): when every plan is CALES_FP32_REFINE with the
 * same sweep count, a non-periodic z and no plan serves two solves, each
 * stage of the solver (x, y, z transforms and sweeps, residual) runs once for
 * all solves of the batch -- one launch per stage and kernel variant, whose
 * CTAs walk a (solve, block) work list; 17 launches and 4 memsets for two
 * sweeps, whatever the batch size.  The argument blocks are built and copied
 * to the device (synchronously) on the first solve or capture with a set of
 * buffers, and again when the buffers change.  Otherwise the solves are
 * forked over up to 8 streams balanced by grid size (solves that share a plan
 * stay on one stream) and joined back on the caller's stream.
 * cales_batch_solve enqueues directly; cales_batch_capture records the same
 * work for fixed f[i], u[i] into one CUDA graph, replayed by
 * cales_batch_launch with a single launch.  Plans, precisions and the
 * pointers captured must stay valid while the graph is used.
 * cales_batch_set_grouped(batch, 0) forces the fork/join path;
 * cales_batch_grouped reports whether the last solve or capture was grouped.
 */
int cales_batch_create(cales_batch_t* out, int n, const cales_plan_t* plans, const int* kinds, const double* alphas);
int cales_batch_solve(cales_batch_t batch, const void* const* f, void* const* u, void* stream);
int cales_batch_capture(cales_batch_t batch, const void* const* f, void* const* u, void* stream);
int cales_batch_launch(cales_batch_t batch, void* stream);
int cales_batch_graph_nodes(cales_batch_t batch, unsigned long* nodes);
int cales_batch_set_grouped(cales_batch_t batch, int on);
int cales_batch_grouped(cales_batch_t batch, int* used);
void cales_batch_destroy(cales_batch_t batch);

/* Asynchronous zero fill of `bytes` bytes of device memory (accumulators). */
int cales_zero(void* p, unsigned long bytes, void* stream);

/* Per-kernel CUDA-event timings: enable (resets the record list), then read
 * name/ms pairs of every launch since (synchronises).  Returns the count. */
int cales_profile_enable(cales_plan_t plan, int on);
int cales_profile_read(cales_plan_t plan, int max, const char** names, float* ms);

/* Read and clear the device status word (synchronises the plan's last stream). */
int cales_get_status(cales_plan_t plan, int* device_status);

/* Human-readable text of a cales_status code. */
const char* cales_strerror(int code);

/* Release the plan and its device memory (after its work has completed). */
void cales_destroy(cales_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* CALES_H */

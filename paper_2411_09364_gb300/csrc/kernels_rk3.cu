// Predictor of the low-storage RK3 pressure-correction substep (Sec. 2.2) on
// a channel (x, y periodic, no-slip walls in z), H_i of Eq. 15:
//   H_i = -d(u_i u_j)/dx_j + d(2 nu_t S_ij)/dx_j,
//   explicit (Eq. 11):   R^k = H^k + nu L u^k,
//                        u*  = u^k + dt (alpha R^k + beta R^{k-1} - gamma grad p^{k-1/2});
//   Crank-Nicolson, all directions (Eqs. 17-18): R^k = H^k and the kernel writes
//                        u** - a L u^k,  a = gamma nu dt / 2, the right-hand side of the
//                        Helmholtz solve;
//   Crank-Nicolson in z (Eqs. 20-21): R^k = H^k + nu (L_x + L_y) u^k and the
//                        right-hand side u** - a L_z u^k of the line solves.
// The last two are followed by the in-place correction and pressure update of
// k_correct_cn (Eqs. 13, 19, 22).
// The signs of H follow the momentum equation (Eq. 2) with the Boussinesq
// closure (Eq. 3).  Advection is in divergence form with every interpolated
// velocity the mean of its two neighbours; the off-diagonal strain rates sit
// on cell edges with nu_t there the mean of the four surrounding centres.
// Beyond a wall u and v take minus the first interior value (at the mirror
// distances dzc[0], dzc[nz]) and nu_t repeats it; w = 0 on the wall faces.
//
// A CTA owns a 32 x 8 column tile and marches down MOM_KC planes of it.  A
// ring of three planes (k-1, k, k+1) of u, v, w, nu_t and p, each 34 x 10
// with a one-cell periodic halo, lives in shared memory; every plane is read
// from global memory once per tile (the wall ghosts of u, v, nu_t are formed
// as it is filled) and the stencils read the ring; plane k+2 is gathered
// into registers while plane k is computed.  One thread per cell
// (i, j, k) forms all three components: x-momentum at the face (i+1/2, j, k),
// y-momentum at (i, j+1/2, k), z-momentum at the face (i, j, k) (k >= 1; the
// wall rows of w* and R_w are written as 0).  R^{k-1} is read from and R^k
// written to the same arrays, point by point.
#include "kernels.cuh"

namespace cales {

constexpr int MOM_TX = 32, MOM_TY = 8, MOM_KC = 16;
constexpr int MOM_LX = MOM_TX + 2, MOM_LY = MOM_TY + 2;

template <typename T> struct MomRing {
    T u[3][MOM_LY][MOM_LX];
    T v[3][MOM_LY][MOM_LX];
    T w[3][MOM_LY][MOM_LX];      // z-faces k-1, k, k+1
    T n[3][MOM_LY][MOM_LX];
    T p[3][MOM_LY][MOM_LX];
};

template <typename T>
__device__ __forceinline__ T sq(T x) { return x * x; }

__device__ __forceinline__ int ring_slot(int m) { return (m + 3) % 3; }   // m >= -1

// Plane m (-1 <= m <= nz) of the tile at (x0, y0), gathered into registers
// (two ring entries per thread) and then put into its ring slot: cell arrays
// beyond a wall take the ghosts (u, v: minus the first interior value; nu_t:
// the value itself; p: unused there, 0); w holds face m.
constexpr int MOM_PER = (MOM_LX * MOM_LY + MOM_TX * MOM_TY - 1) / (MOM_TX * MOM_TY);
template <typename T> struct MomFill {
    T u[MOM_PER], v[MOM_PER], w[MOM_PER], n[MOM_PER], p[MOM_PER];
};

template <typename T>
__device__ __forceinline__ void mom_gather(MomFill<T>& f, const MomArgs<T>& a, int m, int x0, int y0, int tid) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t plane = (size_t)nx * ny;
    const int mc = m < 0 ? 0 : (m >= nz ? nz - 1 : m);
    const T sg = (m < 0 || m >= nz) ? T(-1) : T(1);
    const bool pin = m >= 0 && m < nz, win = m >= 0 && m <= nz;
#pragma unroll
    for (int t = 0; t < MOM_PER; ++t) {
        const int e = tid + t * MOM_TX * MOM_TY;
        if (e < MOM_LX * MOM_LY) {
            const int ly = e / MOM_LX, lx = e - ly * MOM_LX;
            int gi = (x0 + lx - 1) % nx, gj = (y0 + ly - 1) % ny;
            gi = gi < 0 ? gi + nx : gi;
            gj = gj < 0 ? gj + ny : gj;
            const size_t q = (size_t)gj * nx + gi, qc = (size_t)mc * plane + q;
            f.u[t] = sg * a.u[qc];
            f.v[t] = sg * a.v[qc];
            f.n[t] = a.nut[qc];
            f.p[t] = pin ? a.p[qc] : T(0);
            f.w[t] = win ? a.w[(size_t)m * plane + q] : T(0);
        }
    }
}

template <typename T>
__device__ __forceinline__ void mom_put(MomRing<T>& r, const MomFill<T>& f, int m, int tid) {
    const int sl = ring_slot(m);
#pragma unroll
    for (int t = 0; t < MOM_PER; ++t) {
        const int e = tid + t * MOM_TX * MOM_TY;
        if (e < MOM_LX * MOM_LY) {
            const int ly = e / MOM_LX, lx = e - ly * MOM_LX;
            r.u[sl][ly][lx] = f.u[t];
            r.v[sl][ly][lx] = f.v[t];
            r.w[sl][ly][lx] = f.w[t];
            r.n[sl][ly][lx] = f.n[t];
            r.p[sl][ly][lx] = f.p[t];
        }
    }
}

template <typename T>
__device__ __forceinline__ void mom_fill(MomRing<T>& r, const MomArgs<T>& a, int m, int x0, int y0, int tid) {
    MomFill<T> f;
    mom_gather(f, a, m, x0, y0, tid);
    mom_put(r, f, m, tid);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_mom_predict(MomArgs<T> a) {
    __shared__ MomRing<T> ring;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * MOM_TX + tx;
    const int x0 = blockIdx.x * MOM_TX, y0 = blockIdx.y * MOM_TY;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int k0 = blockIdx.z * MOM_KC, k1 = k0 + MOM_KC < nz ? k0 + MOM_KC : nz;
    const int i = x0 + tx, j = y0 + ty;
    const bool active = i < nx && j < ny;
    const size_t plane = (size_t)nx * ny;
    const T idx = a.idx, idy = a.idy, idx2 = idx * idx, idy2 = idy * idy;
    const T h = T(0.5), q = T(0.25), two = T(2);
    const T nu = a.nu, dt = a.dt, al = a.alpha, be = a.beta, ga = a.gamma;
    const T hcn = ga * nu * dt * h;                        // gamma nu dt / 2 of the Crank-Nicolson modes
    const int cx = tx + 1, cy = ty + 1;
    // R (carried to the next stage) and the velocity update from the advection +
    // SGS part hs, the Laplacian parts lxy, lz and the pressure gradient gp:
    //   MODE 0: R = hs + nu (lxy + lz),  out = c + dt (alpha R + beta R' - gamma gp)
    //   MODE 1: R = hs,                  out = c + dt (alpha R + beta R' + gamma (nu L - gp)) - hcn L
    //   MODE 2: R = hs + nu lxy,         out = c + dt (alpha R + beta R' + gamma (nu lz - gp)) - hcn lz
    auto update = [&](T c, T hs, T lxy, T lz, T gp, T rp, T& r) -> T {
        T inc;
        if constexpr (MODE == 0) {
            r = hs + nu * (lxy + lz);
            inc = al * r - ga * gp;
        } else if constexpr (MODE == 1) {
            r = hs;
            inc = al * r - ga * gp + ga * nu * (lxy + lz);
        } else {
            r = hs + nu * lxy;
            inc = al * r - ga * gp + ga * nu * lz;
        }
        if (be != T(0)) inc += be * rp;
        T out = c + dt * inc;
        if constexpr (MODE == 1) out -= hcn * (lxy + lz);
        if constexpr (MODE == 2) out -= hcn * lz;
        return out;
    };

    mom_fill(ring, a, k0 - 1, x0, y0, tid);
    mom_fill(ring, a, k0, x0, y0, tid);
    mom_fill(ring, a, k0 + 1, x0, y0, tid);
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        // plane k+2 and R^{k-1} are loaded before the stencils run, so their
        // latency hides behind the arithmetic of plane k
        const bool more = k + 1 < k1;                       // uniform over the CTA
        MomFill<T> next;
        if (more) mom_gather(next, a, k + 2, x0, y0, tid);
        const size_t c = (size_t)k * plane + (size_t)j * nx + i;
        T rpu = T(0), rpv = T(0), rpw = T(0);
        if (active && be != T(0)) {
            rpu = a.ru[c];
            rpv = a.rv[c];
            if (k > 0) rpw = a.rw[c];
        }
        if (active) {
            const int sd = ring_slot(k - 1), s0 = ring_slot(k), su = ring_slot(k + 1);
            // ring reads relative to the cell: plane (d: k-1, 0: k, u: k+1), y offset, x offset
            auto U = [&](int sl, int dj, int di) -> T { return ring.u[sl][cy + dj][cx + di]; };
            auto V = [&](int sl, int dj, int di) -> T { return ring.v[sl][cy + dj][cx + di]; };
            auto W = [&](int sl, int dj, int di) -> T { return ring.w[sl][cy + dj][cx + di]; };
            auto N = [&](int sl, int dj, int di) -> T { return ring.n[sl][cy + dj][cx + di]; };
            auto P = [&](int sl, int dj, int di) -> T { return ring.p[sl][cy + dj][cx + di]; };
            const T izf = a.idzf[k], izlo = a.idzc[k], izhi = a.idzc[k + 1];
            const T n_c = N(s0, 0, 0), n_e = N(s0, 0, 1), n_w = N(s0, 0, -1);
            const T n_n = N(s0, 1, 0), n_s = N(s0, -1, 0), n_ne = N(s0, 1, 1), n_se = N(s0, -1, 1);
            const T n_nw = N(s0, 1, -1);
            const T n_u = N(su, 0, 0), n_ue = N(su, 0, 1), n_un = N(su, 1, 0);
            const T n_d = N(sd, 0, 0), n_de = N(sd, 0, 1), n_dn = N(sd, 1, 0);
            const T p_c = P(s0, 0, 0);

            // ---- x-momentum at (i+1/2, j, k) ----
            {
                const T uc = U(s0, 0, 0), ue = U(s0, 0, 1), uw = U(s0, 0, -1), un = U(s0, 1, 0), us = U(s0, -1, 0);
                const T uu = U(su, 0, 0), ud = U(sd, 0, 0);
                const T v0 = V(s0, 0, 0), v0e = V(s0, 0, 1), vs0 = V(s0, -1, 0), vse = V(s0, -1, 1);
                const T wa = W(su, 0, 0), wae = W(su, 0, 1), wb = W(s0, 0, 0), wbe = W(s0, 0, 1);
                const T adv = (sq(h * (uc + ue)) - sq(h * (uw + uc))) * idx +
                              (h * (uc + un) * (h * (v0 + v0e)) - h * (us + uc) * (h * (vs0 + vse))) * idy +
                              (h * (uc + uu) * (h * (wa + wae)) - h * (ud + uc) * (h * (wb + wbe))) * izf;
                const T lxy = (ue - two * uc + uw) * idx2 + (un - two * uc + us) * idy2;
                const T lz = ((uu - uc) * izhi - (uc - ud) * izlo) * izf;
                const T t11e = two * n_e * (ue - uc) * idx, t11w = two * n_c * (uc - uw) * idx;
                const T t12n = two * (q * (n_c + n_e + n_n + n_ne)) * (h * ((un - uc) * idy + (v0e - v0) * idx));
                const T t12s = two * (q * (n_s + n_se + n_c + n_e)) * (h * ((uc - us) * idy + (vse - vs0) * idx));
                const T t13u = two * (q * (n_c + n_e + n_u + n_ue)) * (h * ((uu - uc) * izhi + (wae - wa) * idx));
                const T t13d = two * (q * (n_d + n_de + n_c + n_e)) * (h * ((uc - ud) * izlo + (wbe - wb) * idx));
                const T sgs = (t11e - t11w) * idx + (t12n - t12s) * idy + (t13u - t13d) * izf;
                const T gp = (P(s0, 0, 1) - p_c) * idx;
                T r;
                a.us[c] = update(uc, -adv + sgs, lxy, lz, gp, rpu, r);
                a.ru[c] = r;
            }
            // ---- y-momentum at (i, j+1/2, k) ----
            {
                const T vc = V(s0, 0, 0), vn = V(s0, 1, 0), vs = V(s0, -1, 0), ve = V(s0, 0, 1), vw = V(s0, 0, -1);
                const T vu = V(su, 0, 0), vd = V(sd, 0, 0);
                const T uc = U(s0, 0, 0), un = U(s0, 1, 0), uw = U(s0, 0, -1), unw = U(s0, 1, -1);
                const T wa = W(su, 0, 0), wan = W(su, 1, 0), wb = W(s0, 0, 0), wbn = W(s0, 1, 0);
                const T adv = (h * (uc + un) * (h * (vc + ve)) - h * (uw + unw) * (h * (vw + vc))) * idx +
                              (sq(h * (vc + vn)) - sq(h * (vs + vc))) * idy +
                              (h * (vc + vu) * (h * (wa + wan)) - h * (vd + vc) * (h * (wb + wbn))) * izf;
                const T lxy = (ve - two * vc + vw) * idx2 + (vn - two * vc + vs) * idy2;
                const T lz = ((vu - vc) * izhi - (vc - vd) * izlo) * izf;
                const T t22n = two * n_n * (vn - vc) * idy, t22c = two * n_c * (vc - vs) * idy;
                const T t12e = two * (q * (n_c + n_e + n_n + n_ne)) * (h * ((un - uc) * idy + (ve - vc) * idx));
                const T t12w = two * (q * (n_w + n_c + n_nw + n_n)) * (h * ((unw - uw) * idy + (vc - vw) * idx));
                const T t23u = two * (q * (n_c + n_n + n_u + n_un)) * (h * ((vu - vc) * izhi + (wan - wa) * idy));
                const T t23d = two * (q * (n_d + n_dn + n_c + n_n)) * (h * ((vc - vd) * izlo + (wbn - wb) * idy));
                const T sgs = (t12e - t12w) * idx + (t22n - t22c) * idy + (t23u - t23d) * izf;
                const T gp = (P(s0, 1, 0) - p_c) * idy;
                T r;
                a.vs[c] = update(vc, -adv + sgs, lxy, lz, gp, rpv, r);
                a.rv[c] = r;
            }
            // ---- z-momentum at the face (i, j, k), k >= 1; the wall faces stay 0 ----
            if (k == 0) {
                a.ws[c] = T(0);
                a.rw[c] = T(0);
            } else {
                const T izfd = a.idzf[k - 1];
                const T wc = W(s0, 0, 0), we = W(s0, 0, 1), ww = W(s0, 0, -1), wn = W(s0, 1, 0), ws = W(s0, -1, 0);
                const T wu = W(su, 0, 0), wd = W(sd, 0, 0);
                const T ukc = U(s0, 0, 0), ukw = U(s0, 0, -1), udc = U(sd, 0, 0), udw = U(sd, 0, -1);
                const T vkc = V(s0, 0, 0), vks = V(s0, -1, 0), vdc = V(sd, 0, 0), vds = V(sd, -1, 0);
                const T n_dw = N(sd, 0, -1), n_ds = N(sd, -1, 0);
                const T adv = (h * (udc + ukc) * (h * (wc + we)) - h * (udw + ukw) * (h * (ww + wc))) * idx +
                              (h * (vdc + vkc) * (h * (wc + wn)) - h * (vds + vks) * (h * (ws + wc))) * idy +
                              (sq(h * (wc + wu)) - sq(h * (wd + wc))) * izlo;
                const T lxy = (we - two * wc + ww) * idx2 + (wn - two * wc + ws) * idy2;
                const T lz = ((wu - wc) * izf - (wc - wd) * izfd) * izlo;
                const T t33c = two * n_c * (wu - wc) * izf, t33d = two * n_d * (wc - wd) * izfd;
                const T t13e = two * (q * (n_d + n_c + n_de + n_e)) * (h * ((ukc - udc) * izlo + (we - wc) * idx));
                const T t13w = two * (q * (n_dw + n_w + n_d + n_c)) * (h * ((ukw - udw) * izlo + (wc - ww) * idx));
                const T t23n = two * (q * (n_d + n_c + n_dn + n_n)) * (h * ((vkc - vdc) * izlo + (wn - wc) * idy));
                const T t23s = two * (q * (n_ds + n_s + n_d + n_c)) * (h * ((vks - vds) * izlo + (wc - ws) * idy));
                const T sgs = (t13e - t13w) * idx + (t23n - t23s) * idy + (t33c - t33d) * izlo;
                const T gp = (p_c - P(sd, 0, 0)) * izlo;
                T r;
                a.ws[c] = update(wc, -adv + sgs, lxy, lz, gp, rpw, r);
                a.rw[c] = r;
            }
            if (k == nz - 1) {                              // top wall face
                a.ws[c + plane] = T(0);
                a.rw[c + plane] = T(0);
            }
        }
        __syncthreads();                                    // plane k-1's slot is free now
        if (more) {
            mom_put(ring, next, k + 2, tid);
            __syncthreads();
        }
    }
}

// p^{k+1/2} = p^{k-1/2} + scale * phi'  (Eq. 14 with phi = phi' / (gamma dt))
template <typename T>
__global__ void k_pressure_update(T* __restrict__ p, const T* __restrict__ phi, T scale, long n) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        p[e] += scale * phi[e];
}

// Crank-Nicolson correction (Eqs. 13 and 19 / 22) in place, one thread per
// cell (i, j, k): u, v at the faces i+1/2, j+1/2 and w at the face k (k >= 1)
// lose the gradient of phi'; p gains scale (phi' - a L phi') with L the full
// (MODE 1) or z-only (MODE 2) Laplacian of the pressure (Neumann z walls).
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_correct_cn(GridArgs<T> g, T* __restrict__ u, T* __restrict__ v,
                                                   T* __restrict__ w, T* __restrict__ p,
                                                   const T* __restrict__ phi, T a, T scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z, nx = g.nx, ny = g.ny, nz = g.nz;
    if (i >= nx || j >= ny) return;
    const size_t plane = (size_t)nx * ny, row = (size_t)k * plane + (size_t)j * nx;
    const size_t c = row + i;
    const int ip = i + 1 < nx ? i + 1 : 0, im = i > 0 ? i - 1 : nx - 1;
    const int jp = j + 1 < ny ? j + 1 : 0, jm = j > 0 ? j - 1 : ny - 1;
    const T pc = phi[c];
    const T pe = phi[row + ip];
    const T pn = phi[(size_t)k * plane + (size_t)jp * nx + i];
    const T pd = k > 0 ? phi[c - plane] : pc;               // Neumann: the ghost repeats the wall cell
    const T pu = k < nz - 1 ? phi[c + plane] : pc;
    u[c] -= (pe - pc) * g.idx;
    v[c] -= (pn - pc) * g.idy;
    if (k > 0) w[c] -= (pc - pd) * g.idzc[k];
    T lap = ((pu - pc) * g.idzc[k + 1] - (pc - pd) * g.idzc[k]) * g.idzf[k];
    if constexpr (MODE == 1) {
        const T pw = phi[row + im];
        const T ps = phi[(size_t)k * plane + (size_t)jm * nx + i];
        lap = (pe - T(2) * pc + pw) * (g.idx * g.idx) + (pn - T(2) * pc + ps) * (g.idy * g.idy) + lap;
    }
    p[c] += scale * (pc - a * lap);
}

template <typename T>
cudaError_t launch_correct_cn(const GridArgs<T>& g, T* u, T* v, T* w, T* p, const T* phi, T a, T scale,
                              int implicit, cudaStream_t st) {
    if (g.nz < 1 || g.nz > 65535 || g.ny > 8 * 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
    if (implicit == 1) k_correct_cn<T, 1><<<grid, dim3(32, 8), 0, st>>>(g, u, v, w, p, phi, a, scale);
    else if (implicit == 2) k_correct_cn<T, 2><<<grid, dim3(32, 8), 0, st>>>(g, u, v, w, p, phi, a, scale);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mom_predict(const MomArgs<T>& a, cudaStream_t st) {
    if (a.nz < 1 || a.ny > MOM_TY * 65535) return cudaErrorInvalidValue;
    const dim3 block(MOM_TX, MOM_TY);
    const dim3 grid((unsigned)((a.nx + MOM_TX - 1) / MOM_TX), (unsigned)((a.ny + MOM_TY - 1) / MOM_TY),
                    (unsigned)((a.nz + MOM_KC - 1) / MOM_KC));
    switch (a.implicit) {
        case 0: k_mom_predict<T, 0><<<grid, block, 0, st>>>(a); break;
        case 1: k_mom_predict<T, 1><<<grid, block, 0, st>>>(a); break;
        case 2: k_mom_predict<T, 2><<<grid, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pressure_update(T* p, const T* phi, T scale, long n, cudaStream_t st) {
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_pressure_update<T><<<(unsigned)blocks, 256, 0, st>>>(p, phi, scale, n);
    return cudaGetLastError();
}

template cudaError_t launch_mom_predict<float>(const MomArgs<float>&, cudaStream_t);
template cudaError_t launch_mom_predict<double>(const MomArgs<double>&, cudaStream_t);
template cudaError_t launch_pressure_update<float>(float*, const float*, float, long, cudaStream_t);
template cudaError_t launch_pressure_update<double>(double*, const double*, double, long, cudaStream_t);
template cudaError_t launch_correct_cn<float>(const GridArgs<float>&, float*, float*, float*, float*, const float*, float,
                                             float, int, cudaStream_t);
template cudaError_t launch_correct_cn<double>(const GridArgs<double>&, double*, double*, double*, double*,
                                              const double*, double, double, int, cudaStream_t);

}  // namespace cales

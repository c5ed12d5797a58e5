// FP64 integrator kernels: kick (Eq. 9 with the acceleration of Eq. 8), drift
// (Eq. 10), one RK4 step of the Friedmann equation (Eq. 1) for a(t), Eq. 7
// softening, reductions and the caller-order scatter/gather.
//
// The scalars t, a, H = adot/a and the current dt live in device memory
// (SC_* slots), so a whole kick-drift-kick step (Eq. 11) runs without a host
// round trip and can be captured in a CUDA graph.
#include <cfloat>
#include <cuda_runtime.h>

#include <algorithm>
#include <math_constants.h>
#include <stdint.h>

#include "steps_internal.h"

namespace steps {

namespace {

inline unsigned blocks_for(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// Eq. 1: H(a) = H0 sqrt(Om a^-3 + Or a^-4 + OL + Ok a^-2)
__device__ __forceinline__ double hubble(double a, const Cosmo &c) {
    const double ia = 1.0 / a;
    return c.H0 * sqrt(c.Om * ia * ia * ia + c.Or * ia * ia * ia * ia + c.OL + c.Ok * ia * ia);
}

// Half kick: v += (dt/2) A.  Comoving (Eq. 8):
//   A = acc/a^3 - 2 H v + (4 pi G/3) Om rho_crit x / a^3,   rho_crit = 3 H0^2/(8 pi G),
// so the background coefficient is Om H0^2 / 2 (G cancels).  Static: A = acc.
// a and H are the values at this half-kick's time point; v is taken at entry.
__global__ void kick_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ z, double *__restrict__ vx,
                            double *__restrict__ vy, double *__restrict__ vz,
                            const double *__restrict__ ax, const double *__restrict__ ay,
                            const double *__restrict__ az, const double *__restrict__ sc,
                            Cosmo c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double hdt = 0.5 * sc[SC_DT];
    if (!c.comoving) {
        vx[i] += hdt * ax[i];
        vy[i] += hdt * ay[i];
        vz[i] += hdt * az[i];
        return;
    }
    const double a = sc[SC_A], H = sc[SC_H];
    const double ia3 = 1.0 / (a * a * a);
    const double bg = c.periodic ? 0.0 : (c.reversed ? -0.5 : 0.5) * c.Om * c.H0 * c.H0;
    const double Ax = ax[i] * ia3 - 2.0 * H * vx[i] + bg * x[i] * ia3;
    const double Ay = ay[i] * ia3 - 2.0 * H * vy[i] + bg * y[i] * ia3;
    const double Az = az[i] * ia3 - 2.0 * H * vz[i] + bg * z[i] * ia3;
    vx[i] += hdt * Ax;
    vy[i] += hdt * Ay;
    vz[i] += hdt * Az;
}

// Drift (Eq. 10): x += v dt
__global__ void drift_kernel(int64_t n, double *__restrict__ x, double *__restrict__ y,
                             double *__restrict__ z, const double *__restrict__ vx,
                             const double *__restrict__ vy, const double *__restrict__ vz,
                             const double *__restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = sc[SC_DT];
    x[i] += vx[i] * dt;
    y[i] += vy[i] * dt;
    z[i] += vz[i] * dt;
}

// One classical RK4 step of da/dt = a H(a) with the N-body dt; then H, t.
__global__ void rk4_kernel(double *sc, Cosmo c) {
    const double dt = sc[SC_DT];
    double a = sc[SC_A];
    if (c.comoving) {
        const double k1 = a * hubble(a, c);
        const double a2 = a + 0.5 * dt * k1;
        const double k2 = a2 * hubble(a2, c);
        const double a3 = a + 0.5 * dt * k2;
        const double k3 = a3 * hubble(a3, c);
        const double a4 = a + dt * k3;
        const double k4 = a4 * hubble(a4, c);
        a = a + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
        sc[SC_A] = a;
        sc[SC_H] = hubble(a, c);
    }
    sc[SC_T] += dt;
    sc[SC_STEP] += 1.0;
    sc[SC_RUN] += 1.0;
}

// Eq. 12, first level: per block, min over its particles of q_i = 2 eta_i eps / |A_i|
// (eta_i = 2.8 h_i), A_i the acceleration the kick applies at the current state
// (same expression as kick_kernel).  |A_i| = 0 sets no limit (q = +inf).
__global__ void timestep_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                 const double *__restrict__ z, const double *__restrict__ vx,
                                 const double *__restrict__ vy, const double *__restrict__ vz,
                                 const double *__restrict__ ax, const double *__restrict__ ay,
                                 const double *__restrict__ az, const double *__restrict__ h,
                                 const double *__restrict__ sc, Cosmo c, double eps,
                                 double *__restrict__ part) {
    __shared__ double s[256];
    double q = CUDART_INF;
    const double a = sc[SC_A], H = sc[SC_H];
    const double ia3 = 1.0 / (a * a * a);
    const double bg = c.periodic ? 0.0 : (c.reversed ? -0.5 : 0.5) * c.Om * c.H0 * c.H0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double Ax = ax[i], Ay = ay[i], Az = az[i];
        if (c.comoving) {
            Ax = ax[i] * ia3 - 2.0 * H * vx[i] + bg * x[i] * ia3;
            Ay = ay[i] * ia3 - 2.0 * H * vy[i] + bg * y[i] * ia3;
            Az = az[i] * ia3 - 2.0 * H * vz[i] + bg * z[i] * ia3;
        }
        const double amag = sqrt(Ax * Ax + Ay * Ay + Az * Az);
        if (amag > 0.0) q = fmin(q, 2.0 * (2.8 * h[i]) * eps / amag);
    }
    s[threadIdx.x] = q;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Eq. 12, second level: dt = min(dt_max, sqrt(min q)), limited to t_end - t
// (never below 0) when t_end is finite; becomes the next step's dt.
__global__ void timestep_finish(int nblk, const double *__restrict__ part, double dt_max, double t_end,
                                double *sc) {
    double q = CUDART_INF;
    for (int b = 0; b < nblk; ++b) q = fmin(q, part[b]);
    double dt = dt_max;
    if (q < CUDART_INF && sqrt(q) < dt) dt = sqrt(q);
    if (isfinite(t_end)) {
        const double left = t_end - sc[SC_T];
        if (left < dt) dt = left > 0.0 ? left : 0.0;
    }
    sc[SC_DT] = dt;
}

// dt of the next step of a multi-step run: dts[run index]; the index advances
// in rk4_kernel.
__global__ void set_dt_kernel(double *sc, const double *dts) {
    sc[SC_DT] = dts[(int64_t)sc[SC_RUN]];
}

// Deterministic two-level reductions (fixed block partition, fixed order).
__global__ void kinetic_partial(int64_t n, const double *__restrict__ vx,
                                const double *__restrict__ vy, const double *__restrict__ vz,
                                const double *__restrict__ m, double *__restrict__ part) {
    __shared__ double s[4][256];
    double e = 0, px = 0, py = 0, pz = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = vx[i], b = vy[i], cc = vz[i], w = m[i];
        e += 0.5 * w * (a * a + b * b + cc * cc);
        px += w * a;
        py += w * b;
        pz += w * cc;
    }
    s[0][threadIdx.x] = e;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = pz;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 4; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = s[k][0];
}

__global__ void finish_partial(int nblk, int width, const double *__restrict__ part,
                               double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k >= width) return;
    double acc = 0;
    for (int b = 0; b < nblk; ++b) acc += part[width * b + k];
    out[k] = acc;
}

__global__ void sum_partial(int64_t n, const double *__restrict__ v, double *__restrict__ part) {
    __shared__ double s[256];
    double e = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        e += v[i];
    s[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void scatter3_kernel(int64_t n, const int64_t *__restrict__ perm,
                                const double *__restrict__ a, const double *__restrict__ b,
                                const double *__restrict__ c, double *__restrict__ out3) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[k];
    out3[3 * i] = a[k];
    out3[3 * i + 1] = b[k];
    out3[3 * i + 2] = c[k];
}

__global__ void gather3_kernel(int64_t n, const int64_t *__restrict__ perm,
                               const double *__restrict__ in3, double *__restrict__ a,
                               double *__restrict__ b, double *__restrict__ c) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm ? perm[k] : k;
    a[k] = in3[3 * i];
    b[k] = in3[3 * i + 1];
    c[k] = in3[3 * i + 2];
}

__global__ void iota_kernel(int64_t n, int64_t *perm) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) perm[k] = k;
}

__global__ void min_kernel(int64_t n, const double *__restrict__ m, double *__restrict__ out) {
    __shared__ double s[1024];
    double v = DBL_MAX;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v = fmin(v, m[i]);
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

// Eq. 7: h_i = (m_i / m_min)^(1/3) h_min
__global__ void softening_kernel(int64_t n, const double *__restrict__ m, double h_min,
                                 const double *__restrict__ mmin, double *__restrict__ h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) h[i] = cbrt(m[i] / mmin[0]) * h_min;
}

__global__ void finite_kernel(int64_t n, const double *__restrict__ a, int positive, int *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = a[i];
    if (!isfinite(v)) atomicOr(flag, 1);
    else if (positive && !(v > 0.0)) atomicOr(flag, 2);
}

// *flag = 1 if any of a[i], b[i], c[i] (i < n; h[i] >= 0 when h is given) is NaN or Inf.
__global__ void finite3_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                               const double *__restrict__ c, const double *__restrict__ h, int *flag) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!h || !(h[i] < 0.0)) bad |= !isfinite(a[i]) || !isfinite(b[i]) || !isfinite(c[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

__global__ void set_scalar_kernel(double *sc, int slot, double v) { sc[slot] = v; }

}  // namespace

cudaError_t launch_kick(int64_t n, const double *x, const double *y, const double *z, double *vx,
                        double *vy, double *vz, const double *ax, const double *ay,
                        const double *az, const double *sc, const Cosmo &c, cudaStream_t st) {
    kick_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, x, y, z, vx, vy, vz, ax, ay, az, sc, c);
    return cudaGetLastError();
}

__global__ void drift_wrap_kernel(int64_t n, double *__restrict__ x, double *__restrict__ y,
                                  double *__restrict__ z, const double *__restrict__ vx,
                                  const double *__restrict__ vy, const double *__restrict__ vz,
                                  const double *__restrict__ sc, double box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = sc[SC_DT];
    double *p[3] = {x, y, z};
    const double *v[3] = {vx, vy, vz};
    for (int k = 0; k < 3; ++k) {
        const double q = __dadd_rn(p[k][i], __dmul_rn(v[k][i], dt));
        p[k][i] = __dsub_rn(q, __dmul_rn(box, floor(__ddiv_rn(q, box))));
    }
}

__global__ void wrap_kernel(int64_t n, double *__restrict__ v, double box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = __dsub_rn(v[i], __dmul_rn(box, floor(__ddiv_rn(v[i], box))));
}

cudaError_t launch_drift_wrap(int64_t n, double *x, double *y, double *z, const double *vx,
                              const double *vy, const double *vz, const double *sc, double box,
                              cudaStream_t st) {
    drift_wrap_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, x, y, z, vx, vy, vz, sc, box);
    return cudaGetLastError();
}

cudaError_t launch_wrap(int64_t n, double *v, double box, cudaStream_t st) {
    if (n > 0) wrap_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, v, box);
    return cudaGetLastError();
}

cudaError_t launch_drift(int64_t n, double *x, double *y, double *z, const double *vx,
                         const double *vy, const double *vz, const double *sc, cudaStream_t st) {
    drift_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, x, y, z, vx, vy, vz, sc);
    return cudaGetLastError();
}

cudaError_t launch_rk4(double *sc, const Cosmo &c, cudaStream_t st) {
    rk4_kernel<<<1, 1, 0, st>>>(sc, c);
    return cudaGetLastError();
}

cudaError_t launch_timestep(int64_t n, const double *x, const double *y, const double *z,
                            const double *vx, const double *vy, const double *vz, const double *ax,
                            const double *ay, const double *az, const double *h, double *sc,
                            const Cosmo &c, double eps, double dt_max, double t_end, double *part,
                            int nblk, cudaStream_t st) {
    timestep_partial<<<nblk, 256, 0, st>>>(n, x, y, z, vx, vy, vz, ax, ay, az, h, sc, c, eps, part);
    timestep_finish<<<1, 1, 0, st>>>(nblk, part, dt_max, t_end, sc);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(double *sc, const double *dts, cudaStream_t st) {
    set_dt_kernel<<<1, 1, 0, st>>>(sc, dts);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(int64_t n, const double *vx, const double *vy, const double *vz,
                           const double *m, double *block_buf, int nblk, double *out,
                           cudaStream_t st) {
    kinetic_partial<<<nblk, 256, 0, st>>>(n, vx, vy, vz, m, block_buf);
    finish_partial<<<1, 32, 0, st>>>(nblk, 4, block_buf, out);
    return cudaGetLastError();
}

cudaError_t launch_sum(int64_t n, const double *v, double *block_buf, int nblk, double *out,
                       cudaStream_t st) {
    sum_partial<<<nblk, 256, 0, st>>>(n, v, block_buf);
    finish_partial<<<1, 32, 0, st>>>(nblk, 1, block_buf, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter3(int64_t n, const int64_t *perm, const double *a, const double *b,
                            const double *c, double *out3, cudaStream_t st) {
    scatter3_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, a, b, c, out3);
    return cudaGetLastError();
}

cudaError_t launch_gather3(int64_t n, const int64_t *perm, const double *in3, double *a, double *b,
                           double *c, cudaStream_t st) {
    gather3_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, in3, a, b, c);
    return cudaGetLastError();
}

cudaError_t launch_split3(int64_t n, const double *in3, double *a, double *b, double *c,
                          cudaStream_t st) {
    gather3_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, nullptr, in3, a, b, c);
    return cudaGetLastError();
}

cudaError_t launch_iota(int64_t n, int64_t *perm, cudaStream_t st) {
    iota_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, perm);
    return cudaGetLastError();
}

cudaError_t launch_softening(int64_t n, const double *m, double h_min, double *h, double *scratch,
                             cudaStream_t st) {
    min_kernel<<<1, 1024, 0, st>>>(n, m, scratch);
    softening_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, m, h_min, scratch, h);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(int64_t n, const double *a, int positive, int *flag,
                                cudaStream_t st) {
    finite_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, a, positive, flag);
    return cudaGetLastError();
}

cudaError_t launch_check_finite3(int64_t n, const double *a, const double *b, const double *c, int *flag,
                                 cudaStream_t st, const double *h) {
    const int64_t blocks = std::min<int64_t>(blocks_for(n, 256), 4 * 152);
    finite3_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(n, a, b, c, h, flag);
    return cudaGetLastError();
}

cudaError_t launch_set_scalar(double *sc, int slot, double v, cudaStream_t st) {
    set_scalar_kernel<<<1, 1, 0, st>>>(sc, slot, v);
    return cudaGetLastError();
}

}  // namespace steps

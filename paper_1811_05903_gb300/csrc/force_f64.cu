// FP64 direct-summation kernels on the GPU: the comparison variant of the
// pair term (Eq. 3, 4, 8 summed in FP64) and the FP64 pair potential used by
// the energy diagnostic.  Straightforward shared-memory tiling; the GB300's
// narrow FP64 pipe bounds both.
#include <cuda_runtime.h>
#include <stdint.h>

#include "steps_internal.h"

namespace steps {

namespace {

constexpr int kTB = 256;

// Fcal(r, H)/r of Eq. 4 for r < H, FP64 (same well-conditioned arrangement of
// the second branch around v = 1 - u as the FP32 path).
__device__ __forceinline__ double spline_over_r_f64(double r, double H) {
    const double Hinv = 1.0 / H;
    const double u = r * Hinv;
    double g;
    if (u < 0.5) {
        g = 32.0 / 3.0 + u * u * (32.0 * u - 38.4);
    } else {
        const double v = 1.0 - u;
        g = 16.0 / 15.0 + v * (3.2 + v * (6.4 + v * (32.0 / 3.0))) - 1.0 / (15.0 * u * u * u);
    }
    return g * Hinv * Hinv * Hinv;
}

// Pair potential per unit m_i m_j (antiderivative of Eq. 4; W = -1/r for r >= H).
__device__ __forceinline__ double pair_w_f64(double r, double H) {
    if (r >= H) return -1.0 / r;
    const double u = r / H, u2 = u * u;
    if (u < 0.5) return (-2.8 + u2 * (16.0 / 3.0 + u2 * (-9.6 + 6.4 * u))) / H;
    return (-3.2 + 1.0 / (15.0 * u) + u2 * (32.0 / 3.0 + u * (-16.0 + u * (9.6 - 32.0 / 15.0 * u)))) / H;
}

__global__ void __launch_bounds__(kTB) force_f64_kernel(int64_t n, const double *__restrict__ x,
                                                      const double *__restrict__ y,
                                                      const double *__restrict__ z,
                                                      const double *__restrict__ m,
                                                      const double *__restrict__ h, double G,
                                                      int64_t i0, int64_t i1,
                                                      double *__restrict__ ax,
                                                      double *__restrict__ ay,
                                                      double *__restrict__ az) {
    __shared__ double sx[kTB], sy[kTB], sz[kTB], sm[kTB], shh[kTB];
    const int64_t i = i0 + (int64_t)blockIdx.x * kTB + threadIdx.x;
    const bool valid = i < i1;
    const double xi = valid ? x[i] : 0.0, yi = valid ? y[i] : 0.0, zi = valid ? z[i] : 0.0;
    const double hi = valid ? h[i] : 0.0;
    double accx = 0.0, accy = 0.0, accz = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kTB) {
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
            sx[threadIdx.x] = x[j];
            sy[threadIdx.x] = y[j];
            sz[threadIdx.x] = z[j];
            sm[threadIdx.x] = m[j];
            shh[threadIdx.x] = h[j];
        } else {
            sx[threadIdx.x] = sy[threadIdx.x] = sz[threadIdx.x] = 0.0;
            sm[threadIdx.x] = 0.0;
            shh[threadIdx.x] = 1.0;
        }
        __syncthreads();
        const int cnt = (n - j0 < kTB) ? (int)(n - j0) : kTB;
        for (int jj = 0; jj < cnt; ++jj) {
            const double dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.0) {
                const double H = hi + shh[jj];
                const double ri = rsqrt(r2);
                const double g = (r2 >= H * H) ? ri * ri * ri : spline_over_r_f64(r2 * ri, H);
                const double s = sm[jj] * g;
                accx += s * dx;
                accy += s * dy;
                accz += s * dz;
            }
        }
        __syncthreads();
    }
    if (valid) {
        ax[i] = G * accx;
        ay[i] = G * accy;
        az[i] = G * accz;
    }
}

__global__ void __launch_bounds__(kTB) potential_f64_kernel(
    int64_t n, const double *__restrict__ x, const double *__restrict__ y,
    const double *__restrict__ z, const double *__restrict__ m, const double *__restrict__ h,
    double G, double *__restrict__ row) {
    __shared__ double sx[kTB], sy[kTB], sz[kTB], sm[kTB], shh[kTB];
    const int64_t i = (int64_t)blockIdx.x * kTB + threadIdx.x;
    const bool valid = i < n;
    const double xi = valid ? x[i] : 0.0, yi = valid ? y[i] : 0.0, zi = valid ? z[i] : 0.0;
    const double hi = valid ? h[i] : 0.0;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kTB) {
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
            sx[threadIdx.x] = x[j];
            sy[threadIdx.x] = y[j];
            sz[threadIdx.x] = z[j];
            sm[threadIdx.x] = m[j];
            shh[threadIdx.x] = h[j];
        }
        __syncthreads();
        const int cnt = (n - j0 < kTB) ? (int)(n - j0) : kTB;
        for (int jj = 0; jj < cnt; ++jj) {
            if (j0 + jj == i) continue;
            const double dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            acc += sm[jj] * pair_w_f64(r, hi + shh[jj]);
        }
        __syncthreads();
    }
    if (valid) row[i] = G * m[i] * acc;
}

// FP64 pair term for an explicit list of targets (sorted indices); rows of
// out3 follow the list order.  One warp per target, lanes stride over j and
// the 32 lane sums are combined by a shuffle tree.  The kernel is bound by
// the GB300's FP64 pipe (19 FP64 instructions per interaction: 4 DADD, 7 DMUL,
// 8 DFMA counted by ncu).  A variant with shared-memory source tiles and two
// targets per thread ran 4.5 times slower and, summing 2^20 terms in one
// sequential chain per target, less accurately; it is not built.
__global__ void force_f64_list_kernel(int64_t n, const double *__restrict__ x,
                                      const double *__restrict__ y, const double *__restrict__ z,
                                      const double *__restrict__ m, const double *__restrict__ h,
                                      double G, int64_t nt, const int64_t *__restrict__ idx,
                                      double *__restrict__ out3) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;
    const int64_t i = idx[t];
    const double xi = x[i], yi = y[i], zi = z[i], hi = h[i];
    double accx = 0.0, accy = 0.0, accz = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        const double dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > 0.0) {
            const double H = hi + h[j];
            const double ri = rsqrt(r2);
            const double g = (r2 >= H * H) ? ri * ri * ri : spline_over_r_f64(r2 * ri, H);
            const double s = m[j] * g;
            accx += s * dx;
            accy += s * dy;
            accz += s * dz;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        accx += __shfl_xor_sync(0xffffffffu, accx, o);
        accy += __shfl_xor_sync(0xffffffffu, accy, o);
        accz += __shfl_xor_sync(0xffffffffu, accz, o);
    }
    if (lane == 0) {
        out3[3 * t] = G * accx;
        out3[3 * t + 1] = G * accy;
        out3[3 * t + 2] = G * accz;
    }
}

__global__ void invert_perm_kernel(int64_t n, const int64_t *__restrict__ perm, int64_t *__restrict__ inv) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) inv[perm[k]] = k;
}

__global__ void map_targets_kernel(int64_t nt, const int64_t *__restrict__ inv,
                                   const int64_t *__restrict__ caller, int64_t *__restrict__ out,
                                   int64_t n, int *bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t c = caller[t];
    if (c < 0 || c >= n) {
        atomicOr(bad, 1);
        out[t] = 0;
        return;
    }
    out[t] = inv[c];
}

}  // namespace

cudaError_t launch_force_f64_list(int64_t n, const double *x, const double *y, const double *z,
                                  const double *m, const double *h, double G, int64_t nt,
                                  const int64_t *idx, double *out3, cudaStream_t st) {
    if (nt <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((nt * 32 + 255) / 256);
    force_f64_list_kernel<<<blocks, 256, 0, st>>>(n, x, y, z, m, h, G, nt, idx, out3);
    return cudaGetLastError();
}

cudaError_t launch_map_targets(int64_t n, const int64_t *perm, int64_t *inv, int64_t nt,
                               const int64_t *caller, int64_t *out, int *bad, cudaStream_t st) {
    invert_perm_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, perm, inv);
    if (nt > 0)
        map_targets_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, inv, caller, out, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_force_f64(int64_t n, const double *x, const double *y, const double *z,
                             const double *m, const double *h, double G, int64_t i0, int64_t i1,
                             double *ax, double *ay, double *az, cudaStream_t st) {
    if (i1 <= i0) return cudaSuccess;
    const unsigned blocks = (unsigned)((i1 - i0 + kTB - 1) / kTB);
    force_f64_kernel<<<blocks, kTB, 0, st>>>(n, x, y, z, m, h, G, i0, i1, ax, ay, az);
    return cudaGetLastError();
}

cudaError_t launch_potential_f64(int64_t n, const double *x, const double *y, const double *z,
                                 const double *m, const double *h, double G, double *row,
                                 cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + kTB - 1) / kTB);
    potential_f64_kernel<<<blocks, kTB, 0, st>>>(n, x, y, z, m, h, G, row);
    return cudaGetLastError();
}

}  // namespace steps

// Periodic pair term (Sec. 2.2): Eq. 2 with the image sum of Eq. 5,
//   acc_i = G sum_{j != i} m_j sum_n Fcal(|x_j + nL - x_i|, h_i + h_j) (x_j + nL - x_i) / r,
// over the images n with |x_i - x_j - nL| < 2.6 L (the paper's cut), or, for
// quasi-periodic boundaries, only the leading image: the n with
// x_i - x_j - nL in [-L/2, L/2)^3, n = floor((x_i - x_j) / L + 1/2) per component.
//
// FP32 path.  Positions are the FP32 tile staging of the open-boundary path
// (offset o and residual r from an FP32 tile centre c).  For a target tile I,
// a source tile J and an image n, the shift c_I - (c_J + nL) is formed in FP64
// and split into an FP32 value and its FP32 remainder; the pair separation is
// then carried to ~1 ulp of its own size as in the near-field kernel (exact
// rounding errors of the shifted target, both offset residuals).  Whether a
// (pair, image) term belongs to the sum is a hard decision: it is taken on the
// FP32 separation, except within a thin band around the cut sphere (or the
// half-box faces) where it is re-taken in FP64 from the FP64 positions with the
// definition's own expression, so that it matches an FP64 evaluation of the
// definition; images whose whole tile box lies inside the cut sphere (or inside
// the half-box region) skip the per-pair decision.  Each warp owns one target
// tile and a chunk of source tiles (a work item); FP32 partial sums are
// Kahan-folded every 8 sources across all images of a source tile and then
// added into FP64 per-target sums, written per work item and added in item
// order by the reduction kernel: deterministic.
//
// FP64 path.  One thread per target, every source, the image loops of the
// definition in FP64 without contraction (the comparison variant).
#include <cuda_runtime.h>
#include <stdint.h>

#include "steps_internal.h"

namespace steps {
namespace {

constexpr int kWarps = 4;
constexpr int kFold = 8;
constexpr float kCutBand = 4e-6f;  // relative band around (2.6 L)^2 decided in FP64
constexpr float kFaceBand = 2e-6f; // band around +-L/2 (in units of L) decided in FP64

__device__ __forceinline__ float two_sum_f(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ float rsqrt_f(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Fcal(r, H)/r of Eq. 4 for r < H (FP32; second branch arranged around v = 1 - u).
__device__ __forceinline__ float spline_over_r_f(float r, float H) {
    const float Hinv = __frcp_rn(H);
    const float u = r * Hinv;
    const float Hinv3 = Hinv * Hinv * Hinv;
    float g;
    if (u < 0.5f) {
        g = 32.0f / 3.0f + u * u * (32.0f * u - 38.4f);
    } else {
        const float v = 1.0f - u;
        g = 16.0f / 15.0f + v * (3.2f + v * (6.4f + v * (32.0f / 3.0f))) - __frcp_rn(15.0f * u * u * u);
    }
    return g * Hinv3;
}

__device__ __forceinline__ double spline_over_r_d(double r, double H) {
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

// Image k of the candidate table: cut sum |n_c| <= 3 (7^3 entries; a term needs
// |n_c| L < 2.6 L + |x_i - x_j|_c < 3.6 L), quasi-periodic |n_c| <= 1 (27).
__device__ __forceinline__ void image_of(int k, int images, int &nx, int &ny, int &nz) {
    if (images == 1) {
        nx = k / 9 - 1;
        ny = (k / 3) % 3 - 1;
        nz = k % 3 - 1;
    } else {
        nx = k / 49 - 3;
        ny = (k / 7) % 7 - 3;
        nz = k % 7 - 3;
    }
}

// The definition's decision in FP64, with the oracle's expression (no contraction).
__device__ __noinline__ bool include_f64(double xi, double yi, double zi, double xj, double yj, double zj, int nx,
                                        int ny, int nz, double L, int images) {
    const double d0x = __dsub_rn(xi, xj), d0y = __dsub_rn(yi, yj), d0z = __dsub_rn(zi, zj);
    if (images == 1) {
        return floor(__dadd_rn(__ddiv_rn(d0x, L), 0.5)) == (double)nx &&
               floor(__dadd_rn(__ddiv_rn(d0y, L), 0.5)) == (double)ny &&
               floor(__dadd_rn(__ddiv_rn(d0z, L), 0.5)) == (double)nz;
    }
    const double dx = __dsub_rn(d0x, __dmul_rn((double)nx, L));
    const double dy = __dsub_rn(d0y, __dmul_rn((double)ny, L));
    const double dz = __dsub_rn(d0z, __dmul_rn((double)nz, L));
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double cut = __dmul_rn(2.6, L);
    return r2 < __dmul_rn(cut, cut);
}

// The terms of one (source tile, image) for this lane's KI targets, added to
// the targets' compensated sums (folded every kFold sources).  Each source is
// read once from shared memory and used for all KI targets.  DECIDE: some
// pairs of this image may fall outside the cut sphere (or the half-box
// region), so every term is tested; otherwise every pair is a term.
template <int KI, int T, bool DECIDE>
__device__ __forceinline__ void image_terms(const float4 *__restrict__ S, const PeriodicArgs &a,
                                            const float (&nxs)[KI], const float (&nys)[KI], const float (&nzs)[KI],
                                            const float (&nrx)[KI], const float (&nry)[KI], const float (&nrz)[KI],
                                            const float (&hI)[KI], const int64_t (&gi)[KI], int64_t J, int nx,
                                            int ny, int nz, bool self_tile, int lane, float cut2, float halfL,
                                            float L, float (&kh)[KI][3], float (&kc)[KI][3]) {
    for (int f0 = 0; f0 < T; f0 += kFold) {
        float px[KI], py[KI], pz[KI];
#pragma unroll
        for (int t = 0; t < KI; ++t) px[t] = py[t] = pz[t] = 0.f;
#pragma unroll 2
        for (int j = f0; j < f0 + kFold; ++j) {
            const float4 A = S[2 * j], B = S[2 * j + 1];
            const float4 RA = S[2 * T + 2 * j], RB = S[2 * T + 2 * j + 1];
            if (B.z == 0.f) continue;  // padding source (zero mass)
#pragma unroll
            for (int t = 0; t < KI; ++t) {
                // d = x_j + nL - x_i
                const float dx = (A.x + nxs[t]) + (RA.x + nrx[t]);
                const float dy = (A.z + nys[t]) + (RA.z + nry[t]);
                const float dz = (B.x + nzs[t]) + (RB.x + nrz[t]);
                const float r2 = dx * dx + dy * dy + dz * dz;
                bool in = r2 > 0.f && !(self_tile && j == lane * KI + t);  // no self pair, no self images
                if (DECIDE && in) {
                    bool ambiguous;
                    if (a.images == 1) {
                        // x_i - x_j - nL = -d in [-L/2, L/2)  <=>  d in (-L/2, L/2]
                        in = dx > -halfL && dx <= halfL && dy > -halfL && dy <= halfL && dz > -halfL && dz <= halfL;
                        const float band = kFaceBand * L;
                        ambiguous = fabsf(fabsf(dx) - halfL) < band || fabsf(fabsf(dy) - halfL) < band ||
                                    fabsf(fabsf(dz) - halfL) < band;
                    } else {
                        in = r2 < cut2;
                        ambiguous = fabsf(r2 - cut2) < kCutBand * cut2;
                    }
                    if (ambiguous) {
                        const int64_t gj = J * T + j;
                        in = gi[t] < a.n && include_f64(a.x[gi[t]], a.y[gi[t]], a.z[gi[t]], a.x[gj], a.y[gj],
                                                         a.z[gj], nx, ny, nz, a.L, a.images);
                    }
                }
                if (!in) continue;
                const float H = hI[t] + RB.z;
                const float ri = rsqrt_f(r2);
                const float g = (r2 >= H * H) ? ri * ri * ri : spline_over_r_f(r2 * ri, H);
                const float sc = B.z * g;
                px[t] = fmaf(sc, dx, px[t]);
                py[t] = fmaf(sc, dy, py[t]);
                pz[t] = fmaf(sc, dz, pz[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < KI; ++t) {
            const float p[3] = {px[t], py[t], pz[t]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {  // Kahan fold
                const float y = p[c] - kc[t][c], tt = kh[t][c] + y;
                kc[t][c] = (tt - kh[t][c]) - y;
                kh[t][c] = tt;
            }
        }
    }
}

template <int KI>
__global__ void __launch_bounds__(32 * kWarps) periodic_f32_kernel(const PeriodicArgs a) {
    constexpr int T = 32 * KI;
    __shared__ float4 sbuf[kWarps][4 * T];  // per warp: jdup tile [2T] | rdup tile [2T]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarps + warp;
    if (item >= a.ntile * a.nchunk) return;
    const int64_t I = item / a.nchunk, ch = item % a.nchunk;
    const int64_t J0 = ch * a.ntile / a.nchunk, J1 = (ch + 1) * a.ntile / a.nchunk;
    float4 *S = sbuf[warp];
    const float L = (float)a.L;
    const float cut2 = (float)(2.6 * a.L) * (float)(2.6 * a.L);
    const float halfL = 0.5f * L;
    const int nimg = a.images == 1 ? 27 : 343;

    // this lane's targets: offsets, residuals, softening, global index
    float xi[KI], yi[KI], zi[KI], rxi[KI], ryi[KI], rzi[KI], hI[KI];
    int64_t gi[KI];
    double acc[KI][3];
#pragma unroll
    for (int t = 0; t < KI; ++t) {
        gi[t] = I * T + lane * KI + t;
        const float4 p = a.jdup[2 * gi[t]], pz = a.jdup[2 * gi[t] + 1];
        const float4 r = a.rdup[2 * gi[t]], rz = a.rdup[2 * gi[t] + 1];
        xi[t] = p.x;
        yi[t] = p.z;
        zi[t] = pz.x;
        rxi[t] = r.x;
        ryi[t] = r.z;
        rzi[t] = rz.x;
        hI[t] = rz.z;
        acc[t][0] = acc[t][1] = acc[t][2] = 0.0;
    }
    const float4 ci = a.tbox_c[I], ei = a.tbox_e[I];

    for (int64_t J = J0; J < J1; ++J) {
        __syncwarp();
        for (int k = lane; k < 2 * T; k += 32) {
            S[k] = a.jdup[2 * J * T + k];
            S[2 * T + k] = a.rdup[2 * J * T + k];
        }
        __syncwarp();
        const float4 cj = a.tbox_c[J], ej = a.tbox_e[J];
        // compensated FP32 sums over all images and sources of tile J, one FP64 add per tile
        float kh[KI][3], kc[KI][3];
#pragma unroll
        for (int t = 0; t < KI; ++t)
            for (int c = 0; c < 3; ++c) kh[t][c] = kc[t][c] = 0.f;
        for (int k0 = 0; k0 < nimg; k0 += 32) {
            // which images of tile J can hold a term for tile I (box test, FP64), and
            // which hold every pair of the two tiles (no per-pair decision needed)
            bool cand = false, all_in = false;
            const int k = k0 + lane;
            if (k < nimg) {
                int nx, ny, nz;
                image_of(k, a.images, nx, ny, nz);
                const double sx = (double)ci.x - ((double)cj.x + nx * a.L);
                const double sy = (double)ci.y - ((double)cj.y + ny * a.L);
                const double sz = (double)ci.z - ((double)cj.z + nz * a.L);
                const double wx = (double)ei.x + ej.x, wy = (double)ei.y + ej.y, wz = (double)ei.z + ej.z;
                const double margin = 1e-6 * a.L;
                if (a.images == 1) {
                    // some pair separation x_i - x_j - nL may lie in [-L/2, L/2]^3
                    cand = fabs(sx) <= 0.5 * a.L + wx + margin && fabs(sy) <= 0.5 * a.L + wy + margin &&
                           fabs(sz) <= 0.5 * a.L + wz + margin;
                    all_in = fabs(sx) + wx < 0.5 * a.L - margin && fabs(sy) + wy < 0.5 * a.L - margin &&
                             fabs(sz) + wz < 0.5 * a.L - margin;
                } else {
                    const double gx = fmax(0.0, fabs(sx) - wx), gy = fmax(0.0, fabs(sy) - wy),
                                 gz = fmax(0.0, fabs(sz) - wz);
                    const double cutm = 2.6 * a.L + margin, cutn = 2.6 * a.L - margin;
                    cand = gx * gx + gy * gy + gz * gz < cutm * cutm;
                    const double fx = fabs(sx) + wx, fy = fabs(sy) + wy, fz = fabs(sz) + wz;
                    all_in = fx * fx + fy * fy + fz * fz < cutn * cutn;
                }
            }
            unsigned mask = __ballot_sync(0xffffffffu, cand);
            const unsigned inside = __ballot_sync(0xffffffffu, all_in);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                int nx, ny, nz;
                image_of(k0 + b, a.images, nx, ny, nz);
                // c_I - (c_J + nL) in FP64, split into an FP32 value and its remainder
                const double dcx = (double)ci.x - ((double)cj.x + nx * a.L);
                const double dcy = (double)ci.y - ((double)cj.y + ny * a.L);
                const double dcz = (double)ci.z - ((double)cj.z + nz * a.L);
                const float hx = (float)dcx, hy = (float)dcy, hz = (float)dcz;
                const float lx = (float)(dcx - hx), ly = (float)(dcy - hy), lz = (float)(dcz - hz);
                const bool self_tile = (J == I) && (nx | ny | nz);
                const bool decide = !((inside >> b) & 1u);
                // -(s), s = fl(o_i + dc), and -(r_i + remainder(dc) + err(s)), per target
                float nxs[KI], nys[KI], nzs[KI], nrx[KI], nry[KI], nrz[KI];
#pragma unroll
                for (int t = 0; t < KI; ++t) {
                    float e;
                    nxs[t] = -two_sum_f(xi[t], hx, e);
                    nrx[t] = -((rxi[t] + lx) + e);
                    nys[t] = -two_sum_f(yi[t], hy, e);
                    nry[t] = -((ryi[t] + ly) + e);
                    nzs[t] = -two_sum_f(zi[t], hz, e);
                    nrz[t] = -((rzi[t] + lz) + e);
                }
                if (decide)
                    image_terms<KI, T, true>(S, a, nxs, nys, nzs, nrx, nry, nrz, hI, gi, J, nx, ny, nz, self_tile,
                                             lane, cut2, halfL, L, kh, kc);
                else
                    image_terms<KI, T, false>(S, a, nxs, nys, nzs, nrx, nry, nrz, hI, gi, J, nx, ny, nz, self_tile,
                                              lane, cut2, halfL, L, kh, kc);
            }
        }
#pragma unroll
        for (int t = 0; t < KI; ++t)
            for (int c = 0; c < 3; ++c) acc[t][c] += (double)kh[t][c] - (double)kc[t][c];
    }
    double *P = a.item_part + (size_t)item * 3 * T;
#pragma unroll
    for (int t = 0; t < KI; ++t) {
        const int li = lane * KI + t;
        P[li] = acc[t][0];
        P[T + li] = acc[t][1];
        P[2 * T + li] = acc[t][2];
    }
}

// Sum each target's work items in item order and apply G (sorted order).
__global__ void periodic_reduce_kernel(const double *__restrict__ item_part, int64_t n, int T, int64_t nchunk,
                                       double G, double *__restrict__ ax, double *__restrict__ ay,
                                       double *__restrict__ az) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t I = p / T;
    const int li = (int)(p - I * T);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t ch = 0; ch < nchunk; ++ch) {
        const double *Q = item_part + (size_t)(I * nchunk + ch) * 3 * T;
        sx += Q[li];
        sy += Q[T + li];
        sz += Q[2 * T + li];
    }
    ax[p] = G * sx;
    ay[p] = G * sy;
    az[p] = G * sz;
}

// FP64 comparison path: the definition's loops, one thread per target.
__global__ void __launch_bounds__(128) periodic_f64_kernel(int64_t n, const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ m,
                                                         const double *__restrict__ h, double G, double L,
                                                         int images, double *__restrict__ ax,
                                                         double *__restrict__ ay, double *__restrict__ az) {
    __shared__ double sx[128], sy[128], sz[128], sm[128], shh[128];
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const bool valid = i < n;
    const double xi = valid ? x[i] : 0.0, yi = valid ? y[i] : 0.0, zi = valid ? z[i] : 0.0;
    const double hi = valid ? h[i] : 0.0;
    const double cut = __dmul_rn(2.6, L), cut2 = __dmul_rn(cut, cut);
    double accx = 0.0, accy = 0.0, accz = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += 128) {
        const int64_t jl = j0 + threadIdx.x;
        __syncthreads();
        if (jl < n) {
            sx[threadIdx.x] = x[jl];
            sy[threadIdx.x] = y[jl];
            sz[threadIdx.x] = z[jl];
            sm[threadIdx.x] = m[jl];
            shh[threadIdx.x] = h[jl];
        }
        __syncthreads();
        const int cnt = (n - j0 < 128) ? (int)(n - j0) : 128;
        if (!valid) continue;
        for (int jj = 0; jj < cnt; ++jj) {
            if (j0 + jj == i) continue;
            const double d0x = __dsub_rn(xi, sx[jj]), d0y = __dsub_rn(yi, sy[jj]), d0z = __dsub_rn(zi, sz[jj]);
            const double H = hi + shh[jj];
            auto add = [&](double dx, double dy, double dz) {
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 > 0.0)) return;
                const double ri = rsqrt(r2);
                const double g = (r2 >= H * H) ? ri * ri * ri : spline_over_r_d(r2 * ri, H);
                const double s = sm[jj] * g;
                accx -= s * dx;  // d = x_i - x_j - nL points away from the source
                accy -= s * dy;
                accz -= s * dz;
            };
            if (images == 1) {
                const double nx = floor(__dadd_rn(__ddiv_rn(d0x, L), 0.5));
                const double ny = floor(__dadd_rn(__ddiv_rn(d0y, L), 0.5));
                const double nz = floor(__dadd_rn(__ddiv_rn(d0z, L), 0.5));
                add(__dsub_rn(d0x, __dmul_rn(nx, L)), __dsub_rn(d0y, __dmul_rn(ny, L)),
                    __dsub_rn(d0z, __dmul_rn(nz, L)));
                continue;
            }
            const int ax0 = (int)floor((d0x - cut) / L), ax1 = (int)ceil((d0x + cut) / L);
            const int ay0 = (int)floor((d0y - cut) / L), ay1 = (int)ceil((d0y + cut) / L);
            const int az0 = (int)floor((d0z - cut) / L), az1 = (int)ceil((d0z + cut) / L);
            for (int nx = ax0; nx <= ax1; ++nx)
                for (int ny = ay0; ny <= ay1; ++ny)
                    for (int nz = az0; nz <= az1; ++nz) {
                        const double dx = __dsub_rn(d0x, __dmul_rn((double)nx, L));
                        const double dy = __dsub_rn(d0y, __dmul_rn((double)ny, L));
                        const double dz = __dsub_rn(d0z, __dmul_rn((double)nz, L));
                        const double r2 =
                            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                        if (r2 < cut2) add(dx, dy, dz);
                    }
        }
    }
    if (valid) {
        ax[i] = G * accx;
        ay[i] = G * accy;
        az[i] = G * accz;
    }
}

}  // namespace

int64_t periodic_chunks(int64_t ntile) { return ntile < 8 ? ntile : 8; }

cudaError_t launch_periodic_f32(const Staging &s, const double *x, const double *y, const double *z, double L,
                                int images, double G, double *item_part, double *ax, double *ay, double *az,
                                cudaStream_t st) {
    PeriodicArgs a;
    a.jdup = s.jdup;
    a.rdup = s.rdup;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.x = x;
    a.y = y;
    a.z = z;
    a.item_part = item_part;
    a.ntile = s.ntile;
    a.nchunk = periodic_chunks(s.ntile);
    a.n = s.n;
    a.L = L;
    a.images = images;
    const int64_t items = a.ntile * a.nchunk;
    const unsigned blocks = (unsigned)((items + kWarps - 1) / kWarps);
    switch (s.T) {
        case 64: periodic_f32_kernel<2><<<blocks, 32 * kWarps, 0, st>>>(a); break;
        case 128: periodic_f32_kernel<4><<<blocks, 32 * kWarps, 0, st>>>(a); break;
        case 192: periodic_f32_kernel<6><<<blocks, 32 * kWarps, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    periodic_reduce_kernel<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(item_part, s.n, s.T, a.nchunk, G, ax, ay,
                                                                         az);
    return cudaGetLastError();
}

cudaError_t launch_periodic_f64(int64_t n, const double *x, const double *y, const double *z, const double *m,
                                const double *h, double G, double L, int images, double *ax, double *ay,
                                double *az, cudaStream_t st) {
    periodic_f64_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, x, y, z, m, h, G, L, images, ax, ay, az);
    return cudaGetLastError();
}

}  // namespace steps

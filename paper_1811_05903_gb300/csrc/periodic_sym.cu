// Symmetric FP32 periodic pair term (Sec. 2.2): Eq. 2 with the image sum of
// Eq. 5 cut at |x_i - x_j - nL| < 2.6 L, for the images whose pairs are all
// Newtonian.
//
// The term of particle j's image n on particle i, m_j d / r^3 with
// d = x_j + nL - x_i, and the term of particle i's image -n on particle j are
// the same separation with opposite sign, and the cut test |d| < 2.6 L is the
// same test.  So every (tile pair I < J, image n) -- and, for a tile with
// itself, every image in the positive half n > 0 (lexicographic) -- is
// evaluated once and its force is added to both particles.  For a tile with
// itself the pair of each particle with its own image is left out (the
// definition sums over j != i).
//
// Coordinates are in box units (L = 1) with tile centres on a grid of
// 2^-21, so c_I - c_J - n is exact in FP32 and the separation
// (o_j - o_i) - (c_I - c_J - n) is rounded relative to itself only.
//
// Work: the images of every tile pair are sorted by box tests
// (periodic_class.cuh) into none / inside the cut sphere / straddling it /
// soft (some pair may lie within h_i + h_j, or the n = 0 image of a tile with
// itself).  This kernel takes the inside and straddling images; the soft ones
// stay with the per-target kernel (periodic.cu), which classifies with the same
// function.  A count pass stores each tile pair's work units (slices of at
// most kSlice of its images) and a bound on each tile's sums; a scan turns the
// unit counts into offsets; persistent warps take units from a global counter,
// so that the warps the schedulers favour take more of them.
//
// Inside a warp (as in the open-boundary symmetric kernel): the target tile's
// 128 particles, 4 per lane as 2 packed pairs; the source tile in shared
// memory, 2 sources per lane and step, the sources' running sums passed lane to
// lane by shuffles (the two packed target halves added first: one shuffle per
// component); two images per pass share o_j - o_i, the loads, the
// shuffles and the sums; target partials Kahan-folded every 32 sources, source
// sums Kahan-accumulated over the unit's images.  Straddling images keep a term
// when r^2 <= (2.6)^2 (1 - 1.5e-6) in FP32 and flag terms within the band
// (1 +- 1.5e-6) (2.6)^2; after each step a warp vote sends the lanes holding
// flagged terms to recompute that step's terms and decide the band ones in FP64
// from the FP64 positions with the definition's expression.  All sums go to
// 64-bit fixed point (red.global.add.u64) with a per-tile power-of-two scale
// from the count pass's bound; each unit starts and flushes its own sums, so
// the result does not depend on which warp takes which unit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pair_terms.cuh"
#include "periodic_class.cuh"
#include "steps_internal.h"

namespace steps {

namespace {

constexpr int kKI = 4;          // targets per lane: 128-particle tiles
constexpr int kT = 32 * kKI;    // particles per tile
constexpr int kNP = kKI / 2;    // packed target pairs per lane
constexpr int kKJ = 2;          // sources per lane and step
constexpr int kR = kKI / kKJ;   // rounds of 32 steps per image
constexpr int kFoldS = 16;      // steps (32 sources) per compensated fold of the target partials
constexpr int kWarpsS = 4;      // independent warps per CTA
constexpr int kMinBlocks = 3;   // CTAs per SM the register budget is sized for
constexpr int kUnroll = 2;      // steps unrolled
constexpr int kPass = 2;        // images per pass
constexpr int kSlice = 32;      // images per work unit at most
constexpr float kCut2 = 2.6f * 2.6f;
// Relative band around (2.6)^2 decided in FP64.  The FP32 r^2 of a pair near
// the cut is within 4.4e-7 relative of the exact value: offsets rounded once
// from FP64 (|o| <= 1/2 box), o_j - o_i and (o_j - o_i) - D rounded once each
// (D exact), three roundings in r^2; the band leaves a factor 3.4.
constexpr float kBandRel = 1.5e-6f;
// Quasi-periodic sum: band around the half-box faces, max_c |d_c| within
// 2e-6 of 1/2 (box units; the FP32 separation is within ~1e-7 of exact).
constexpr float kQuasiBand = 2e-6f;
constexpr uint16_t kStraddle = 0x8000;

struct PSymWarp {
    float4 sj[2 * kT];                   // source tile: per 32 particles, 32 x (ox, ox, oy, oy), 32 x (oz, oz, m, m)
    float4 myk[3 * kNP * 32];            // target sums: [component][pair][lane] (hi.x, hi.y, nc.x, nc.y)
    float2 myio[3 * kNP * 32];           // -(target offsets): [component][pair][lane]
    float2 srck[3 * kR * kKJ * 32];      // source sums: [component][round * kKJ + k][lane] (hi, nc)
    uint16_t lst[kPerImages + 1];        // images of the current tile pair: index | kStraddle
};

struct PSymArgs {
    const float4 *__restrict__ sdup;
    const float4 *__restrict__ tbox_c;
    const float4 *__restrict__ tbox_e;
    const double *__restrict__ x;
    const double *__restrict__ y;
    const double *__restrict__ z;
    const int64_t *__restrict__ uoff;  // [npairs + 1] first work unit of each tile pair
    unsigned long long *next;          // work-unit counter (zeroed by the scan)
    const float *__restrict__ tscale;  // [ntile]
    unsigned long long *__restrict__ acc;  // [3][np]
    int *nonfinite;
    int64_t ntile, npairs, np, n;
    double L;  // box length of x, y, z
};

// What the FP64 re-decision of a band term needs.
struct BandCtx {
    const double *x, *y, *z;
    unsigned long long *acc;
    int *nonfinite;
    int64_t np, n, I, J;
    double L;
    float scJ;
};

// Tile pairs (I <= J) in row-major order: row I starts at R(I).
__device__ __forceinline__ int64_t pair_row_start(int64_t I, int64_t ntile) {
    return I * ntile - I * (I - 1) / 2;
}

__device__ __forceinline__ void pair_of(int64_t p, int64_t ntile, int64_t &I, int64_t &J) {
    int64_t lo = 0, hi = ntile;  // R(lo) <= p < R(hi)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (pair_row_start(mid, ntile) <= p) lo = mid; else hi = mid;
    }
    I = lo;
    J = lo + (p - pair_row_start(lo, ntile));
}

// Candidate images of a tile pair: the cut sum's 343 or the quasi-periodic 27.
template <bool QUASI>
__device__ __forceinline__ void image_vec(int k, int &nx, int &ny, int &nz) {
    if (QUASI) quasi_image_of(k, nx, ny, nz); else periodic_image_of(k, nx, ny, nz);
}

template <bool QUASI>
__device__ __forceinline__ int image_class(const float4 ci, const float4 ei, const float4 cj, const float4 ej, int k,
                                           bool self, float *gap2) {
    int nx, ny, nz;
    image_vec<QUASI>(k, nx, ny, nz);
    return QUASI ? quasi_image_class(ci, ei, cj, ej, nx, ny, nz, self, gap2)
                 : periodic_image_class(ci, ei, cj, ej, nx, ny, nz, self, gap2);
}

// Whether image k of the tile pair (I, J), I <= J, is this kernel's work.
template <bool QUASI>
__device__ __forceinline__ int pair_image_class(const float4 ci, const float4 ei, const float4 cj, const float4 ej,
                                                bool self, int k, float *gap2) {
    *gap2 = 0.f;
    const int nimg = QUASI ? kQuasiImages : kPerImages, zero = QUASI ? kQuasiZeroImage : kPerZeroImage;
    if (k >= nimg || (self && k <= zero)) return kPerNone;
    return image_class<QUASI>(ci, ei, cj, ej, k, self, gap2);
}

__device__ __forceinline__ void red_fixed_p(unsigned long long *addr, float v, float sc, int *nonfinite) {
    if (!isfinite(v)) {
        if (nonfinite) *nonfinite = 1;
        return;
    }
    atomicAdd(addr, (unsigned long long)__float2ll_rn(v * sc));
}

// One warp per tile pair: its work units (slices of at most kSlice of the
// images this kernel evaluates), and the bound sum over those images of
// M / gap^2 for each side (gap: distance between the boxes, so every term is
// at most M / gap^2).
template <bool QUASI>
__global__ void psym_count_kernel(const float4 *__restrict__ tbox_c, const float4 *__restrict__ tbox_e,
                                  int64_t ntile, int64_t npairs, int64_t *__restrict__ uoff,
                                  float2 *__restrict__ bnd, int *__restrict__ soft) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= npairs) return;
    int64_t I, J;
    pair_of(p, ntile, I, J);
    const float4 ci = tbox_c[I], ei = tbox_e[I], cj = tbox_c[J], ej = tbox_e[J];
    int cnt = 0, nsoft = 0;
    double s = 0.0;
    const int nimg = QUASI ? kQuasiImages : kPerImages;
    for (int k0 = 0; k0 < nimg; k0 += 32) {
        const int k = k0 + lane;
        float gap2;
        const int cls = pair_image_class<QUASI>(ci, ei, cj, ej, I == J, k, &gap2);
        if (cls == kPerInside || cls == kPerStraddle) {
            ++cnt;
            s += 1.0 / (double)gap2;
        }
        // images the per-target kernel takes (either half for a tile with itself)
        if (k < nimg) nsoft += image_class<QUASI>(ci, ei, cj, ej, k, I == J, &gap2) == kPerSoft ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        nsoft += __shfl_xor_sync(0xffffffffu, nsoft, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
        soft[p] = nsoft;
        uoff[p + 1] = (cnt + kSlice - 1) / kSlice;
        // tile I feels tile J's mass and tile J feels tile I's; a tile with
        // itself feels both halves n and -n (equal gaps)
        bnd[p] = make_float2(__double2float_ru((double)ej.w * s), __double2float_ru((double)ei.w * s));
    }
}

// Inclusive scan of one value per thread over a 1,024-thread CTA.
__device__ __forceinline__ int64_t block_scan_1024(int64_t v, int64_t *part) {
    const int t = threadIdx.x;
    part[t] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int64_t w = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += w;
        __syncthreads();
    }
    const int64_t r = part[t];
    __syncthreads();
    return r;
}

// One CTA: unit counts -> offsets (uoff[0] = 0, uoff[p + 1] = units of pairs
// <= p), the work counter zeroed, each tile's fixed-point scale from the sum
// of its bounds (in a fixed order: with 2 B < 2^E every partial sum stays
// below 2^61 at scale 2^(62 - E)), and for every tile the list of tiles it
// shares a softened image with, in tile order (soff[I] .. soff[I + 1] into
// slist, at most cap entries; soff[ntile] is the total even beyond cap).
__global__ void __launch_bounds__(1024) psym_scan_kernel(int64_t *__restrict__ uoff, int64_t npairs,
                                                         unsigned long long *__restrict__ next,
                                                         const float2 *__restrict__ bnd, int64_t ntile,
                                                         float *__restrict__ tscale, double *__restrict__ tinv,
                                                         const int *__restrict__ soft, int64_t *__restrict__ soff,
                                                         int *__restrict__ slist, int64_t cap) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (npairs + 1023) / 1024;
    const int64_t b0 = t * chunk, b = b0 < npairs ? b0 : npairs;
    const int64_t e = b + chunk < npairs ? b + chunk : npairs;
    int64_t s = 0;
    for (int64_t p = b; p < e; ++p) s += uoff[p + 1];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // inclusive scan of the chunk sums
        const int64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t p = b; p < e; ++p) {
        run += uoff[p + 1];
        uoff[p + 1] = run;
    }
    if (t == 0) {
        uoff[0] = 0;
        *next = 0;
    }
    for (int64_t I = t; I < ntile; I += 1024) {
        double B = 0.0;
        for (int64_t J = I; J < ntile; ++J) B += (double)bnd[pair_row_start(I, ntile) + (J - I)].x;
        for (int64_t J = 0; J <= I; ++J) B += (double)bnd[pair_row_start(J, ntile) + (I - J)].y;
        int ex = -200;
        if (B > 0.0) frexp(2.0 * B, &ex);  // 2 B < 2^ex
        int sh = 62 - ex;
        sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
        tscale[I] = ldexpf(1.0f, sh);
        tinv[I] = ldexp(1.0, -sh);
    }
    // soft partner lists: contiguous tile ranges per thread
    const int64_t tch = (ntile + 1023) / 1024;
    const int64_t i0 = t * tch < ntile ? t * tch : ntile, i1 = i0 + tch < ntile ? i0 + tch : ntile;
    int64_t c = 0;
    for (int64_t I = i0; I < i1; ++I)
        for (int64_t J = 0; J < ntile; ++J)
            c += soft[I <= J ? pair_row_start(I, ntile) + (J - I) : pair_row_start(J, ntile) + (I - J)] > 0;
    int64_t o = block_scan_1024(c, part) - c;
    for (int64_t I = i0; I < i1; ++I) {
        soff[I] = o;
        for (int64_t J = 0; J < ntile; ++J) {
            if (soft[I <= J ? pair_row_start(I, ntile) + (J - I) : pair_row_start(J, ntile) + (I - J)] > 0) {
                if (o < cap) slist[o] = (int)J;
                ++o;
            }
        }
    }
    if (t == 1023) soff[ntile] = o;
}

// The band terms of one step (rare): this lane's terms of the step's kKJ
// sources are recomputed with the main loop's FP32 operations, and those in
// the band are decided in FP64 from the FP64 positions with the definition's
// expression.  The cut sum's decision is the same for both particles; the
// quasi-periodic one is taken for each side (the half-open interval makes the
// image of (j, i) differ from -n exactly on a face), and each side gets its
// term only when its own decision keeps it.
template <int M, bool QUASI>
__device__ __noinline__ void psym_band_step(const BandCtx &bc, PSymWarp &Wm, const float2 (&mi)[kNP],
                                            const float (&D)[M][3], const int (&nn)[M][3], int r, int st,
                                            int lane) {
    const float band = QUASI ? kQuasiBand : kBandRel * kCut2;
    const int g = (lane + st) & 31;
    for (int k = 0; k < kKJ; ++k) {
        const float4 A = Wm.sj[(r * kKJ + k) * 64 + g], B = Wm.sj[(r * kKJ + k) * 64 + 32 + g];
        const int64_t gj = bc.J * kT + (r * kKJ + k) * 32 + g;
        for (int t = 0; t < kKI; ++t) {
            const int q = t >> 1, e = t & 1;
            const float2 vx = Wm.myio[(0 * kNP + q) * 32 + lane], vy = Wm.myio[(1 * kNP + q) * 32 + lane],
                         vz = Wm.myio[(2 * kNP + q) * 32 + lane];
            const float ex = __fadd_rn(A.x, e ? vx.y : vx.x);
            const float ey = __fadd_rn(A.z, e ? vy.y : vy.x);
            const float ez = __fadd_rn(B.x, e ? vz.y : vz.x);
            const int64_t gi = bc.I * kT + 32 * t + lane;
            for (int im = 0; im < M; ++im) {
                const float dx = __fadd_rn(ex, -D[im][0]), dy = __fadd_rn(ey, -D[im][1]),
                            dz = __fadd_rn(ez, -D[im][2]);
                float r2 = __fmul_rn(dx, dx);
                r2 = __fmaf_rn(dy, dy, r2);
                r2 = __fmaf_rn(dz, dz, r2);
                const float u = QUASI ? __fadd_rn(fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))), -0.5f)
                                      : __fadd_rn(r2, -kCut2);
                if (!(fabsf(u) < band)) continue;
                if (gj == gi || gi >= bc.n || gj >= bc.n) continue;
                const bool in_t = include_f64(bc.x[gi], bc.y[gi], bc.z[gi], bc.x[gj], bc.y[gj], bc.z[gj], nn[im][0],
                                              nn[im][1], nn[im][2], bc.L, QUASI ? 1 : 0);
                const bool in_s = QUASI ? include_f64(bc.x[gj], bc.y[gj], bc.z[gj], bc.x[gi], bc.y[gi], bc.z[gi],
                                                      -nn[im][0], -nn[im][1], -nn[im][2], bc.L, 1)
                                        : in_t;
                if (!in_t && !in_s) continue;
                const float w = rsqrt_approx(r2);
                const float u3 = w * w * w;
                const float d3[3] = {dx, dy, dz};
                const float m_i = e ? mi[q].y : mi[q].x;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (in_t) {
                        float4 &K = Wm.myk[(c * kNP + q) * 32 + lane];
                        float hi = e ? K.y : K.x, nc = e ? K.w : K.z;
                        kahan1(hi, nc, u3 * B.z * d3[c]);
                        if (e) {
                            K.y = hi;
                            K.w = nc;
                        } else {
                            K.x = hi;
                            K.z = nc;
                        }
                    }
                    if (in_s) red_fixed_p(bc.acc + c * bc.np + gj, -(u3 * m_i * d3[c]), bc.scJ, bc.nonfinite);
                }
            }
        }
    }
}

// M images of the current tile pair for this warp in one pass: the tile's 128
// targets against the staged 128 sources, shifts D_m = c_I - c_J - n_m.  The
// offset difference o_j - o_i, the source loads, the shuffles and the source
// and target sums are shared by the M images; each image's separation is
// (o_j - o_i) - D_m, the same FP32 operations as for one image.  CUT: some
// image straddles the cut sphere (the test keeps every term of an image wholly
// inside); after each step a warp vote sends the lanes holding band terms to
// psym_band_step.  DIAG: a tile with itself; a particle meets its own image at
// step 0 of round r (target 2 r + k against source k of the step), and that
// pair is left out.
template <int M, bool CUT, bool DIAG, bool QUASI>
__device__ __forceinline__ void psym_images(PSymWarp &Wm, const float2 (&mi)[kNP], const float (&D)[M][3],
                                            const int (&nn)[M][3], const BandCtx &bc, const int lane) {
    float2 ndx[M], ndy[M], ndz[M];
#pragma unroll
    for (int im = 0; im < M; ++im) {
        ndx[im] = make_float2(-D[im][0], -D[im][0]);
        ndy[im] = make_float2(-D[im][1], -D[im][1]);
        ndz[im] = make_float2(-D[im][2], -D[im][2]);
    }
    const float2 ncut = make_float2(-kCut2, -kCut2);
    const float band = QUASI ? kQuasiBand : kBandRel * kCut2;
    const float2 nhalf = make_float2(-0.5f, -0.5f);
    float2 nox[kNP], noy[kNP], noz[kNP];
    float2 px[kNP], py[kNP], pz[kNP];
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        nox[q] = Wm.myio[(0 * kNP + q) * 32 + lane];
        noy[q] = Wm.myio[(1 * kNP + q) * 32 + lane];
        noz[q] = Wm.myio[(2 * kNP + q) * 32 + lane];
        px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
    }
    const int from = (lane + 1) & 31;
#pragma unroll 1
    for (int r = 0; r < kR; ++r) {
        float2 Sx[kKJ], Sy[kKJ], Sz[kKJ];
#pragma unroll
        for (int k = 0; k < kKJ; ++k) Sx[k] = Sy[k] = Sz[k] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int h = 0; h < 32; h += kFoldS) {
#pragma unroll kUnroll
            for (int st = h; st < h + kFoldS; ++st) {
                const int g = (lane + st) & 31;
                bool amb = false;
#pragma unroll
                for (int k = 0; k < kKJ; ++k) {
                    const float4 *src = Wm.sj + (r * kKJ + k) * 64 + g;
                    const float4 A = src[0], B = src[32];
                    const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
                    const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
                    float2 tx, ty, tz;
#pragma unroll
                    for (int q = 0; q < kNP; ++q) {
                        const float2 ex = __fadd2_rn(xj, nox[q]);  // o_j - o_i
                        const float2 ey = __fadd2_rn(yj, noy[q]);
                        const float2 ez = __fadd2_rn(zj, noz[q]);
#pragma unroll
                        for (int im = 0; im < M; ++im) {
                            const float2 dx = __fadd2_rn(ex, ndx[im]);  // x_j + n - x_i
                            const float2 dy = __fadd2_rn(ey, ndy[im]);
                            const float2 dz = __fadd2_rn(ez, ndz[im]);
                            float2 r2 = __fmul2_rn(dx, dx);
                            r2 = __ffma2_rn(dy, dy, r2);
                            r2 = __ffma2_rn(dz, dz, r2);
                            float2 w = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                            if (DIAG && q == r && st == 0) {
                                if (k == 0) w.x = 0.f; else w.y = 0.f;
                            }
                            if (CUT) {
                                // r^2 - (2.6)^2, or max_c |d_c| - 1/2 (quasi-periodic)
                                const float2 u =
                                    QUASI ? __fadd2_rn(make_float2(fmaxf(fabsf(dx.x), fmaxf(fabsf(dy.x), fabsf(dz.x))),
                                                                   fmaxf(fabsf(dx.y), fmaxf(fabsf(dy.y), fabsf(dz.y)))),
                                                       nhalf)
                                          : __fadd2_rn(r2, ncut);
                                amb = amb | (fabsf(u.x) < band) | (fabsf(u.y) < band);
                                w.x = u.x <= -band ? w.x : 0.f;
                                w.y = u.y <= -band ? w.y : 0.f;
                            }
                            const float2 u3 = __fmul2_rn(__fmul2_rn(w, w), w);  // 1/r^3
                            const float2 si = __fmul2_rn(u3, mj);
                            px[q] = __ffma2_rn(si, dx, px[q]);
                            py[q] = __ffma2_rn(si, dy, py[q]);
                            pz[q] = __ffma2_rn(si, dz, pz[q]);
                            const float2 sj = __fmul2_rn(u3, mi[q]);
                            if (q == 0 && im == 0) {
                                tx = __fmul2_rn(sj, dx);
                                ty = __fmul2_rn(sj, dy);
                                tz = __fmul2_rn(sj, dz);
                            } else {
                                tx = __ffma2_rn(sj, dx, tx);
                                ty = __ffma2_rn(sj, dy, ty);
                                tz = __ffma2_rn(sj, dz, tz);
                            }
                        }
                    }
                    // the two packed target halves are added before the rotation
                    Sx[k].x = __fadd_rn(Sx[k].x, __fadd_rn(tx.x, tx.y));
                    Sy[k].x = __fadd_rn(Sy[k].x, __fadd_rn(ty.x, ty.y));
                    Sz[k].x = __fadd_rn(Sz[k].x, __fadd_rn(tz.x, tz.y));
                }
#pragma unroll
                for (int k = 0; k < kKJ; ++k) {
                    Sx[k].x = __shfl_sync(0xffffffffu, Sx[k].x, from);
                    Sy[k].x = __shfl_sync(0xffffffffu, Sy[k].x, from);
                    Sz[k].x = __shfl_sync(0xffffffffu, Sz[k].x, from);
                }
                if (CUT && __any_sync(0xffffffffu, amb)) {
                    if (amb) psym_band_step<M, QUASI>(bc, Wm, mi, D, nn, r, st, lane);
                    __syncwarp();
                }
            }
#pragma unroll
            for (int q = 0; q < kNP; ++q) {
                float4 *K = Wm.myk + q * 32 + lane;
                float4 kx = K[0], ky = K[kNP * 32], kz = K[2 * kNP * 32];
                float2 hx = make_float2(kx.x, kx.y), cx = make_float2(kx.z, kx.w);
                float2 hy = make_float2(ky.x, ky.y), cy = make_float2(ky.z, ky.w);
                float2 hz = make_float2(kz.x, kz.y), cz = make_float2(kz.z, kz.w);
                kahan2(hx, cx, px[q]);
                kahan2(hy, cy, py[q]);
                kahan2(hz, cz, pz[q]);
                K[0] = make_float4(hx.x, hx.y, cx.x, cx.y);
                K[kNP * 32] = make_float4(hy.x, hy.y, cy.x, cy.y);
                K[2 * kNP * 32] = make_float4(hz.x, hz.y, cz.x, cz.y);
                px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
            }
        }
        // this lane holds the complete sums of sources (r, k, lane) for these images
#pragma unroll
        for (int k = 0; k < kKJ; ++k) {
            const float v[3] = {Sx[k].x + Sx[k].y, Sy[k].x + Sy[k].y, Sz[k].x + Sz[k].y};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 &S = Wm.srck[(c * kR * kKJ + r * kKJ + k) * 32 + lane];
                float hi = S.x, nc = S.y;
                kahan1(hi, nc, v[c]);
                S = make_float2(hi, nc);
            }
        }
    }
}

template <int M, bool QUASI>
__device__ __forceinline__ void psym_pass(PSymWarp &Wm, const float2 (&mi)[kNP], const float (&D)[M][3],
                                          const int (&nn)[M][3], const BandCtx &bc, bool cut, bool self,
                                          int lane) {
    if (cut) {
        if (self) psym_images<M, true, true, QUASI>(Wm, mi, D, nn, bc, lane);
        else psym_images<M, true, false, QUASI>(Wm, mi, D, nn, bc, lane);
    } else {
        if (self) psym_images<M, false, true, QUASI>(Wm, mi, D, nn, bc, lane);
        else psym_images<M, false, false, QUASI>(Wm, mi, D, nn, bc, lane);
    }
}

// Persistent warps take work units (a tile pair and a slice of its images)
// from a global counter, so that warps the scheduler favours take more units
// and all finish together.
template <bool QUASI>
__global__ void __launch_bounds__(kWarpsS * 32, kMinBlocks) psym_far_kernel(const PSymArgs a) {
    extern __shared__ __align__(16) unsigned char psym_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PSymWarp &Wm = reinterpret_cast<PSymWarp *>(psym_smem)[warp];
    const int64_t total = a.uoff[a.npairs];
    int64_t Icur = -1;
    float2 mi[kNP];
#pragma unroll
    for (int q = 0; q < kNP; ++q) mi[q] = make_float2(0.f, 0.f);
    BandCtx bc{a.x, a.y, a.z, a.acc, a.nonfinite, a.np, a.n, 0, 0, a.L, 0.f};

    auto flush_targets = [&](int64_t It) {
        __syncwarp();
        const float sc = a.tscale[It];
#pragma unroll
        for (int q = 0; q < kNP; ++q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 K = Wm.myk[(c * kNP + q) * 32 + lane];
                unsigned long long *dst = a.acc + c * a.np + It * kT + 64 * q + lane;
                red_fixed_p(dst, K.x, sc, a.nonfinite);
                red_fixed_p(dst, K.z, sc, a.nonfinite);
                red_fixed_p(dst + 32, K.y, sc, a.nonfinite);
                red_fixed_p(dst + 32, K.w, sc, a.nonfinite);
            }
        }
    };

    for (;;) {
        unsigned long long uu = 0;
        if (lane == 0) uu = atomicAdd(a.next, 1ull);
        const int64_t u = (int64_t)__shfl_sync(0xffffffffu, uu, 0);
        if (u >= total) break;
        int64_t p;
        {
            int64_t lo = 0, hi = a.npairs;  // uoff[lo] <= u < uoff[hi]
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (a.uoff[mid] <= u) lo = mid; else hi = mid;
            }
            p = lo;
        }
        const int64_t nu = a.uoff[p + 1] - a.uoff[p], sl = u - a.uoff[p];
        int64_t I, J;
        pair_of(p, a.ntile, I, J);
        __syncwarp();
        if (I != Icur) {
#pragma unroll
            for (int q = 0; q < kNP; ++q) {
                const float4 *p0 = a.sdup + (I * kKI + 2 * q) * 64 + lane;  // particle 64 q + lane
                const float4 *p1 = p0 + 64;                                  // particle 64 q + 32 + lane
                const float4 A0 = p0[0], B0 = p0[32], A1 = p1[0], B1 = p1[32];
                Wm.myio[(0 * kNP + q) * 32 + lane] = make_float2(-A0.x, -A1.x);
                Wm.myio[(1 * kNP + q) * 32 + lane] = make_float2(-A0.z, -A1.z);
                Wm.myio[(2 * kNP + q) * 32 + lane] = make_float2(-B0.x, -B1.x);
                mi[q] = make_float2(B0.z, B1.z);
            }
            Icur = I;
        }
        // the unit's sums start from zero and are flushed at its end, so the
        // result does not depend on which warp takes which unit
#pragma unroll
        for (int k = 0; k < 3 * kNP; ++k) Wm.myk[k * 32 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 *src = a.sdup + J * 2 * kT;
        for (int k = lane; k < 2 * kT; k += 32) Wm.sj[k] = src[k];
        for (int k = lane; k < 3 * kR * kKJ * 32; k += 32) Wm.srck[k] = make_float2(0.f, 0.f);
        // this tile pair's images, in index order within each class (the count pass's decisions)
        const float4 ci = a.tbox_c[I], ei = a.tbox_e[I], cj = a.tbox_c[J], ej = a.tbox_e[J];
        const bool self = I == J;
        int cnt = 0;
        for (int pass = 0; pass < 2; ++pass) {  // images wholly inside the cut sphere, then straddling ones
            const int want = pass == 0 ? kPerInside : kPerStraddle;
            for (int k0 = 0; k0 < (QUASI ? kQuasiImages : kPerImages); k0 += 32) {
                float gap2;
                const bool keep = pair_image_class<QUASI>(ci, ei, cj, ej, self, k0 + lane, &gap2) == want;
                const unsigned bk = __ballot_sync(0xffffffffu, keep);
                if (keep)
                    Wm.lst[cnt + __popc(bk & ((1u << lane) - 1u))] = (uint16_t)((k0 + lane) | (pass ? kStraddle : 0));
                cnt += __popc(bk);
            }
        }
        __syncwarp();
        const float dcx = __fsub_rn(ci.x, cj.x), dcy = __fsub_rn(ci.y, cj.y), dcz = __fsub_rn(ci.z, cj.z);
        const float scJ = a.tscale[J];
        bc.I = I;
        bc.J = J;
        bc.scJ = scJ;
        // this unit's slice of the list
        const int lo = (int)(sl * cnt / nu), hi = (int)((sl + 1) * cnt / nu);
        for (int l = lo; l < hi;) {
            const int M = (kPass == 2 && l + 1 < hi) ? 2 : 1;
            int nn[2][3];
            float D[2][3];
            bool cut = false;
            for (int im = 0; im < M; ++im) {
                const int code = Wm.lst[l + im];
                image_vec<QUASI>(code & 0x1ff, nn[im][0], nn[im][1], nn[im][2]);
                // exact: grid centres, integer n
                D[im][0] = __fsub_rn(dcx, (float)nn[im][0]);
                D[im][1] = __fsub_rn(dcy, (float)nn[im][1]);
                D[im][2] = __fsub_rn(dcz, (float)nn[im][2]);
                cut = cut || (code & kStraddle);
            }
            if (M == 2) {
                psym_pass<2, QUASI>(Wm, mi, D, nn, bc, cut, self, lane);
            } else {
                const float D1[1][3] = {{D[0][0], D[0][1], D[0][2]}};
                const int n1[1][3] = {{nn[0][0], nn[0][1], nn[0][2]}};
                psym_pass<1, QUASI>(Wm, mi, D1, n1, bc, cut, self, lane);
            }
            l += M;
        }
        // the target and source tiles' sums: force on j is minus the sum of m_i d / r^3
        flush_targets(I);
#pragma unroll
        for (int r = 0; r < kR; ++r) {
#pragma unroll
            for (int k = 0; k < kKJ; ++k) {
                const int64_t idx = J * kT + (r * kKJ + k) * 32 + lane;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 S = Wm.srck[(c * kR * kKJ + r * kKJ + k) * 32 + lane];
                    red_fixed_p(a.acc + c * a.np + idx, -S.x, scJ, a.nonfinite);
                    red_fixed_p(a.acc + c * a.np + idx, -S.y, scJ, a.nonfinite);
                }
            }
        }
    }
}

template <bool QUASI>
int psym_blocks_per_sm() {
    static int cached = 0;
    if (cached > 0) return cached;
    const size_t smem = sizeof(PSymWarp) * kWarpsS;
    cudaFuncSetAttribute(psym_far_kernel<QUASI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, psym_far_kernel<QUASI>, kWarpsS * 32, smem) !=
            cudaSuccess ||
        per < 1)
        per = 1;
    cached = per;
    return per;
}

}  // namespace

int64_t periodic_sym_pairs(int64_t ntile) { return ntile * (ntile + 1) / 2; }

int periodic_sym_tile() { return kT; }

cudaError_t launch_periodic_sym(const Staging &s, const double *x, const double *y, const double *z, double L,
                                int images, const PeriodicSymScratch &ps, int num_sms, cudaStream_t st) {
    const bool quasi = images == 1;
    if (s.T != kT || !s.sdup) return cudaErrorInvalidValue;
    const int64_t npairs = periodic_sym_pairs(s.ntile);
    cudaError_t e = cudaMemsetAsync(ps.acc, 0, sizeof(unsigned long long) * 3 * s.np, st);
    if (e != cudaSuccess) return e;
    const unsigned cblocks = (unsigned)((npairs * 32 + 255) / 256);
    if (quasi)
        psym_count_kernel<true><<<cblocks, 256, 0, st>>>(s.tbox_c, s.tbox_e, s.ntile, npairs, ps.off, ps.bnd, ps.soft);
    else
        psym_count_kernel<false><<<cblocks, 256, 0, st>>>(s.tbox_c, s.tbox_e, s.ntile, npairs, ps.off, ps.bnd, ps.soft);
    unsigned long long *next = reinterpret_cast<unsigned long long *>(ps.off + npairs + 1);
    psym_scan_kernel<<<1, 1024, 0, st>>>(ps.off, npairs, next, ps.bnd, s.ntile, ps.tscale, ps.tinv, ps.soft,
                                         ps.soff, ps.slist, ps.cap_items);
    PSymArgs a;
    a.sdup = s.sdup;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.x = x;
    a.y = y;
    a.z = z;
    a.uoff = ps.off;
    a.next = next;
    a.tscale = ps.tscale;
    a.acc = ps.acc;
    a.nonfinite = ps.nonfinite;
    a.ntile = s.ntile;
    a.npairs = npairs;
    a.np = s.np;
    a.n = s.n;
    a.L = L;
    const size_t smem = sizeof(PSymWarp) * kWarpsS;
    if (quasi)
        psym_far_kernel<true><<<std::max(num_sms, 1) * psym_blocks_per_sm<true>(), kWarpsS * 32, smem, st>>>(a);
    else
        psym_far_kernel<false><<<std::max(num_sms, 1) * psym_blocks_per_sm<false>(), kWarpsS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace steps

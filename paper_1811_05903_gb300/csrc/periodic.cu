// Periodic pair term (Sec. 2.2): Eq. 2 with the image sum of Eq. 5,
//   acc_i = G sum_{j != i} m_j sum_n Fcal(|x_j + nL - x_i|, h_i + h_j) (x_j + nL - x_i) / r,
// over the images n with |x_i - x_j - nL| < 2.6 L (the paper's cut), or, for
// quasi-periodic boundaries, only the leading image: the n with
// x_i - x_j - nL in [-L/2, L/2)^3, n = floor((x_i - x_j) / L + 1/2) per component.
//
// FP32 path.  Positions are the FP32 tile staging of the open-boundary path
// (offset o and residual r from an FP32 tile centre c, plus the far-field
// expansion layout).  For a target tile I, a source tile J and an image n the
// shift D = c_I - (c_J + nL) is formed in FP64 and split into an FP32 value and
// its FP32 remainder (per axis: seven values of n per tile pair).  FP32 box
// tests with conservative margins sort the images of a tile pair into
//  * far, wholly inside the cut sphere (or the half-box region): every pair is
//    a Newtonian term; summed by expansion about the source tile's centre
//    with packed FP32x2 arithmetic (10 lane operations + 1 MUFU per term), the
//    target shift's rounding undone to first order from the kept terms;
//  * far, straddling the cut sphere: the same, and each term is kept when
//    k_j r^2 < k_j (2.6 L)^2 (branch-free); terms within a thin band of the
//    cut are decided again in FP64 from the FP64 positions with the
//    definition's expression;
//  * explicit: every pair Newtonian, but the tiles are too close for the
//    expansion's first-order shift correction, or a quasi-periodic image
//    straddles the half-box faces: separations to ~1 ulp of their own size
//    (offset residuals and the exact rounding error of the shifted target),
//    packed FP32x2, a branch-free boundary test with FP64 re-decisions in the
//    thin bands;
//  * near (some pair may lie inside h_i + h_j, or I = J): the same
//    separations, scalar, with the full spline of Eq. 4 and per-pair FP64
//    re-decisions in the bands.
// Each warp owns one target tile and a chunk of source tiles (a work item);
// lanes are grouped into image slots so that one warp runs 32 / (T / KF)
// images at once with KF targets per lane and the source loads are shared
// (broadcast) by all slots.  FP32 partial sums are Kahan-folded every 32 (far),
// 16 (explicit) or 8 (near) sources, added into FP64 per source tile, combined across the
// slots in a fixed order and written per work item; the reduction kernel adds
// the items in order: deterministic.
//
// FP64 path.  One thread per target, every source, the image loops of the
// definition in FP64 without contraction (the comparison variant).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pair_terms.cuh"
#include "periodic_class.cuh"
#include "steps_internal.h"

namespace steps {
namespace {

constexpr int kWarps = 4;            // independent work items (warps) per CTA
constexpr int kFoldFar = 32;         // sources per FP32 partial before a Kahan fold (far images)
constexpr int kFoldExact = 8;        // the same on the exact (near) path
constexpr int kFoldExplicit = 16;    // the same on the explicit-separation path
constexpr float kCutBand = 4e-6f;    // relative band around (2.6 L)^2 decided in FP64
constexpr float kFaceBand = 2e-6f;   // band around +-L/2 (in units of L) decided in FP64
constexpr float kAlpha2 = 0.03125f * 0.03125f;  // expansion needs gap >= alpha (distance + extents)
constexpr int kListCap = 344;        // >= 343 candidate images
constexpr uint16_t kAllIn = 0x200;   // list flag: every pair of the image is a term

// Per-warp shared memory.
template <int T, int KF>
struct WarpSmem {
    float4 sf[4 * T];          // tile J in the far-field expansion layout
    float4 sk[T];              // per source: (-k c2, -k c2, band k c2, band k c2), c2 = (2.6 L)^2
    double acc[3 * KF][32];    // FP64 sums of this lane's targets, [component * KF + target][lane]
    float tx[T], ty[T], tz[T]; // tile I: target offsets
    float dh[24], dl[24];      // [axis * 7 + n + 3]: FP32 value and remainder of c_I - (c_J + nL)
    uint16_t lf[kListCap], lc[kListCap], le[kListCap], lx[kListCap];  // far inside / straddling, near, explicit
};

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

// What the per-term FP64 decisions need (sorted FP64 positions and indices).
struct DecideCtx {
    const double *x, *y, *z;
    int64_t n;
    double L;
    int images;
    int nx, ny, nz;  // the image
    int64_t gi0;     // global index of this lane's first target
    int64_t gj0;     // global index of the source tile's first particle
};

// The terms of one far image (source tile J shifted by nL) for this lane's KF
// targets, every pair Newtonian.  With s = fl(o_i + D) the target relative to
// the shifted source tile's centre, n = -s and k_j = m_j^(-2/3) rounded to FP32,
//     k_j |o_j - s|^2 = k_j |n|^2 + k_j |o_j|^2 + (2 k_j o_j) . n
// (a four-step FMA chain on the staged coefficients), and
// w^3 = (k_j |o_j - s|^2)^(-3/2) = m_j / |x_j + nL - x_i|^3; the image adds
// sum_j w^3 (o_j - s) = sum_j w^3 o_j + n sum_j w^3.
// The rounding of the target shift, l = (o_i + D) - s, is the same for every
// source of the tile; to first order it changes each term by
// w^3 (3 n (n.l) / R^2 - l) (R = |s|, the tile small against R), so the image
// adds (3 n (n.l) / R^2 - l) sum_j w^3 over the terms it keeps.
// CUT: the image straddles the cut sphere; a term counts when
// k_j r^2 < k_j (2.6 L)^2.  Terms within a relative band of 4e-6 of the cut
// are left out of the branch-free loop, flagged, and after the fold decided in
// FP64 from the FP64 positions with the definition's expression (a warp vote:
// the whole warp calls this with the same CUT).
template <int T, int NPAIR, bool CUT>
__device__ __forceinline__ void far_image(const WarpSmem<T, 2 * NPAIR> &W, const float (&D)[6], const int ti0,
                                          const bool act, const DecideCtx &dc, float2 (&hx)[NPAIR],
                                          float2 (&hy)[NPAIR], float2 (&hz)[NPAIR], float2 (&cx)[NPAIR],
                                          float2 (&cy)[NPAIR], float2 (&cz)[NPAIR]) {
    const float2 neg1 = make_float2(-1.f, -1.f);
    float2 nx[NPAIR], ny[NPAIR], nz[NPAIR], ss[NPAIR], pw[NPAIR];  // pw: sum of w^3 over the image
    {
        const float2 ndx = make_float2(-D[0], -D[0]), ndy = make_float2(-D[1], -D[1]),
                     ndz = make_float2(-D[2], -D[2]);
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const float2 xi = *reinterpret_cast<const float2 *>(&W.tx[ti0 + 2 * q]);
            const float2 yi = *reinterpret_cast<const float2 *>(&W.ty[ti0 + 2 * q]);
            const float2 zi = *reinterpret_cast<const float2 *>(&W.tz[ti0 + 2 * q]);
            nx[q] = __ffma2_rn(xi, neg1, ndx);
            ny[q] = __ffma2_rn(yi, neg1, ndy);
            nz[q] = __ffma2_rn(zi, neg1, ndz);
            float2 R2 = __fmul2_rn(nx[q], nx[q]);
            R2 = __ffma2_rn(ny[q], ny[q], R2);
            ss[q] = __ffma2_rn(nz[q], nz[q], R2);
            pw[q] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll 1
    for (int j0 = 0; j0 < T; j0 += kFoldFar) {
        float2 px[NPAIR], py[NPAIR], pz[NPAIR], p0[NPAIR];  // sums of w^3 o_j and of w^3
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) px[q] = py[q] = pz[q] = p0[q] = make_float2(0.f, 0.f);
        bool amb = false;  // some term of this lane lies in the band around the cut
#pragma unroll 8
        for (int j = j0; j < j0 + kFoldFar; ++j) {
            const float4 A = W.sf[4 * j], B = W.sf[4 * j + 1], C = W.sf[4 * j + 2], E = W.sf[4 * j + 3];
            const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
            const float2 zj = make_float2(B.x, B.y), kj = make_float2(B.z, B.w);
            const float2 axj = make_float2(C.x, C.y), ayj = make_float2(C.z, C.w);
            const float2 azj = make_float2(E.x, E.y), bj = make_float2(E.z, E.w);
            float4 K = make_float4(0.f, 0.f, 0.f, 0.f);
            if (CUT) K = W.sk[j];
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                float2 t = __ffma2_rn(kj, ss[q], bj);
                t = __ffma2_rn(axj, nx[q], t);
                t = __ffma2_rn(ayj, ny[q], t);
                t = __ffma2_rn(azj, nz[q], t);
                float2 w = make_float2(rsqrt_approx(t.x), rsqrt_approx(t.y));
                if (CUT) {
                    const float2 dt = __fadd2_rn(t, make_float2(K.x, K.y));  // k_j (r^2 - (2.6 L)^2)
                    amb = amb | (fabsf(dt.x) < K.z) | (fabsf(dt.y) < K.z);
                    w.x = dt.x <= -K.z ? w.x : 0.f;
                    w.y = dt.y <= -K.z ? w.y : 0.f;
                }
                const float2 sc = __fmul2_rn(__fmul2_rn(w, w), w);
                px[q] = __ffma2_rn(sc, xj, px[q]);
                py[q] = __ffma2_rn(sc, yj, py[q]);
                pz[q] = __ffma2_rn(sc, zj, pz[q]);
                p0[q] = __fadd2_rn(p0[q], sc);
            }
        }
        if (CUT && __any_sync(0xffffffffu, amb) && amb) {
            // the band terms of this fold, decided in FP64
            for (int j = j0; j < j0 + kFoldFar; ++j) {
                const float4 A = W.sf[4 * j], B = W.sf[4 * j + 1], C = W.sf[4 * j + 2], E = W.sf[4 * j + 3];
                const float4 K = W.sk[j];
                const int64_t gj = dc.gj0 + j;
#pragma unroll
                for (int q = 0; q < NPAIR; ++q) {
                    float2 t = __ffma2_rn(make_float2(B.z, B.w), ss[q], make_float2(E.z, E.w));
                    t = __ffma2_rn(make_float2(C.x, C.y), nx[q], t);
                    t = __ffma2_rn(make_float2(C.z, C.w), ny[q], t);
                    t = __ffma2_rn(make_float2(E.x, E.y), nz[q], t);
                    const float2 dt = __fadd2_rn(t, make_float2(K.x, K.y));
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int64_t gi = dc.gi0 + 2 * q + e;
                        if (fabsf(e ? dt.y : dt.x) < K.z && gi < dc.n && gj < dc.n &&
                            include_f64(dc.x[gi], dc.y[gi], dc.z[gi], dc.x[gj], dc.y[gj], dc.z[gj], dc.nx, dc.ny,
                                        dc.nz, dc.L, 0)) {
                            const float w = rsqrt_approx(e ? t.y : t.x);
                            const float sc = w * w * w;
                            if (e) {
                                px[q].y = fmaf(sc, A.x, px[q].y);
                                py[q].y = fmaf(sc, A.z, py[q].y);
                                pz[q].y = fmaf(sc, B.x, pz[q].y);
                                p0[q].y += sc;
                            } else {
                                px[q].x = fmaf(sc, A.x, px[q].x);
                                py[q].x = fmaf(sc, A.z, py[q].x);
                                pz[q].x = fmaf(sc, B.x, pz[q].x);
                                p0[q].x += sc;
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            // sum of w^3 (o_j - s) = px + n p0
            const float2 qx = __ffma2_rn(nx[q], p0[q], px[q]);
            const float2 qy = __ffma2_rn(ny[q], p0[q], py[q]);
            const float2 qz = __ffma2_rn(nz[q], p0[q], pz[q]);
            if (act) {
                kahan2(hx[q], cx[q], qx);
                kahan2(hy[q], cy[q], qy);
                kahan2(hz[q], cz[q], qz);
            }
            pw[q] = __fadd2_rn(pw[q], p0[q]);
        }
    }
    // first-order correction of the target shift's rounding
    const float2 dhx = make_float2(D[0], D[0]), dhy = make_float2(D[1], D[1]), dhz = make_float2(D[2], D[2]);
    const float2 dlx = make_float2(D[3], D[3]), dly = make_float2(D[4], D[4]), dlz = make_float2(D[5], D[5]);
#pragma unroll
    for (int q = 0; q < NPAIR; ++q) {
        const float2 xi = *reinterpret_cast<const float2 *>(&W.tx[ti0 + 2 * q]);
        const float2 yi = *reinterpret_cast<const float2 *>(&W.ty[ti0 + 2 * q]);
        const float2 zi = *reinterpret_cast<const float2 *>(&W.tz[ti0 + 2 * q]);
        // l: rounding error of s (Fast2Sum) plus the remainder of D
        const float2 lx = __fadd2_rn(__fadd2_rn(xi, __fadd2_rn(nx[q], dhx)), dlx);
        const float2 ly = __fadd2_rn(__fadd2_rn(yi, __fadd2_rn(ny[q], dhy)), dly);
        const float2 lz = __fadd2_rn(__fadd2_rn(zi, __fadd2_rn(nz[q], dhz)), dlz);
        float2 proj = __fmul2_rn(nx[q], lx);
        proj = __ffma2_rn(ny[q], ly, proj);
        proj = __ffma2_rn(nz[q], lz, proj);
        const float2 ri = make_float2(rsqrt_approx(ss[q].x), rsqrt_approx(ss[q].y));
        const float2 c3 = __fmul2_rn(__fmul2_rn(make_float2(3.f, 3.f), proj), __fmul2_rn(ri, ri));
        const float2 qx = __fmul2_rn(__ffma2_rn(c3, nx[q], __fmul2_rn(lx, neg1)), pw[q]);
        const float2 qy = __fmul2_rn(__ffma2_rn(c3, ny[q], __fmul2_rn(ly, neg1)), pw[q]);
        const float2 qz = __fmul2_rn(__ffma2_rn(c3, nz[q], __fmul2_rn(lz, neg1)), pw[q]);
        if (act) {
            kahan2(hx[q], cx[q], qx);
            kahan2(hy[q], cy[q], qy);
            kahan2(hz[q], cz[q], qz);
        }
    }
}

// The terms of one near image for this lane's KF targets with exact
// separations: for target t, x_j + nL - x_i = (o_j + s'_t) + (r_j + r'_t) with
// -s'_t = fl(o_i + D) and -r'_t = r_i + remainder(D) + err(fl(o_i + D)), so the
// separation carries ~1 ulp of its own size; Eq. 4's spline inside h_i + h_j;
// self pairs and the self's images add nothing.  Sources are read from the
// global staging (near images are few).  DECIDE: some pairs may fall outside
// the cut sphere (or the half-box region), so every term is tested, and
// re-decided in FP64 within the thin bands.
template <int T, int KF, bool DECIDE>
__device__ __forceinline__ void exact_image(const float4 *__restrict__ S, const float4 *__restrict__ R,
                                            const float4 *__restrict__ rdup, const float (&D)[6],
                                            const WarpSmem<T, KF> &W, const int ti0, const bool self_tile,
                                            const bool act, const DecideCtx &dc, const float cut2, const float halfL,
                                            const float L, float2 (&hx)[KF / 2], float2 (&hy)[KF / 2],
                                            float2 (&hz)[KF / 2], float2 (&cx)[KF / 2], float2 (&cy)[KF / 2],
                                            float2 (&cz)[KF / 2]) {
    float nxs[KF], nys[KF], nzs[KF], nrx[KF], nry[KF], nrz[KF], hI[KF];
#pragma unroll
    for (int t = 0; t < KF; ++t) {
        const int64_t gi = dc.gi0 + t;
        const float4 r0 = rdup[2 * gi], r1 = rdup[2 * gi + 1];
        const float ox = W.tx[ti0 + t], oy = W.ty[ti0 + t], oz = W.tz[ti0 + t];
        float e;
        nxs[t] = -two_sum(ox, D[0], e);
        nrx[t] = -((r0.x + D[3]) + e);
        nys[t] = -two_sum(oy, D[1], e);
        nry[t] = -((r0.z + D[4]) + e);
        nzs[t] = -two_sum(oz, D[2], e);
        nrz[t] = -((r1.x + D[5]) + e);
        hI[t] = r1.z;
    }
#pragma unroll 1
    for (int f0 = 0; f0 < T; f0 += kFoldExact) {
        float px[KF], py[KF], pz[KF];
#pragma unroll
        for (int t = 0; t < KF; ++t) px[t] = py[t] = pz[t] = 0.f;
#pragma unroll 2
        for (int j = f0; j < f0 + kFoldExact; ++j) {
            const float4 A = S[2 * j], B = S[2 * j + 1];
            const float4 RA = R[2 * j], RB = R[2 * j + 1];
            if (B.z == 0.f) continue;  // padding source (zero mass)
#pragma unroll
            for (int t = 0; t < KF; ++t) {
                // d = x_j + nL - x_i
                const float dx = (A.x + nxs[t]) + (RA.x + nrx[t]);
                const float dy = (A.z + nys[t]) + (RA.z + nry[t]);
                const float dz = (B.x + nzs[t]) + (RB.x + nrz[t]);
                const float r2 = dx * dx + dy * dy + dz * dz;
                bool in = r2 > 0.f && !(self_tile && j == ti0 + t);  // no self pair, no self images
                if (DECIDE && in) {
                    bool ambiguous;
                    if (dc.images == 1) {
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
                        const int64_t gi = dc.gi0 + t, gj = dc.gj0 + j;
                        in = gi < dc.n && gj < dc.n &&
                             include_f64(dc.x[gi], dc.y[gi], dc.z[gi], dc.x[gj], dc.y[gj], dc.z[gj], dc.nx, dc.ny,
                                         dc.nz, dc.L, dc.images);
                    }
                }
                if (!in) continue;
                const float H = hI[t] + RB.z;
                const float ri = rsqrt_approx(r2);
                const float g = (r2 >= H * H) ? ri * ri * ri : spline_over_r_f32(r2 * ri, H);
                const float sc = B.z * g;
                px[t] = fmaf(sc, dx, px[t]);
                py[t] = fmaf(sc, dy, py[t]);
                pz[t] = fmaf(sc, dz, pz[t]);
            }
        }
        if (act) {
#pragma unroll
            for (int q = 0; q < KF / 2; ++q) {
                kahan2(hx[q], cx[q], make_float2(px[2 * q], px[2 * q + 1]));
                kahan2(hy[q], cy[q], make_float2(py[2 * q], py[2 * q + 1]));
                kahan2(hz[q], cz[q], make_float2(pz[2 * q], pz[2 * q + 1]));
            }
        }
    }
}

// The terms of one image whose pairs are all Newtonian (no pair within
// h_i + h_j, no self pair) but which the expansion form does not take: tiles
// too close for its first-order shift correction, or a quasi-periodic image
// straddling the half-box faces.  Separations as on the exact path,
// x_j + nL - x_i = (o_j + s'_t) + (r_j + r'_t), packed two targets at a time
// (FP32x2).  DECIDE: a term counts when r^2 < (2.6 L)^2 (cut sum) or when
// max_c |d_c| < L/2 (QUASI); terms within the thin bands are left out of the
// branch-free loop, flagged, and after the fold decided in FP64 (a warp vote:
// the whole warp calls this with the same DECIDE).  Sources are read from the
// global staging.
template <int T, int KF, bool DECIDE, bool QUASI>
__device__ __forceinline__ void explicit_image(const float4 *__restrict__ S, const float4 *__restrict__ R,
                                               const float4 *__restrict__ rdup, const float (&D)[6],
                                               const WarpSmem<T, KF> &W, const int ti0, const bool act,
                                               const DecideCtx &dc, const float cut2, const float halfL,
                                               const float L, float2 (&hx)[KF / 2], float2 (&hy)[KF / 2],
                                               float2 (&hz)[KF / 2], float2 (&cx)[KF / 2], float2 (&cy)[KF / 2],
                                               float2 (&cz)[KF / 2]) {
    constexpr int NPAIR = KF / 2;
    float2 nxs[NPAIR], nys[NPAIR], nzs[NPAIR], nrx[NPAIR], nry[NPAIR], nrz[NPAIR];
#pragma unroll
    for (int q = 0; q < NPAIR; ++q) {
        float v[2][6];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int t = 2 * q + e;
            const int64_t gi = dc.gi0 + t;
            const float4 r0 = rdup[2 * gi], r1 = rdup[2 * gi + 1];
            float err;
            v[e][0] = -two_sum(W.tx[ti0 + t], D[0], err);
            v[e][3] = -((r0.x + D[3]) + err);
            v[e][1] = -two_sum(W.ty[ti0 + t], D[1], err);
            v[e][4] = -((r0.z + D[4]) + err);
            v[e][2] = -two_sum(W.tz[ti0 + t], D[2], err);
            v[e][5] = -((r1.x + D[5]) + err);
        }
        nxs[q] = make_float2(v[0][0], v[1][0]);
        nys[q] = make_float2(v[0][1], v[1][1]);
        nzs[q] = make_float2(v[0][2], v[1][2]);
        nrx[q] = make_float2(v[0][3], v[1][3]);
        nry[q] = make_float2(v[0][4], v[1][4]);
        nrz[q] = make_float2(v[0][5], v[1][5]);
    }
    const float band = QUASI ? kFaceBand * L : kCutBand * cut2;
    const float2 lim = QUASI ? make_float2(-halfL, -halfL) : make_float2(-cut2, -cut2);
#pragma unroll 1
    for (int f0 = 0; f0 < T; f0 += kFoldExplicit) {
        float2 px[NPAIR], py[NPAIR], pz[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
        bool amb = false;
#pragma unroll 2
        for (int j = f0; j < f0 + kFoldExplicit; ++j) {
            const float4 A = S[2 * j], B = S[2 * j + 1];
            const float4 RA = R[2 * j], RB = R[2 * j + 1];
            const float2 mj = make_float2(B.z, B.w);
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), nxs[q]),
                                             __fadd2_rn(make_float2(RA.x, RA.y), nrx[q]));
                const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), nys[q]),
                                             __fadd2_rn(make_float2(RA.z, RA.w), nry[q]));
                const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), nzs[q]),
                                             __fadd2_rn(make_float2(RB.x, RB.y), nrz[q]));
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                if (DECIDE) {
                    float2 u;  // signed distance from the boundary: r^2 - (2.6 L)^2, or max_c |d_c| - L/2
                    if (QUASI)
                        u = __fadd2_rn(make_float2(fmaxf(fabsf(dx.x), fmaxf(fabsf(dy.x), fabsf(dz.x))),
                                                   fmaxf(fabsf(dx.y), fmaxf(fabsf(dy.y), fabsf(dz.y)))),
                                       lim);
                    else
                        u = __fadd2_rn(r2, lim);
                    amb = amb | (fabsf(u.x) < band) | (fabsf(u.y) < band);
                    ri.x = u.x <= -band ? ri.x : 0.f;
                    ri.y = u.y <= -band ? ri.y : 0.f;
                }
                const float2 sc = __fmul2_rn(__fmul2_rn(mj, ri), __fmul2_rn(ri, ri));
                px[q] = __ffma2_rn(sc, dx, px[q]);
                py[q] = __ffma2_rn(sc, dy, py[q]);
                pz[q] = __ffma2_rn(sc, dz, pz[q]);
            }
        }
        if (DECIDE && __any_sync(0xffffffffu, amb) && amb) {
            // the band terms of this fold, decided in FP64
            for (int j = f0; j < f0 + kFoldExplicit; ++j) {
                const float4 A = S[2 * j], B = S[2 * j + 1];
                const float4 RA = R[2 * j], RB = R[2 * j + 1];
                const int64_t gj = dc.gj0 + j;
#pragma unroll
                for (int q = 0; q < NPAIR; ++q) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float dx = (e ? (A.y + nxs[q].y) : (A.x + nxs[q].x)) +
                                         (e ? (RA.y + nrx[q].y) : (RA.x + nrx[q].x));
                        const float dy = (e ? (A.w + nys[q].y) : (A.z + nys[q].x)) +
                                         (e ? (RA.w + nry[q].y) : (RA.z + nry[q].x));
                        const float dz = (e ? (B.y + nzs[q].y) : (B.x + nzs[q].x)) +
                                         (e ? (RB.y + nrz[q].y) : (RB.x + nrz[q].x));
                        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                        const float u = QUASI ? fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) + lim.x : r2 + lim.x;
                        const int64_t gi = dc.gi0 + 2 * q + e;
                        if (fabsf(u) < band && gi < dc.n && gj < dc.n &&
                            include_f64(dc.x[gi], dc.y[gi], dc.z[gi], dc.x[gj], dc.y[gj], dc.z[gj], dc.nx, dc.ny,
                                        dc.nz, dc.L, dc.images)) {
                            const float ri = rsqrt_approx(r2);
                            const float sc = B.z * ri * (ri * ri);
                            if (e) {
                                px[q].y = fmaf(sc, dx, px[q].y);
                                py[q].y = fmaf(sc, dy, py[q].y);
                                pz[q].y = fmaf(sc, dz, pz[q].y);
                            } else {
                                px[q].x = fmaf(sc, dx, px[q].x);
                                py[q].x = fmaf(sc, dy, py[q].x);
                                pz[q].x = fmaf(sc, dz, pz[q].x);
                            }
                        }
                    }
                }
            }
        }
        if (act) {
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                kahan2(hx[q], cx[q], px[q]);
                kahan2(hy[q], cy[q], py[q]);
                kahan2(hz[q], cz[q], pz[q]);
            }
        }
    }
}

// The shift of image k for this tile pair: FP32 values and remainders.
__device__ __forceinline__ void image_shift(const float *dh, const float *dl, int nx, int ny, int nz,
                                            float (&D)[6]) {
    D[0] = dh[nx + 3];
    D[1] = dh[10 + ny];
    D[2] = dh[17 + nz];
    D[3] = dl[nx + 3];
    D[4] = dl[10 + ny];
    D[5] = dl[17 + nz];
}

// One work item per warp: target tile I (T targets, KF per lane in slots of
// T / KF lanes) against source tiles [J0, J1) of its chunk, every image.
template <int T, int KF>
__global__ void __launch_bounds__(32 * kWarps, 3) periodic_f32_kernel(const PeriodicArgs a) {
    constexpr int LPI = T / KF;    // lanes per image slot
    constexpr int IPW = 32 / LPI;  // images per warp step
    constexpr int NPAIR = KF / 2;
    static_assert(LPI * IPW == 32 && KF % 2 == 0, "lanes must split into whole image slots");
    extern __shared__ float4 periodic_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<T, KF> &W = reinterpret_cast<WarpSmem<T, KF> *>(periodic_smem)[warp];
    const int64_t item = (int64_t)blockIdx.x * kWarps + warp;
    int64_t I, J0, J1;
    if (a.residual && a.soff[a.ntile] <= a.cap_items) {
        // one source tile that shares a softened image with the target tile
        if (item >= a.soff[a.ntile]) return;  // whole warp; warps of a CTA never synchronise
        int64_t lo = 0, hi = a.ntile;         // soff[lo] <= item < soff[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (a.soff[mid] <= item) lo = mid; else hi = mid;
        }
        I = lo;
        J0 = a.slist[item];
        J1 = J0 + 1;
    } else {
        if (item >= a.ntile * a.nchunk) return;
        I = item / a.nchunk;
        const int64_t ch = item % a.nchunk;
        J0 = ch * a.ntile / a.nchunk;
        J1 = (ch + 1) * a.ntile / a.nchunk;
    }
    const int g = lane / LPI;           // image slot
    const int ti0 = (lane % LPI) * KF;  // this lane's first target within the tile
    const float L = (float)a.Ls;  // staging units
    const double cutd = 2.6 * a.Ls;
    const float cut2 = (float)(cutd * cutd);
    const float halfL = 0.5f * L;
    const int nimg = a.images == 1 ? 27 : 343;
    const float up = 1.0f + 0x1p-18f, dn = 1.0f - 0x1p-18f;
    const float mg = 1e-5f * L;  // margin of the FP32 box tests (their rounding is ~1e-7 L)

    const int64_t gi0 = I * T + ti0;
    for (int k = lane; k < T; k += 32) {
        const float4 p = a.jdup[2 * (I * T + k)], pz = a.jdup[2 * (I * T + k) + 1];
        W.tx[k] = p.x;
        W.ty[k] = p.z;
        W.tz[k] = pz.x;
    }
#pragma unroll
    for (int t = 0; t < 3 * KF; ++t) W.acc[t][lane] = 0.0;
    const float4 ci = a.tbox_c[I], ei = a.tbox_e[I];
    const float eIn = sqrtf(ei.x * ei.x + ei.y * ei.y + ei.z * ei.z);

    for (int64_t J = J0; J < J1; ++J) {
        __syncwarp();
        if (!a.residual) {
            const float4 *src = a.fdup + 4 * J * T;
            for (int k = lane; k < 4 * T; k += 32) W.sf[k] = src[k];
        }
        const float4 cj = a.tbox_c[J], ej = a.tbox_e[J];
        if (lane < 21) {
            // c_I - (c_J + nL) in FP64 per axis and n in [-3, 3], split into FP32 value + remainder
            const int ax = lane / 7, nn = lane % 7 - 3;
            const float c0 = ax == 0 ? ci.x : (ax == 1 ? ci.y : ci.z);
            const float c1 = ax == 0 ? cj.x : (ax == 1 ? cj.y : cj.z);
            const double d = (double)c0 - ((double)c1 + nn * a.Ls);
            const float hi = (float)d;
            W.dh[lane] = hi;
            W.dl[lane] = (float)(d - (double)hi);
        }
        __syncwarp();
        if (!a.residual) {
            for (int j = lane; j < T; j += 32) {
                const float kc = W.sf[4 * j + 1].z * cut2;
                W.sk[j] = make_float4(-kc, -kc, kCutBand * kc, kCutBand * kc);
            }
        }
        // sort the candidate images of this tile pair into the four lists
        const float wx = __fadd_rn(ei.x, ej.x) * up + mg, wy = __fadd_rn(ei.y, ej.y) * up + mg,
                    wz = __fadd_rn(ei.z, ej.z) * up + mg;
        const float hs = __fadd_rn(ci.w, cj.w) * up;
        const float ext = (eIn + sqrtf(ej.x * ej.x + ej.y * ej.y + ej.z * ej.z)) * up;
        const bool self_tile = (I == J);
        int nF = 0, nC = 0, nE = 0, nX = 0;
        for (int k0 = 0; k0 < nimg; k0 += 32) {
            const int k = k0 + lane;
            int cls = 0;  // 0 none, 1 far inside, 2 far straddling the cut, 3 near, 4 explicit
            bool allin = false;
            if (k < nimg && a.residual) {
                // only the images the symmetric kernel leaves out: those that may
                // hold a softened pair (the same decision, periodic_class.cuh)
                int nx, ny, nz;
                image_of(k, a.images, nx, ny, nz);
                float gap2;
                const int pc = a.images == 1 ? quasi_image_class(ci, ei, cj, ej, nx, ny, nz, self_tile, &gap2)
                                             : periodic_image_class(ci, ei, cj, ej, nx, ny, nz, self_tile, &gap2);
                if (pc == kPerSoft) cls = 3;
            } else if (k < nimg) {
                int nx, ny, nz;
                image_of(k, a.images, nx, ny, nz);
                const float sx = W.dh[nx + 3], sy = W.dh[10 + ny], sz = W.dh[17 + nz];
                const float ax_ = fabsf(sx), ay_ = fabsf(sy), az_ = fabsf(sz);
                const float gx = fmaxf(0.f, ax_ - wx), gy = fmaxf(0.f, ay_ - wy), gz = fmaxf(0.f, az_ - wz);
                const float fx = ax_ + wx, fy = ay_ + wy, fz = az_ + wz;
                const float gap2 = gx * gx + gy * gy + gz * gz;
                bool cand;
                if (a.images == 1) {
                    cand = ax_ <= halfL + wx && ay_ <= halfL + wy && az_ <= halfL + wz;
                    allin = fx < halfL && fy < halfL && fz < halfL;
                } else {
                    cand = gap2 < cut2 * up;
                    allin = fx * fx + fy * fy + fz * fz < cut2 * dn;
                }
                if (cand) {
                    const float dist2 = sx * sx + sy * sy + sz * sz;
                    const float scale = sqrtf(dist2) + ext;
                    const bool soft = self_tile || gap2 <= hs * hs;
                    const bool expansion = ext * ext <= dist2 * dn && gap2 >= kAlpha2 * scale * scale;
                    if (soft)
                        cls = 3;
                    else if (!expansion || (a.images == 1 && !allin))
                        cls = 4;
                    else
                        cls = allin ? 1 : 2;
                }
            }
            const unsigned lt = (1u << lane) - 1u;
            const unsigned bF = __ballot_sync(0xffffffffu, cls == 1);
            const unsigned bC = __ballot_sync(0xffffffffu, cls == 2);
            const unsigned bE = __ballot_sync(0xffffffffu, cls == 3);
            const unsigned bX = __ballot_sync(0xffffffffu, cls == 4);
            if (cls == 1)
                W.lf[nF + __popc(bF & lt)] = (uint16_t)k;
            else if (cls == 2)
                W.lc[nC + __popc(bC & lt)] = (uint16_t)k;
            else if (cls == 3)
                W.le[nE + __popc(bE & lt)] = (uint16_t)(k | (allin ? kAllIn : 0));
            else if (cls == 4)
                W.lx[nX + __popc(bX & lt)] = (uint16_t)(k | (allin ? kAllIn : 0));
            nF += __popc(bF);
            nC += __popc(bC);
            nE += __popc(bE);
            nX += __popc(bX);
        }
        __syncwarp();

        // compensated FP32 sums over every image of tile J, one FP64 add per tile
        float2 hx[NPAIR], hy[NPAIR], hz[NPAIR], cx[NPAIR], cy[NPAIR], cz[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q)
            hx[q] = hy[q] = hz[q] = cx[q] = cy[q] = cz[q] = make_float2(0.f, 0.f);
        DecideCtx dc{a.x, a.y, a.z, a.n, a.L, a.images, 0, 0, 0, gi0, J * T};  // FP64 positions, FP64 box
        for (int b = 0; b < nF; b += IPW) {
            const bool act = b + g < nF;  // idle slots repeat the step's first image and add nothing
            const int k = W.lf[act ? b + g : b];
            float D[6];
            image_of(k, a.images, dc.nx, dc.ny, dc.nz);
            image_shift(W.dh, W.dl, dc.nx, dc.ny, dc.nz, D);
            far_image<T, NPAIR, false>(W, D, ti0, act, dc, hx, hy, hz, cx, cy, cz);
        }
        for (int b = 0; b < nC; b += IPW) {
            const bool act = b + g < nC;
            const int k = W.lc[act ? b + g : b];
            float D[6];
            image_of(k, a.images, dc.nx, dc.ny, dc.nz);
            image_shift(W.dh, W.dl, dc.nx, dc.ny, dc.nz, D);
            far_image<T, NPAIR, true>(W, D, ti0, act, dc, hx, hy, hz, cx, cy, cz);
        }
        const float4 *S = a.jdup + 2 * J * T, *R = a.rdup + 2 * J * T;
        for (int b = 0; b < nX; b += IPW) {
            const bool act = b + g < nX;
            const int code = W.lx[act ? b + g : b];
            float D[6];
            image_of(code & 0x1ff, a.images, dc.nx, dc.ny, dc.nz);
            image_shift(W.dh, W.dl, dc.nx, dc.ny, dc.nz, D);
            // one choice for the whole warp (the image slots may differ): the
            // deciding loop votes across the warp after each fold
            const bool decide = __any_sync(0xffffffffu, !(code & kAllIn));
            if (!decide)
                explicit_image<T, KF, false, false>(S, R, a.rdup, D, W, ti0, act, dc, cut2, halfL, L, hx, hy, hz, cx,
                                                    cy, cz);
            else if (a.images == 1)
                explicit_image<T, KF, true, true>(S, R, a.rdup, D, W, ti0, act, dc, cut2, halfL, L, hx, hy, hz, cx,
                                                  cy, cz);
            else
                explicit_image<T, KF, true, false>(S, R, a.rdup, D, W, ti0, act, dc, cut2, halfL, L, hx, hy, hz, cx,
                                                   cy, cz);
        }
        for (int b = 0; b < nE; b += IPW) {
            const bool act = b + g < nE;
            const int code = W.le[act ? b + g : b];
            float D[6];
            image_of(code & 0x1ff, a.images, dc.nx, dc.ny, dc.nz);
            image_shift(W.dh, W.dl, dc.nx, dc.ny, dc.nz, D);
            if (code & kAllIn)
                exact_image<T, KF, false>(S, R, a.rdup, D, W, ti0, self_tile, act, dc, cut2, halfL, L, hx,
                                          hy, hz, cx, cy, cz);
            else
                exact_image<T, KF, true>(S, R, a.rdup, D, W, ti0, self_tile, act, dc, cut2, halfL, L, hx,
                                         hy, hz, cx, cy, cz);
        }
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            // value = hi - c, the compensation kept negated
            W.acc[2 * q][lane] += (double)hx[q].x + (double)cx[q].x;
            W.acc[2 * q + 1][lane] += (double)hx[q].y + (double)cx[q].y;
            W.acc[KF + 2 * q][lane] += (double)hy[q].x + (double)cy[q].x;
            W.acc[KF + 2 * q + 1][lane] += (double)hy[q].y + (double)cy[q].y;
            W.acc[2 * KF + 2 * q][lane] += (double)hz[q].x + (double)cz[q].x;
            W.acc[2 * KF + 2 * q + 1][lane] += (double)hz[q].y + (double)cz[q].y;
        }
    }
    // slots hold the same targets: add them in a fixed order (slot 0 first)
    __syncwarp();
    if (g == 0) {
        double *P = a.item_part + (size_t)item * 3 * T;
#pragma unroll
        for (int t = 0; t < KF; ++t) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = W.acc[c * KF + t][lane];
#pragma unroll
                for (int s = 1; s < IPW; ++s) v += W.acc[c * KF + t][lane + s * LPI];
                P[c * T + ti0 + t] = v;
            }
        }
    }
}

// Sum each target's work items in item order, add the symmetric kernel's
// fixed-point sums (acc, or null), and apply G (sorted order).
__global__ void periodic_reduce_kernel(const double *__restrict__ item_part, int64_t n, int T, int64_t ntile,
                                       int64_t nchunk, const int64_t *__restrict__ soff, int64_t cap_items,
                                       const unsigned long long *__restrict__ acc, const double *__restrict__ tinv,
                                       int64_t np, double G, double *__restrict__ ax, double *__restrict__ ay,
                                       double *__restrict__ az, int *nonfinite) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t I = p / T;
    const int li = (int)(p - I * T);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    // the items of target tile I, in item order
    const bool lists = soff && soff[ntile] <= cap_items;
    const int64_t it0 = lists ? soff[I] : I * nchunk, it1 = lists ? soff[I + 1] : (I + 1) * nchunk;
    for (int64_t it = it0; it < it1; ++it) {
        const double *Q = item_part + (size_t)it * 3 * T;
        sx += Q[li];
        sy += Q[T + li];
        sz += Q[2 * T + li];
    }
    if (acc) {
        const double inv = tinv[I];
        sx += (double)(long long)acc[p] * inv;
        sy += (double)(long long)acc[np + p] * inv;
        sz += (double)(long long)acc[2 * np + p] * inv;
    }
    ax[p] = G * sx;
    ay[p] = G * sy;
    az[p] = G * sz;
    if (nonfinite && (!isfinite(sx) || !isfinite(sy) || !isfinite(sz))) *nonfinite = 1;
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

template <int T, int KF>
cudaError_t launch_tile(const PeriodicArgs &a, unsigned blocks, cudaStream_t st) {
    const size_t smem = sizeof(WarpSmem<T, KF>) * kWarps;
    // the shared-memory opt-in is set outside graph capture (the first force
    // evaluation of a context always runs outside one)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone) {
        e = cudaFuncSetAttribute(periodic_f32_kernel<T, KF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    periodic_f32_kernel<T, KF><<<blocks, 32 * kWarps, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Enough work items (one warp each) for several waves of 16 warps per SM, at
// most 64 chunks of source tiles per target tile.
int64_t periodic_chunks(int64_t ntile, int num_sms) {
    const int64_t want = (int64_t)std::max(num_sms, 1) * 16 * 8;
    int64_t c = (want + ntile - 1) / ntile;
    c = std::min<int64_t>(c, 64);
    c = std::min<int64_t>(c, ntile);
    return std::max<int64_t>(c, 1);
}

// Upper bound over every tile count x <= np / T: x * periodic_chunks(x) is at
// most min(64 x, want + x).
size_t periodic_part_elems(int64_t np, int num_sms) {
    const int64_t want = (int64_t)std::max(num_sms, 1) * 16 * 8;
    size_t m = 0;
    for (int T : {64, 128, 192}) {
        const int64_t nt = (np + T - 1) / T;
        m = std::max(m, (size_t)std::min<int64_t>(64 * nt, want + nt) * 3 * T);
    }
    return m;
}

cudaError_t launch_periodic_f32(const Staging &s, const double *x, const double *y, const double *z, double L,
                                int images, double G, double *item_part, const PeriodicSymScratch *ps,
                                int num_sms, double *ax, double *ay, double *az, cudaStream_t st,
                                cudaEvent_t far_begin, cudaEvent_t far_end) {
    // the symmetric kernel takes the Newtonian images on 128-particle tiles with
    // its layout; the per-target kernel everything else
    const bool sym = ps && s.sdup && s.T == periodic_sym_tile();
    if (!sym && !s.fdup) return cudaErrorInvalidValue;
    cudaError_t e;
    if (sym) {
        if (far_begin && (e = cudaEventRecord(far_begin, st)) != cudaSuccess) return e;
        e = launch_periodic_sym(s, x, y, z, L, images, *ps, num_sms, st);
        if (e != cudaSuccess) return e;
        if (far_end && (e = cudaEventRecord(far_end, st)) != cudaSuccess) return e;
    }
    PeriodicArgs a;
    a.jdup = s.jdup;
    a.rdup = s.rdup;
    a.fdup = s.fdup;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.x = x;
    a.y = y;
    a.z = z;
    a.item_part = item_part;
    a.ntile = s.ntile;
    a.nchunk = periodic_chunks(s.ntile, num_sms);
    a.n = s.n;
    a.L = L;
    a.Ls = 1.0;  // the staging is in box units
    a.images = images;
    a.residual = sym ? 1 : 0;
    a.soff = sym ? ps->soff : nullptr;
    a.slist = sym ? ps->slist : nullptr;
    a.cap_items = sym ? ps->cap_items : 0;
    // residual mode: enough warps for the soft partner lists or the chunks
    const int64_t items = sym ? std::max<int64_t>(a.ntile * a.nchunk, ps->cap_items) : a.ntile * a.nchunk;
    const unsigned blocks = (unsigned)((items + kWarps - 1) / kWarps);
    if (!sym && far_begin && (e = cudaEventRecord(far_begin, st)) != cudaSuccess) return e;
    switch (s.T) {
        case 64: e = launch_tile<64, 4>(a, blocks, st); break;
        case 128: e = launch_tile<128, 4>(a, blocks, st); break;
        case 192: e = launch_tile<192, 6>(a, blocks, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (!sym && far_end && (e = cudaEventRecord(far_end, st)) != cudaSuccess) return e;
    // forces in box units scale as 1 / L^2
    const double Gs = G / (L * L);
    periodic_reduce_kernel<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(
        item_part, s.n, s.T, a.ntile, a.nchunk, a.soff, a.cap_items, sym ? ps->acc : nullptr,
        sym ? ps->tinv : nullptr, s.np, Gs, ax, ay, az, ps ? ps->nonfinite : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_periodic_f64(int64_t n, const double *x, const double *y, const double *z, const double *m,
                                const double *h, double G, double L, int images, double *ax, double *ay,
                                double *az, cudaStream_t st) {
    periodic_f64_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, x, y, z, m, h, G, L, images, ax, ay, az);
    return cudaGetLastError();
}

}  // namespace steps

// Symmetric FP32 far field of the pair term (Eq. 8; Eq. 3 with the Newtonian
// branch of Eq. 4) for sm_103a.
//
// The pair term is antisymmetric: particle i feels m_j (x_j - x_i)/r^3 and
// particle j feels m_i (x_i - x_j)/r^3 from the same separation and the same
// 1/r^3 (Newton's third law).  This kernel evaluates every far pair of tiles
// (I < J) once and adds the pair's force to both particles: per pair the
// separation (3), r^2 (3), MUFU rsqrt, 1/r^3 (2), and two scaled
// accumulations (1 + 3 each) -- 16 FP32 lane operations and one MUFU for two
// interactions, against 20 and two for evaluating each order separately
// (plus 3 additions per pair for the exact separation and 3 per source and
// step that bound the rounding of the source-side sums).
//
// Work layout (GB300-first):
//  * Tiles of T = 256 Morton-ordered particles with FP32 offsets from an FP32
//    tile centre; the centres are rounded to a grid that makes every
//    difference of two centres exact in FP32, so a tile pair shares one exact
//    shift dc = c_I - c_J.
//  * A unit is (target block b of W tiles, source tile J) with J after the
//    block's first tile; warp w takes target tile b W + w only when it
//    precedes J, so each pair of distinct tiles is one unit of one warp.  A
//    persistent grid takes fixed chunks of consecutive units from a global
//    counter; source tiles stream into a shared-memory ring with TMA bulk
//    copies (cp.async.bulk completing on mbarriers), each stage refilled by
//    the last warp done with it; warp w owns target tile b W + w.
//  * Inside a warp, lane l holds 8 targets (particles l + 32 t) as 4 packed
//    pairs (FFMA2).  The source tile is processed in 4 rounds of 32 steps; at
//    step s lane l takes the 2 sources of group (l + s) mod 32, so no two
//    lanes touch the same source, and the sources' running sums travel with
//    the group from lane to lane by one shuffle per step.  After a round each
//    lane holds the complete contribution of the warp's 256 targets to its own
//    group's sources.
//  * The separation is (o_j - o_i) - (c_I - c_J): offsets first (both at tile
//    scale), then the exact centre difference, so every rounding is relative
//    to the pair's own separation and varies from pair to pair.
//  * Target sums: FP32 partials over 32 sources folded into a per-target
//    compensated (Kahan) pair kept in shared memory.  Source sums: a fresh
//    partial of the step's 8 targets added once per step to the group's
//    running sum (32 additions per round).
//  * Both sides are accumulated in 64-bit fixed point with red.global.add:
//    every partial is scaled by a per-tile power of two, chosen from a bound
//    on the tile's far-field sum computed by the classification pass, and
//    rounded to an integer.  Integer addition is associative, so the result
//    does not depend on the order of the atomic adds: evaluations are
//    bit-for-bit reproducible.
//  * Every mbarrier wait is bounded (%globaltimer); a wait that runs out
//    records STEPS_ETIMEOUT, the warp waits (bounded) for the copies issued so
//    far and exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "async_copy.cuh"
#include "pair_terms.cuh"
#include "steps_internal.h"
#include "systems.cuh"

namespace steps {

namespace {

// KI targets per lane (8: 256-particle tiles, 4: 128-particle tiles) as KI/2
// packed pairs; kKJ sources per lane and step; a source tile is taken in
// 32 KI / (32 kKJ) rounds of 32 steps.
constexpr int kKJ = 2;                  // sources per lane and step
constexpr int kFold = 16;               // steps (32 sources) per compensated fold

struct SymArgs {
    const float4 *__restrict__ sdup;      // [np / 32][2][32] (ox, ox, oy, oy), (oz, oz, m, m)
    const float4 *__restrict__ tbox_c;    // [ntile] (cx, cy, cz, hmax)
    const float4 *__restrict__ tbox_e;    // [ntile] (ex, ey, ez, tile mass)
    const uint32_t *__restrict__ nearbits;
    const uint8_t *__restrict__ submask;  // sub-block near masks, or null (whole tile pairs)
    const float *__restrict__ tscale;     // [ntile] fixed-point scale
    unsigned long long *__restrict__ acc; // [3][np]
    int *nonfinite;
    int *err;
    const SimDesc *__restrict__ sims;
    int nsims;
    int64_t np;
    int64_t units;
    int64_t chunk;              // units per chunk
    unsigned long long *next;   // chunk counter, zeroed before the launch
    long long wait_ns;
};

// Units of one system in row-major order: row b holds (b, J) for
// J = b W + 1 .. ntile - 1.  In unit (b, J) warp w takes target tile b W + w
// only when that tile precedes J, so every pair of distinct tiles belongs to
// exactly one unit and one warp (the first W - 1 units of a row reach into the
// block itself).
template <int W>
struct UnitCursor {
    int sidx;
    SimDesc d;
    int64_t b, J;

    __device__ __forceinline__ int64_t row_off(int64_t bb) const {
        return bb * (d.ntile - 1) - (int64_t)W * bb * (bb - 1) / 2;
    }
    __device__ __forceinline__ void locate(const SimDesc *__restrict__ sims, int nsims, int64_t u) {
        sidx = sim_of_unit(sims, nsims, u);
        d = sims[sidx];
        const int64_t v = u - d.unit_off;
        int64_t lo = 0, hi = d.ntile / W;  // row_off(lo) <= v < row_off(hi)
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (row_off(mid) <= v) lo = mid; else hi = mid;
        }
        b = lo;
        J = b * W + 1 + (v - row_off(b));
    }
    __device__ __forceinline__ void next(const SimDesc *__restrict__ sims, int nsims) {
        if (++J < d.ntile) return;
        ++b;
        J = b * W + 1;
        while (J >= d.ntile) {  // past the last row: the next system with units
            if (++sidx >= nsims) return;
            d = sims[sidx];
            b = 0;
            J = 1;
        }
    }
};

// Add v (FP32) times the power of two sc to a fixed-point sum.
__device__ __forceinline__ void red_fixed(unsigned long long *addr, float v, float sc, int *nonfinite) {
    if (!isfinite(v)) {
        if (nonfinite) *nonfinite = 1;
        return;
    }
    atomicAdd(addr, (unsigned long long)__float2ll_rn(v * sc));
}

// One round of a unit (32 steps: the sources (r, k, g) for all groups g)
// for the warp's targets in packed pairs [Q0, Q1): the two halves of a
// 256-particle target tile are q = 0, 1 and q = 2, 3, so a round may skip
// the half whose sub-block against this round's sources is near.
template <int KI, int UNR, int Q0, int Q1>
__device__ __forceinline__ void sym_round(const float4 *__restrict__ S, int r, const float2 ndx, const float2 ndy,
                                          const float2 ndz, const float2 (&nox)[KI / 2], const float2 (&noy)[KI / 2],
                                          const float2 (&noz)[KI / 2], float2 (&px)[KI / 2], float2 (&py)[KI / 2],
                                          float2 (&pz)[KI / 2], const float2 (&mi)[KI / 2],
                                          float4 *__restrict__ myk, int lane, int from, int64_t jbase, float scJ,
                                          unsigned long long *__restrict__ acc, int64_t np, int *nonfinite) {
    constexpr int kNP = KI / 2;
    // running sums of the sources of group (lane + step) mod 32: with 4 targets
    // per lane the two packed halves are added before the rotation (6
    // shuffles per step instead of 12; measured 2% faster there, 1% slower
    // with 8 targets per lane)
    constexpr bool kOne = KI == 4;
    float2 Sx[kKJ], Sy[kKJ], Sz[kKJ];
#pragma unroll
    for (int k = 0; k < kKJ; ++k) Sx[k] = Sy[k] = Sz[k] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int h = 0; h < 32; h += kFold) {
#pragma unroll UNR
        for (int st = h; st < h + kFold; ++st) {
            const int g = (lane + st) & 31;
#pragma unroll
            for (int k = 0; k < kKJ; ++k) {
                const float4 *src = S + (r * kKJ + k) * 64 + g;
                const float4 A = src[0], B = src[32];
                const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
                const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
                // this step's targets on the two sources form a fresh partial that is
                // added to the group's running sum once: the sum grows by 32 additions
                // per round instead of 32 per packed pair
                float2 tx, ty, tz;
#pragma unroll
                for (int q = Q0; q < Q1; ++q) {
                    const float2 dx = __fadd2_rn(__fadd2_rn(xj, nox[q]), ndx);  // x_j - x_i
                    const float2 dy = __fadd2_rn(__fadd2_rn(yj, noy[q]), ndy);
                    const float2 dz = __fadd2_rn(__fadd2_rn(zj, noz[q]), ndz);
                    float2 r2 = __fmul2_rn(dx, dx);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dz, dz, r2);
                    const float2 w = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                    const float2 u = __fmul2_rn(__fmul2_rn(w, w), w);  // 1/r^3
                    const float2 si = __fmul2_rn(u, mj);
                    px[q] = __ffma2_rn(si, dx, px[q]);
                    py[q] = __ffma2_rn(si, dy, py[q]);
                    pz[q] = __ffma2_rn(si, dz, pz[q]);
                    const float2 sj = __fmul2_rn(u, mi[q]);
                    if (q == Q0) {
                        tx = __fmul2_rn(sj, dx);
                        ty = __fmul2_rn(sj, dy);
                        tz = __fmul2_rn(sj, dz);
                    } else {
                        tx = __ffma2_rn(sj, dx, tx);
                        ty = __ffma2_rn(sj, dy, ty);
                        tz = __ffma2_rn(sj, dz, tz);
                    }
                }
                if constexpr (kOne) {
                    Sx[k].x = __fadd_rn(Sx[k].x, __fadd_rn(tx.x, tx.y));
                    Sy[k].x = __fadd_rn(Sy[k].x, __fadd_rn(ty.x, ty.y));
                    Sz[k].x = __fadd_rn(Sz[k].x, __fadd_rn(tz.x, tz.y));
                } else {
                    Sx[k] = __fadd2_rn(Sx[k], tx);
                    Sy[k] = __fadd2_rn(Sy[k], ty);
                    Sz[k] = __fadd2_rn(Sz[k], tz);
                }
            }
            // pass the group's sums on: lane l takes over group (l + st + 1) mod 32
#pragma unroll
            for (int k = 0; k < kKJ; ++k) {
                Sx[k].x = __shfl_sync(0xffffffffu, Sx[k].x, from);
                Sy[k].x = __shfl_sync(0xffffffffu, Sy[k].x, from);
                Sz[k].x = __shfl_sync(0xffffffffu, Sz[k].x, from);
                if constexpr (!kOne) {
                    Sx[k].y = __shfl_sync(0xffffffffu, Sx[k].y, from);
                    Sy[k].y = __shfl_sync(0xffffffffu, Sy[k].y, from);
                    Sz[k].y = __shfl_sync(0xffffffffu, Sz[k].y, from);
                }
            }
        }
        // fold the target partials into the compensated sums
#pragma unroll
        for (int q = Q0; q < Q1; ++q) {
            float4 *K = myk + q * 32 + lane;
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
    // this lane now holds its own group: sources (r, k, lane); the force on
    // a source is minus the sum of m_i (x_j - x_i) / r^3
#pragma unroll
    for (int k = 0; k < kKJ; ++k) {
        const int64_t idx = jbase + (r * kKJ + k) * 32 + lane;
        red_fixed(acc + idx, -(Sx[k].x + Sx[k].y), scJ, nonfinite);
        red_fixed(acc + np + idx, -(Sy[k].x + Sy[k].y), scJ, nonfinite);
        red_fixed(acc + 2 * np + idx, -(Sz[k].x + Sz[k].y), scJ, nonfinite);
    }
}

// One far unit for this warp without sub-blocks (every round over all the
// warp's targets): the same terms and order as sym_far_unit with mask 0,
// written as one loop nest (the round bodies of the sub-block kernel cost this
// kernel 0.6-1.6% when it shared them).
template <int KI, int UNR>
__device__ __forceinline__ void sym_far_unit_plain(const float4 *__restrict__ S, const float4 meta,
                                             const float2 *__restrict__ myio, float4 *__restrict__ myk,
                                             const float2 (&mi)[KI / 2], int lane, int64_t jbase, float scJ,
                                             unsigned long long *__restrict__ acc, int64_t np, int *nonfinite) {
    constexpr int kNP = KI / 2;
    constexpr int kR = KI / kKJ;  // rounds of 32 steps (32 KI sources, kKJ per lane and step)
    // The separation is formed as (o_j - o_i) - dc: the offsets are small (tile
    // scale) and dc is exact, so d carries only rounding relative to itself.
    // (Forming a shifted target s = o_i + dc once per unit would save one
    // addition, but its rounding acts as a shift of the target that is the same
    // for all its sources: a coherent error that does not average out.)
    float2 nox[kNP], noy[kNP], noz[kNP];  // -o_i
    float2 px[kNP], py[kNP], pz[kNP];     // FP32 target partials
    const float2 ndx = make_float2(-meta.x, -meta.x), ndy = make_float2(-meta.y, -meta.y),
                 ndz = make_float2(-meta.z, -meta.z);
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        nox[q] = myio[(0 * kNP + q) * 32 + lane];
        noy[q] = myio[(1 * kNP + q) * 32 + lane];
        noz[q] = myio[(2 * kNP + q) * 32 + lane];
        px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
    }
    const int from = (lane + 1) & 31;
#pragma unroll 1
    for (int r = 0; r < kR; ++r) {
        // running sums of the sources of group (lane + step) mod 32: with 4 targets
        // per lane the two packed halves are added before the rotation (6
        // shuffles per step instead of 12; measured 2% faster there, 1% slower
        // with 8 targets per lane)
        constexpr bool kOne = KI == 4;
        float2 Sx[kKJ], Sy[kKJ], Sz[kKJ];
#pragma unroll
        for (int k = 0; k < kKJ; ++k) Sx[k] = Sy[k] = Sz[k] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int h = 0; h < 32; h += kFold) {
#pragma unroll UNR
            for (int st = h; st < h + kFold; ++st) {
                const int g = (lane + st) & 31;
#pragma unroll
                for (int k = 0; k < kKJ; ++k) {
                    const float4 *src = S + (r * kKJ + k) * 64 + g;
                    const float4 A = src[0], B = src[32];
                    const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
                    const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
                    // this step's 8 targets on the two sources form a fresh partial that is
                    // added to the group's running sum once: the sum grows by 32 additions
                    // per round instead of 128 (its rounding grows with the additions)
                    float2 tx, ty, tz;
#pragma unroll
                    for (int q = 0; q < kNP; ++q) {
                        const float2 dx = __fadd2_rn(__fadd2_rn(xj, nox[q]), ndx);  // x_j - x_i
                        const float2 dy = __fadd2_rn(__fadd2_rn(yj, noy[q]), ndy);
                        const float2 dz = __fadd2_rn(__fadd2_rn(zj, noz[q]), ndz);
                        float2 r2 = __fmul2_rn(dx, dx);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        const float2 w = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                        const float2 u = __fmul2_rn(__fmul2_rn(w, w), w);  // 1/r^3
                        const float2 si = __fmul2_rn(u, mj);
                        px[q] = __ffma2_rn(si, dx, px[q]);
                        py[q] = __ffma2_rn(si, dy, py[q]);
                        pz[q] = __ffma2_rn(si, dz, pz[q]);
                        const float2 sj = __fmul2_rn(u, mi[q]);
                        if (q == 0) {
                            tx = __fmul2_rn(sj, dx);
                            ty = __fmul2_rn(sj, dy);
                            tz = __fmul2_rn(sj, dz);
                        } else {
                            tx = __ffma2_rn(sj, dx, tx);
                            ty = __ffma2_rn(sj, dy, ty);
                            tz = __ffma2_rn(sj, dz, tz);
                        }
                    }
                    if constexpr (kOne) {
                        Sx[k].x = __fadd_rn(Sx[k].x, __fadd_rn(tx.x, tx.y));
                        Sy[k].x = __fadd_rn(Sy[k].x, __fadd_rn(ty.x, ty.y));
                        Sz[k].x = __fadd_rn(Sz[k].x, __fadd_rn(tz.x, tz.y));
                    } else {
                        Sx[k] = __fadd2_rn(Sx[k], tx);
                        Sy[k] = __fadd2_rn(Sy[k], ty);
                        Sz[k] = __fadd2_rn(Sz[k], tz);
                    }
                }
                // pass the group's sums on: lane l takes over group (l + st + 1) mod 32
#pragma unroll
                for (int k = 0; k < kKJ; ++k) {
                    Sx[k].x = __shfl_sync(0xffffffffu, Sx[k].x, from);
                    Sy[k].x = __shfl_sync(0xffffffffu, Sy[k].x, from);
                    Sz[k].x = __shfl_sync(0xffffffffu, Sz[k].x, from);
                    if constexpr (!kOne) {
                        Sx[k].y = __shfl_sync(0xffffffffu, Sx[k].y, from);
                        Sy[k].y = __shfl_sync(0xffffffffu, Sy[k].y, from);
                        Sz[k].y = __shfl_sync(0xffffffffu, Sz[k].y, from);
                    }
                }
            }
            // fold the target partials into the compensated sums
#pragma unroll
            for (int q = 0; q < kNP; ++q) {
                float4 *K = myk + q * 32 + lane;
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
        // this lane now holds its own group: sources (r, k, lane); the force on
        // a source is minus the sum of m_i (x_j - x_i) / r^3
#pragma unroll
        for (int k = 0; k < kKJ; ++k) {
            const int64_t idx = jbase + (r * kKJ + k) * 32 + lane;
            red_fixed(acc + idx, -(Sx[k].x + Sx[k].y), scJ, nonfinite);
            red_fixed(acc + np + idx, -(Sy[k].x + Sy[k].y), scJ, nonfinite);
            red_fixed(acc + 2 * np + idx, -(Sz[k].x + Sz[k].y), scJ, nonfinite);
        }
    }
}

// One far unit for this warp: the warp's 32 KI targets against the 32 KI
// sources of the staged tile S.  meta = (dc = c_I - c_J, M_J); myio holds the
// negated target offsets.  Target sums go to the Kahan state myk; source sums
// to the fixed-point array (scale scJ) of the source tile starting at
// particle jbase.  mask (256-particle tiles only): bit 2 hI + hJ set = the
// sub-block of target half hI and source half hJ is near and left to the
// near-field kernel.
template <int KI, int UNR, bool SUB>
__device__ __forceinline__ void sym_far_unit(const float4 *__restrict__ S, const float4 meta, int mask,
                                             const float2 *__restrict__ myio, float4 *__restrict__ myk,
                                             const float2 (&mi)[KI / 2], int lane, int64_t jbase, float scJ,
                                             unsigned long long *__restrict__ acc, int64_t np, int *nonfinite) {
    constexpr int kNP = KI / 2;
    constexpr int kR = KI / kKJ;  // rounds of 32 steps (32 KI sources, kKJ per lane and step)
    // The separation is formed as (o_j - o_i) - dc: the offsets are small (tile
    // scale) and dc is exact, so d carries only rounding relative to itself.
    // (Forming a shifted target s = o_i + dc once per unit would save one
    // addition, but its rounding acts as a shift of the target that is the same
    // for all its sources: a coherent error that does not average out.)
    float2 nox[kNP], noy[kNP], noz[kNP];  // -o_i
    float2 px[kNP], py[kNP], pz[kNP];     // FP32 target partials
    const float2 ndx = make_float2(-meta.x, -meta.x), ndy = make_float2(-meta.y, -meta.y),
                 ndz = make_float2(-meta.z, -meta.z);
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        nox[q] = myio[(0 * kNP + q) * 32 + lane];
        noy[q] = myio[(1 * kNP + q) * 32 + lane];
        noz[q] = myio[(2 * kNP + q) * 32 + lane];
        px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
    }
    const int from = (lane + 1) & 31;
#pragma unroll 1
    for (int r = 0; r < kR; ++r) {
        if constexpr (KI == 8 && SUB) {
            const int hJ = r / (kR / 2);  // source half of this round
            const bool a0 = !((mask >> hJ) & 1), a1 = !((mask >> (2 + hJ)) & 1);
            if (a0 && a1)
                sym_round<KI, UNR, 0, kNP>(S, r, ndx, ndy, ndz, nox, noy, noz, px, py, pz, mi, myk, lane, from,
                                           jbase, scJ, acc, np, nonfinite);
            else if (a0)
                sym_round<KI, UNR, 0, kNP / 2>(S, r, ndx, ndy, ndz, nox, noy, noz, px, py, pz, mi, myk, lane,
                                               from, jbase, scJ, acc, np, nonfinite);
            else if (a1)
                sym_round<KI, UNR, kNP / 2, kNP>(S, r, ndx, ndy, ndz, nox, noy, noz, px, py, pz, mi, myk, lane,
                                                 from, jbase, scJ, acc, np, nonfinite);
        } else {
            sym_round<KI, UNR, 0, kNP>(S, r, ndx, ndy, ndz, nox, noy, noz, px, py, pz, mi, myk, lane, from, jbase,
                                       scJ, acc, np, nonfinite);
        }
    }
}

// Fill stage s = k mod NS with unit k of this CTA's range (cursor c): the W
// warps' metadata (dc, and M_J, or minus the near sub-block mask, or -16
// when the pair is another unit's) and the bulk copy of the source tile.
// Called by one whole warp.
template <int KI, int W, int NS, bool SUB>
__device__ __forceinline__ void sym_issue(const SymArgs &a, const UnitCursor<W> &c, int64_t k, float4 *sj,
                                          float4 *smeta, uint64_t *full, long long *issued, int lane) {
    constexpr int kT = 32 * KI;
    constexpr uint32_t BYTES_J = kT * 32u;
    const int s = (int)(k % NS);
    const int64_t jg = c.d.tile_off + c.J;
    if (lane < W) {
        const int64_t il = c.b * W + lane;
        const uint32_t word = a.nearbits[c.d.bits_off + il * c.d.words + (c.J >> 5)];
        // w: M_J for a far tile pair; -mask (the near sub-blocks, 15: all) for a
        // near one; -16 for target tiles at or after J (their pair with J is
        // another unit's)
        const bool near = (word >> (c.J & 31)) & 1u;
        const bool other = il >= c.J;
        int mask = 15;
        if constexpr (SUB)
            if (!other && near) mask = a.submask[(c.d.bits_off + il * c.d.words) * 32 + c.J];
        const float4 ci = a.tbox_c[c.d.tile_off + il], cj = a.tbox_c[jg];
        // exact: the tile centres lie on a common grid (staging)
        smeta[s * W + lane] = make_float4(__fsub_rn(ci.x, cj.x), __fsub_rn(ci.y, cj.y), __fsub_rn(ci.z, cj.z),
                                          other ? -16.f : (near ? -(float)mask : a.tbox_e[jg].w));
    }
    __syncwarp();
    if (lane == 0) {
        issued[s] = k;
        __threadfence_block();  // the metadata before the release-arrive
        // every warp's reads of the stage's previous tile before the async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t fb = smem_u32(&full[s]);
        mbar_arrive_expect_tx(fb, BYTES_J);
        bulk_g2s(smem_u32(sj + (size_t)s * 2 * kT), a.sdup + jg * 2 * kT, BYTES_J, fb);
    }
}

// The CTA's W warps share an NS-stage ring of source tiles.  There is no
// producer warp: warp 0 fills the first NS stages of a chunk, and afterwards
// the last warp done with a stage (a shared-memory counter) refills it with
// the unit NS further on, so every warp of the CTA computes.  (Measured against
// a dedicated producer warp: the same speed at equal compute warps, and the
// producer's registers go to a third CTA per SM.)
//
// The units are cut into fixed chunks of a.chunk consecutive units, and the
// persistent CTAs take chunks from a global counter: the warp schedulers favour
// the CTAs that arrived first on an SM, and with equal static shares the last
// CTA of each SM ran ~30% longer than the first.  Every chunk starts and
// flushes its own target sums, so the result does not depend on which CTA
// takes which chunk.
template <int KI, int W, int NS, int MINB, int UNR, bool SUB>
__global__ void __launch_bounds__(W * 32, MINB) sym_far_kernel(const SymArgs a) {
    constexpr int kT = 32 * KI;
    constexpr int kNP = KI / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *sj = reinterpret_cast<float4 *>(smem);                          // [NS][2 kT] source tiles
    float4 *smeta = sj + NS * 2 * kT;                                       // [NS][W] (dc, M_J or -1: near)
    float2 *sio = reinterpret_cast<float2 *>(smeta + NS * W);               // [W][3][kNP][32] -(target offsets)
    float4 *skah = reinterpret_cast<float4 *>(sio + W * 3 * kNP * 32);      // [W][3][kNP][32] Kahan (hi, -c)
    uint64_t *full = reinterpret_cast<uint64_t *>(skah + W * 3 * kNP * 32); // [NS]
    long long *issued = reinterpret_cast<long long *>(full + NS);          // [NS] last unit copied into a stage
    long long *chunk_slot = issued + NS;                                     // [2] the chunk taken, abort flag
    int *done = reinterpret_cast<int *>(chunk_slot + 2);                    // [NS] warps finished with a stage

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            issued[s] = -1;
            done[s] = 0;
        }
        chunk_slot[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    float2 *myio = sio + warp * 3 * kNP * 32;
    float4 *myk = skah + warp * 3 * kNP * 32;
    int64_t k = 0;  // units this CTA has taken through the ring (stage k mod NS, phase k / NS)
    for (;;) {
        if (threadIdx.x == 0) chunk_slot[0] = (long long)atomicAdd(a.next, 1ull);
        __syncthreads();
        const int64_t u0 = chunk_slot[0] * a.chunk;
        const bool abort = chunk_slot[1] != 0;
        __syncthreads();  // every thread has read the slot before it is written again
        if (abort || u0 >= a.units) break;
        const int64_t u1 = min(a.units, u0 + a.chunk);
        const int64_t count = u1 - u0;
        const int64_t k0 = k;

        UnitCursor<W> c;
        c.locate(a.sims, a.nsims, u0);
        if (warp == 0) {
            UnitCursor<W> p = c;
            for (int64_t t = 0; t < NS && t < count; ++t) {
                sym_issue<KI, W, NS, SUB>(a, p, k0 + t, sj, smeta, full, issued, lane);
                p.next(a.sims, a.nsims);
            }
        }

        int64_t u = u0;
        bool failed = false;
        while (u < u1 && !failed) {
            const int64_t seg_end = min(u1, c.d.unit_off + c.row_off(c.b + 1));
            const int64_t ig = c.d.tile_off + c.b * W + warp;  // this warp's target tile
            float2 mi[kNP];
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kNP; ++q) {
                const float4 *p0 = a.sdup + (ig * KI + 2 * q) * 64 + lane;  // particle 64 q + lane
                const float4 *p1 = p0 + 64;                                   // particle 64 q + 32 + lane
                const float4 A0 = p0[0], B0 = p0[32], A1 = p1[0], B1 = p1[32];
                myio[(0 * kNP + q) * 32 + lane] = make_float2(-A0.x, -A1.x);
                myio[(1 * kNP + q) * 32 + lane] = make_float2(-A0.z, -A1.z);
                myio[(2 * kNP + q) * 32 + lane] = make_float2(-B0.x, -B1.x);
                mi[q] = make_float2(B0.z, B1.z);
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) myk[(cc * kNP + q) * 32 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
            for (; u < seg_end; ++u, ++k) {
                const int s = (int)(k % NS);
                if (!mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((k / NS) & 1), a.wait_ns)) {
                    if (lane == 0) {
                        atomicExch(a.err, (int)STEPS_ETIMEOUT);
                        // drain the copies issued so far before the CTA leaves
                        for (int t = 0; t < NS; ++t) {
                            const long long q = ((volatile long long *)issued)[t];
                            if (q >= 0) mbar_wait_bounded(smem_u32(&full[t]), (uint32_t)((q / NS) & 1), kDrainNs);
                        }
                        ((volatile long long *)chunk_slot)[1] = 1;
                    }
                    failed = true;
                    break;
                }
                const float4 meta = smeta[s * W + warp];
                if constexpr (SUB) {
                    const int64_t jg = c.d.tile_off + c.J;
                    // far: mask 0; partly near: the near sub-blocks; 15 (all near) or 16: skip
                    const int mask = meta.w >= 0.f ? 0 : (int)(-meta.w);
                    if (mask < 15)
                        sym_far_unit<KI, UNR, SUB>(sj + (size_t)s * 2 * kT, meta, mask, myio, myk, mi, lane,
                                                   jg * kT, a.tscale[jg], a.acc, a.np, a.nonfinite);
                } else if (meta.w >= 0.f) {
                    const int64_t jg = c.d.tile_off + c.J;
                    sym_far_unit_plain<KI, UNR>(sj + (size_t)s * 2 * kT, meta, myio, myk, mi, lane, jg * kT,
                                                a.tscale[jg], a.acc, a.np, a.nonfinite);
                }
                // done with the stage: the last warp refills it with unit k + NS of the chunk
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    __threadfence_block();
                    last = atomicAdd(&done[s], 1) == W - 1;
                    if (last) done[s] = 0;
                }
                if (__shfl_sync(0xffffffffu, last, 0) && k - k0 + NS < count) {
                    UnitCursor<W> p = c;
                    for (int t = 0; t < NS; ++t) p.next(a.sims, a.nsims);
                    sym_issue<KI, W, NS, SUB>(a, p, k + NS, sj, smeta, full, issued, lane);
                }
                c.next(a.sims, a.nsims);
            }
            if (failed) break;
            // ---- segment done: this warp's target sums into the fixed-point array ----
            const float scI = a.tscale[ig];
#pragma unroll
            for (int q = 0; q < kNP; ++q) {
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    const float4 K = myk[(cc * kNP + q) * 32 + lane];
                    unsigned long long *dst = a.acc + cc * a.np + ig * kT + 64 * q + lane;
                    red_fixed(dst, K.x, scI, a.nonfinite);
                    red_fixed(dst, K.z, scI, a.nonfinite);
                    red_fixed(dst + 32, K.y, scI, a.nonfinite);
                    red_fixed(dst + 32, K.w, scI, a.nonfinite);
                }
            }
        }
        // a warp that timed out leaves its ring position behind: every warp
        // stops at this chunk's end
        k = k0 + count;
        __syncthreads();  // every warp is done with every stage before the next chunk's copies
    }
}

// Near bitmap of every ordered tile pair of a system (each tile with itself is
// near; tiles larger than their distance may be far: the separations are
// exact, and the alpha rule bounds their rounding), and the per-tile
// fixed-point scale.  The scale bounds the tile's far-field sums: a
// far pair of tiles contributes at most M_J / gap^2 to any particle of I (gap
// = the distance between their boxes, r >= gap for every pair), so every
// partial sum of tile I stays below B_I = sum_J M_J / gap_IJ^2; with
// 2 B_I < 2^E the scale 2^(62 - E) keeps every fixed-point value below 2^61.
// One warp per tile row.
template <int W>
__global__ void sym_classify_kernel(const float4 *__restrict__ tbox_c, const float4 *__restrict__ tbox_e,
                                    const float4 *__restrict__ hbox_c, const float4 *__restrict__ hbox_e,
                                    uint8_t *__restrict__ submask,
                                    const SimDesc *__restrict__ sims, int nsims, int64_t ntile_all,
                                    float alpha2, uint32_t *__restrict__ bits, float *__restrict__ tscale,
                                    double *__restrict__ tinv, unsigned long long *stats) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= ntile_all) return;
    const SimDesc d = sims[sim_of_tile(sims, nsims, row)];
    const int64_t I = row - d.tile_off;
    const float4 ci = tbox_c[row], ei = tbox_e[row];
    double bound = 0.0, bh[2] = {0.0, 0.0};  // bh: per half of I when sub-blocks are classified
    unsigned long long nn = 0;  // near tile pairs, or near sub-blocks (quarters of a pair)
    for (int64_t j0 = 0; j0 < d.ntile; j0 += 32) {
        const int64_t J = j0 + lane;
        bool near = false;
        if (J < d.ntile) {
            if (J == I) {
                near = true;
                if (submask) {
                    submask[(d.bits_off + I * d.words) * 32 + J] = 15;
                    nn += 3;  // with the 1 below: all four sub-blocks
                }
            } else if (submask) {
                // 128 x 128 sub-blocks: bit 2 hI + hJ marks half hI of I against
                // half hJ of J near; the far kernel takes the other sub-blocks.
                // A tile pair that is far as a whole has far halves (their boxes
                // lie inside the tiles'; the tile gap bounds both halves' sums).
                const float4 cj = tbox_c[d.tile_off + J], ej = tbox_e[d.tile_off + J];
                float tgap2 = 0.f;
                const bool tnear = tile_pair_near(ci, ei, cj, ej, alpha2, &tgap2, false);
                int mask = 0;
                if (!tnear) {
                    bh[0] += (double)ej.w / (double)tgap2;
                    bh[1] += (double)ej.w / (double)tgap2;
                }
#pragma unroll
                for (int hI = 0; hI < 2 && tnear; ++hI) {
#pragma unroll
                    for (int hJ = 0; hJ < 2; ++hJ) {
                        const float4 a = hbox_c[2 * row + hI], ae = hbox_e[2 * row + hI];
                        const float4 b = hbox_c[2 * (d.tile_off + J) + hJ], be = hbox_e[2 * (d.tile_off + J) + hJ];
                        float gap2 = 0.f;
                        if (tile_pair_near(a, ae, b, be, alpha2, &gap2, false))
                            mask |= 1 << (2 * hI + hJ);
                        else
                            bh[hI] += (double)be.w / (double)gap2;
                    }
                }
                near = mask != 0;
                submask[(d.bits_off + I * d.words) * 32 + J] = (uint8_t)mask;
                if (near) nn += __popc(mask) - 1;  // with the 1 below: the near sub-blocks
            } else {
                const float4 cj = tbox_c[d.tile_off + J], ej = tbox_e[d.tile_off + J];
                float gap2 = 0.f;
                near = tile_pair_near(ci, ei, cj, ej, alpha2, &gap2, false);
                if (!near) bound += (double)ej.w / (double)gap2;
            }
        }
        const unsigned word = __ballot_sync(0xffffffffu, near);
        if (lane == 0) bits[d.bits_off + I * d.words + (j0 >> 5)] = word;
        nn += near ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        bound += __shfl_xor_sync(0xffffffffu, bound, o);
        bh[0] += __shfl_xor_sync(0xffffffffu, bh[0], o);
        bh[1] += __shfl_xor_sync(0xffffffffu, bh[1], o);
        nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    // with sub-blocks every particle of half hI sums at most bh[hI]
    if (submask) bound = fmax(bh[0], bh[1]);
    if (lane == 0) {
        int e = -200;
        if (bound > 0.0) frexp(2.0 * bound, &e);  // 2 B < 2^e
        int sh = 62 - e;
        sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
        tscale[row] = ldexpf(1.0f, sh);
        tinv[row] = ldexp(1.0, -sh);
        if (stats) {
            atomicAdd(&stats[0], nn);
            atomicAdd(&stats[1], (unsigned long long)d.ntile * (submask ? 4 : 1));
        }
    }
}

// acc = G (far field in fixed point + near-field items in item order), sorted order.
__global__ void sym_fixup_kernel(const unsigned long long *__restrict__ acc, int64_t np, int kT,
                                 const double *__restrict__ tinv, const double *__restrict__ item_part,
                                 const int64_t *__restrict__ item_off, int64_t n, double Gc,
                                 double *__restrict__ ax, double *__restrict__ ay, double *__restrict__ az,
                                 int *nonfinite) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t row = p / kT;
    const int li = (int)(p - row * kT);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t it = item_off[row]; it < item_off[row + 1]; ++it) {
        const double *Q = item_part + (size_t)it * 3 * kT;
        sx += Q[li];
        sy += Q[kT + li];
        sz += Q[2 * kT + li];
    }
    const double inv = tinv[row];
    sx += (double)(long long)acc[p] * inv;
    sy += (double)(long long)acc[np + p] * inv;
    sz += (double)(long long)acc[2 * np + p] * inv;
    ax[p] = Gc * sx;
    ay[p] = Gc * sy;
    az[p] = Gc * sz;
    if (nonfinite && (!isfinite(sx) || !isfinite(sy) || !isfinite(sz))) *nonfinite = 1;
}

constexpr int kNS = 4;   // stages of the source-tile ring
constexpr int kUNR = 4;  // steps unrolled

template <int KI, int W>
constexpr size_t sym_smem_of() {
    return (size_t)kNS * 2 * (32 * KI) * 16 + (size_t)kNS * W * 16 + (size_t)W * 3 * (KI / 2) * 32 * 8 +
           (size_t)W * 3 * (KI / 2) * 32 * 16 + kNS * (sizeof(uint64_t) + sizeof(long long) + sizeof(int)) +
           2 * sizeof(long long);
}

using SymFn = void (*)(const SymArgs);

// The built kernels: 256-particle tiles at 3 CTAs per SM (up to 168
// registers), with or without 128 x 128 sub-blocks (the partial rounds are
// compiled into their own kernel: the extra round bodies cost the plain kernel
// 1.6% when they were in it), and 128-particle tiles at 4 CTAs per SM (up to 128).
SymFn sym_fn(int KI, int W, int ctas, bool sub) {
    if (W != 4) return nullptr;
    if (KI == 8 && ctas == 3) return sub ? sym_far_kernel<8, 4, kNS, 3, kUNR, true> : sym_far_kernel<8, 4, kNS, 3, kUNR, false>;
    if (KI == 4 && ctas == 4 && !sub) return sym_far_kernel<4, 4, kNS, 4, kUNR, false>;
    return nullptr;
}

}  // namespace

int64_t sym_units(int64_t ntile, int W) {
    const int64_t nb = ntile / W;
    return nb >= 1 ? nb * (ntile - 1) - (int64_t)W * nb * (nb - 1) / 2 : 0;
}

size_t sym_smem_bytes(int KI, int W) {
    if (W != 4) return 0;
    return KI == 8 ? sym_smem_of<8, 4>() : (KI == 4 ? sym_smem_of<4, 4>() : 0);
}

int sym_blocks_per_sm(int KI, int W, int ctas, bool sub) {
    SymFn fn = sym_fn(KI, W, ctas, sub);
    if (!fn) return 0;
    const size_t smem = sym_smem_bytes(KI, W);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, W * 32, smem) != cudaSuccess || per < 1)
        per = 1;
    return per;
}

cudaError_t launch_sym_classify(const Staging &s, const ForcePlan &p, const NearScratch &nr, float alpha,
                                unsigned long long *stats, cudaStream_t st) {
    const int W = variant(p.variant).W;
    const unsigned blocks = (unsigned)((s.ntile * 32 + 255) / 256);
    if (W != 4) return cudaErrorInvalidValue;
    // sub-block masks for the 256-particle variant when the staging has half boxes
    const bool sub = variant(p.variant).KI == 8 && s.tbox_hc && nr.submask;
    sym_classify_kernel<4><<<blocks, 256, 0, st>>>(s.tbox_c, s.tbox_e, sub ? s.tbox_hc : nullptr,
                                                   sub ? s.tbox_he : nullptr, sub ? nr.submask : nullptr, p.sims,
                                                   p.nsims, s.ntile, alpha * alpha, nr.bits, nr.tscale, nr.tinv,
                                                   stats);
    return cudaGetLastError();
}

cudaError_t launch_sym_far(const Staging &s, const ForcePlan &p, const NearScratch &nr, int *err,
                           long long wait_ns, cudaStream_t st) {
    const Variant &v = variant(p.variant);
    const int W = v.W;
    SymFn fn = sym_fn(v.KI, W, v.ctas, v.sub);
    if (!fn) return cudaErrorInvalidValue;
    SymArgs a;
    a.sdup = s.sdup;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.nearbits = nr.bits;
    a.submask = (v.KI == 8 && s.tbox_hc) ? nr.submask : nullptr;
    a.tscale = nr.tscale;
    a.acc = nr.sym_acc;
    a.nonfinite = nr.nonfinite;
    a.err = err;
    a.sims = p.sims;
    a.nsims = p.nsims;
    a.np = s.np;
    a.units = p.units;
    a.wait_ns = wait_ns;
    if (p.units <= 0) return cudaSuccess;
    if (!nr.sym_next) return cudaErrorInvalidValue;
    // about 64 chunks per CTA: a finishing tail of ~1/64 of a CTA's share (16, 32 and
    // 64 measured within 0.5% of each other at 262,144 and 2^20, 64 best)
    const int64_t want = (int64_t)std::max(p.grid, 1) * 64;
    a.chunk = std::max<int64_t>(1, (p.units + want - 1) / want);
    a.next = nr.sym_next;
    cudaError_t e = cudaMemsetAsync(nr.sym_next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    fn<<<p.grid, W * 32, sym_smem_bytes(v.KI, W), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sym_fixup(const Staging &s, const ForcePlan &p, const NearScratch &nr, double G,
                             double *ax, double *ay, double *az, cudaStream_t st) {
    (void)p;
    const int tb = 256;
    const int64_t blocks = (s.n + tb - 1) / tb;
    sym_fixup_kernel<<<(unsigned)blocks, tb, 0, st>>>(nr.sym_acc, s.np, s.T, nr.tinv, nr.item_part, nr.item_off, s.n,
                                                      G, ax, ay, az, nr.nonfinite);
    return cudaGetLastError();
}

}  // namespace steps

// Device helpers of the FP32 pair term shared by the force kernels
// (open-boundary near field, periodic images): MUFU rsqrt, the spline of
// Eq. 4, error-free sums, compensated folds, and the terms of one tile pair
// with exact separations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace steps {

// MUFU reciprocal square root (approximate, flush-to-zero).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Fcal(r, H)/r of Eq. 4 for r < H (u = r/H), in FP32.  The second branch is
// rewritten around v = 1 - u so that its polynomial has only positive terms
// (16/15 + 16/5 v + 32/5 v^2 + 32/3 v^3, algebraically identical to the printed
// form) and does not cancel near u = 1.
__device__ __forceinline__ float spline_over_r_f32(float r, float H) {
    const float Hinv = __frcp_rn(H);
    const float u = r * Hinv;
    const float Hinv3 = Hinv * Hinv * Hinv;
    float g;
    if (u < 0.5f) {
        g = 32.0f / 3.0f + u * u * (32.0f * u - 38.4f);
    } else {
        const float v = 1.0f - u;
        const float P = 16.0f / 15.0f + v * (3.2f + v * (6.4f + v * (32.0f / 3.0f)));
        g = P - __frcp_rn(15.0f * u * u * u);
    }
    return g * Hinv3;
}

// Error-free difference: a - b = s + e exactly (Knuth's TwoSum on a + (-b)).
__device__ __forceinline__ float two_diff(float a, float b, float &e) {
    const float s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
    return s;
}

// Error-free sum: a + b = s + e exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// Packed Kahan step for two targets at once: (hi, -c) absorbs p.
//   y = p - c;  t = hi + y;  c' = (t - hi) - y;  hi = t
// with nc = -c kept negated so that every step is one packed add or FMA.
__device__ __forceinline__ void kahan2(float2 &hi, float2 &nc, const float2 p) {
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float2 y = __fadd2_rn(p, nc);
    const float2 t = __fadd2_rn(hi, y);
    const float2 u = __ffma2_rn(hi, neg1, t);  // t - hi
    nc = __ffma2_rn(u, neg1, y);               // y - (t - hi) = -c'
    hi = t;
}

// Scalar Kahan step, same convention as kahan2 (nc holds the negated compensation).
__device__ __forceinline__ void kahan1(float &hi, float &nc, const float p) {
    const float y = __fadd_rn(p, nc);
    const float t = __fadd_rn(hi, y);
    nc = __fsub_rn(y, __fsub_rn(t, hi));
    hi = t;
}

// The terms of one near tile pair for this lane's KI targets (KI/2 packed
// pairs), folded into the targets' sums every FOLD sources.  Each source is
// read once from shared memory for all pairs.  SOFT: some pair may lie inside
// h_i + h_j (or the tile pair is a tile with itself): the packed loop leaves
// every pair with r^2 <= hT2 out, hT2 = (h_i + the source tile's largest h)^2
// (so every pair inside h_i + h_j, and the self pairs, r = 0), and flags the
// lane; after the fold the flagged lanes add those pairs, with the spline of
// Eq. 4 where r < h_i + h_j (h_i from RI) and the Newtonian term elsewhere
// (a warp vote: the whole warp calls this with the same SOFT).  Otherwise
// every pair is Newtonian and d != 0.
// NSRC: sources in the staged tile (default: a tile of 32 KI); only the
// sources [j_begin, j_end) are summed (multiples of FOLD).
template <int KI, bool COMP, int FOLD, bool SOFT, int NSRC = 32 * KI>
__device__ __forceinline__ void near_tile_terms(
    const float4 *__restrict__ S, const float4 *__restrict__ Rr, const float2 (&nxs)[KI / 2],
    const float2 (&nys)[KI / 2], const float2 (&nzs)[KI / 2], const float2 (&nrx)[KI / 2],
    const float2 (&nry)[KI / 2], const float2 (&nrz)[KI / 2], const float2 (&hT2)[KI / 2],
    const float4 *__restrict__ RI, float2 (&hx)[KI / 2],
    float2 (&hy)[KI / 2], float2 (&hz)[KI / 2], float2 (&cx_)[KI / 2], float2 (&cy_)[KI / 2],
    float2 (&cz_)[KI / 2], int j_begin = 0, int j_end = NSRC) {
    constexpr int NPAIR = KI / 2;
#pragma unroll 1
    for (int f0 = j_begin; f0 < j_end; f0 += FOLD) {
        float2 px[NPAIR], py[NPAIR], pz[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            if (COMP) {
                px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
            } else {
                px[q] = hx[q];
                py[q] = hy[q];
                pz[q] = hz[q];
            }
        }
        bool inner = false;  // this lane left a pair inside the softening out of the packed sum
#pragma unroll 4
        for (int j = f0; j < f0 + FOLD; ++j) {
            const float4 A = S[2 * j], B = S[2 * j + 1];
            const float4 RA = Rr[2 * j], RB = Rr[2 * j + 1];
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
                if (SOFT) {
                    const bool ix = r2.x <= hT2[q].x, iy = r2.y <= hT2[q].y;
                    inner = inner | ix | iy;
                    ri.x = ix ? 0.f : ri.x;
                    ri.y = iy ? 0.f : ri.y;
                }
                const float2 ri2 = __fmul2_rn(ri, ri);
                const float2 sc = __fmul2_rn(__fmul2_rn(make_float2(B.z, B.w), ri), ri2);
                px[q] = __ffma2_rn(sc, dx, px[q]);
                py[q] = __ffma2_rn(sc, dy, py[q]);
                pz[q] = __ffma2_rn(sc, dz, pz[q]);
            }
        }
        if (SOFT && __any_sync(0xffffffffu, inner) && inner) {
            // the pairs inside h_i + h_j of this fold, with the same FP32 separations
            for (int j = f0; j < f0 + FOLD; ++j) {
                const float4 A = S[2 * j], B = S[2 * j + 1];
                const float4 RA = Rr[2 * j], RB = Rr[2 * j + 1];
#pragma unroll
                for (int q = 0; q < NPAIR; ++q) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float dx = __fadd_rn(__fadd_rn(e ? A.y : A.x, e ? nxs[q].y : nxs[q].x),
                                                   __fadd_rn(e ? RA.y : RA.x, e ? nrx[q].y : nrx[q].x));
                        const float dy = __fadd_rn(__fadd_rn(e ? A.w : A.z, e ? nys[q].y : nys[q].x),
                                                   __fadd_rn(e ? RA.w : RA.z, e ? nry[q].y : nry[q].x));
                        const float dz = __fadd_rn(__fadd_rn(e ? B.y : B.x, e ? nzs[q].y : nzs[q].x),
                                                   __fadd_rn(e ? RB.y : RB.x, e ? nrz[q].y : nrz[q].x));
                        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                        if (r2 <= (e ? hT2[q].y : hT2[q].x) && r2 > 0.f) {
                            // RI: this lane's targets in the (rx, rx, ry, ry), (rz, rz, h, h) layout
                            const float H = __fadd_rn(RI[2 * (2 * q + e) + 1].z, e ? RB.w : RB.z);
                            const float H2 = __fmul_rn(H, H);
                            const float ri = rsqrt_approx(r2);
                            const float g = (r2 >= H2) ? ri * ri * ri : spline_over_r_f32(r2 * ri, H);
                            const float sc = (e ? B.w : B.z) * g;
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
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            if (COMP) {
                kahan2(hx[q], cx_[q], px[q]);
                kahan2(hy[q], cy_[q], py[q]);
                kahan2(hz[q], cz_[q], pz[q]);
            } else {
                hx[q] = px[q];
                hy[q] = py[q];
                hz[q] = pz[q];
            }
        }
    }
}

// Tile-pair classification (done once per pair by the far-field producer;
// the near-field kernel reads the resulting bitmap).  Conservative margins of
// 2^-18 cover the FP32 rounding of the box arithmetic.
//  * near if some pair may be closer than h_i + h_j (spline branches of Eq. 4);
//  * near if the boxes are closer than alpha x (|c_I - c_J| + |e_I| + |e_J|),
//    where one FP32 difference of offsets could lose relative precision in d;
//  * near if |e_I| + |e_J| > |c_I - c_J| (extents_rule): the one-sided far
//    field's first-order correction of the target shift uses the source
//    tile's monopole tidal tensor, which needs the tiles to be smaller than
//    their distance.  The symmetric far field forms exact separations and
//    has no such correction, so it classifies without this rule.
// gap2_out (may be null) receives the squared distance between the two boxes
// (rounded down), which bounds r^2 from below for every pair of the tiles.
__device__ __forceinline__ bool tile_pair_near(const float4 ci, const float4 ei, const float4 cj,
                                               const float4 ej, const float alpha2,
                                               float *gap2_out = nullptr, bool extents_rule = true) {
    const float up = 1.0f + 0x1p-18f, dn = 1.0f - 0x1p-18f;
    const float dcx = __fsub_rn(ci.x, cj.x), dcy = __fsub_rn(ci.y, cj.y), dcz = __fsub_rn(ci.z, cj.z);
    const float gx = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcx), dn), __fmul_rn(__fadd_rn(ei.x, ej.x), up)));
    const float gy = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcy), dn), __fmul_rn(__fadd_rn(ei.y, ej.y), up)));
    const float gz = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcz), dn), __fmul_rn(__fadd_rn(ei.z, ej.z), up)));
    const float gap2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    if (gap2_out) *gap2_out = gap2;
    const float hs = __fmul_rn(__fadd_rn(ci.w, cj.w), up);
    if (gap2 <= __fmul_rn(hs, hs)) return true;
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dcx, dcx), __fmul_rn(dcy, dcy)), __fmul_rn(dcz, dcz));
    const float ni = __fadd_rn(__fadd_rn(__fmul_rn(ei.x, ei.x), __fmul_rn(ei.y, ei.y)), __fmul_rn(ei.z, ei.z));
    const float nj = __fadd_rn(__fadd_rn(__fmul_rn(ej.x, ej.x), __fmul_rn(ej.y, ej.y)), __fmul_rn(ej.z, ej.z));
    const float dist = __fsqrt_rn(n2);
    const float ext = __fadd_rn(__fsqrt_rn(ni), __fsqrt_rn(nj));
    if (extents_rule && __fmul_rn(ext, up) > dist) return true;
    const float scale = __fadd_rn(dist, ext);
    return gap2 < __fmul_rn(alpha2, __fmul_rn(scale, scale));
}

}  // namespace steps

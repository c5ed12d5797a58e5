// FP32 direct-summation force kernels for sm_103a.
//
// Computes the pair term of the spherical comoving equation of motion (Eq. 8;
// Eq. 3 with the spline kernel of Eq. 4 and pair softening h_i + h_j):
//     acc_i = sum_{j != i} m_j (x_j - x_i) Fcal(|x_j - x_i|, h_i + h_j) / |x_j - x_i|
// (G is applied by the fixup kernel).  The O(N^2) sum is the most expensive
// part of the method ("the execution time scales as N(N-1)/2", Sec. 2.4).
//
// Design (GB300-first, not the paper's GTX 1080 Ti kernel):
//  * Particles are Morton-sorted; every tile of T = 32*KI consecutive particles
//    has an FP32 centre and half-extents.  Positions are stored as FP32 offsets
//    from the tile centre, computed from FP64.  A pair's separation is
//    (o_j - (o_i + (c_I - c_J))): its rounding error is relative to the local
//    scale (tile size or pair distance), never to the box size.
//  * Work is a stream-K split of the (i-block x j-tile) grid over a persistent
//    grid: every CTA gets the same number of tile pairs; per-CTA partial sums
//    per i-block are combined in a fixed order by the fixup kernel, so results
//    are deterministic and there are no atomics on the sums.
//  * A producer warp streams j tiles (32 B/particle duplicated layout + 4 B
//    softening) into an NS-stage shared-memory ring with cp.async.bulk
//    (TMA bulk copies) completing on mbarriers.
//  * Compute warps hold KI targets per thread as KI/2 packed pairs and use
//    Blackwell's packed FP32x2 FMA/ADD/MUL (FFMA2): 12 FP32 lane operations
//    + 1 MUFU rsqrt per interaction.  Each j element is one pair of
//    broadcast shared-memory loads.
//  * Tile pairs whose boxes are provably farther apart than the largest
//    h_i + h_j take a warp-uniform Newtonian fast path; the rest (neighbouring
//    tiles, self pairs) take the full spline path of Eq. 4.
//  * STEPS_F32_COMP: per-tile FP32 partial sums are folded into a per-target
//    (hi, lo) pair with TwoSum (compensated summation), O(N/T) per target.
//    STEPS_F32_NAIVE: a single FP32 running sum per target.
//  * Every mbarrier wait is bounded by a %globaltimer deadline; a wait that
//    runs out records STEPS_ETIMEOUT, the producer drains its own copies and
//    the CTA exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "steps_internal.h"

namespace steps {

namespace {

constexpr long long kDrainNs = 2000000000LL;  // bound for draining in-flight copies

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier to complete, giving up after
// limit_ns nanoseconds (limit_ns == 0: give up at once; used by tests).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit_ns) {
    if (limit_ns == 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 16; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

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

struct ForceArgs {
    const float4 *__restrict__ jdup;   // [2 np] (ox, ox, oy, oy), (oz, oz, m, m)
    const float4 *__restrict__ res;    // [np]   (rx, ry, rz, h): FP32 residual of the offset
    const float4 *__restrict__ tbox_c; // [ntile] (cx, cy, cz, hmax)
    const float4 *__restrict__ tbox_e; // [ntile] (ex, ey, ez, tile mass)
    double *__restrict__ partial;
    int *err;
    unsigned long long *stats;         // [2]: near tile pairs, all tile pairs (may be null)
    int64_t ntile;
    int64_t units;
    int smax;
    float alpha2;                      // near-field criterion (gap < alpha * scale), squared
    long long wait_ns;
};

// Pair term over all tile pairs of this CTA's stream-K range.
//   KI    targets per thread (KI/2 packed pairs), T = 32 KI particles per tile
//   W     compute warps; warp w owns target tile (block * W + w)
//   NS    shared-memory stages of j tiles
//   COMP  compensated (Kahan, every FOLD j) or naive FP32 running sums
template <int KI, int W, int NS, bool COMP, int FOLD, int MINB>
__global__ void __launch_bounds__((W + 1) * 32, MINB) force_f32_kernel(const ForceArgs a) {
    constexpr int T = 32 * KI;
    constexpr int NPAIR = KI / 2;
    constexpr int B_I = W * T;
    constexpr uint32_t BYTES_J = T * 32u;
    constexpr uint32_t BYTES_R = T * 16u;
    static_assert(T % FOLD == 0, "fold length must divide the tile");

    extern __shared__ __align__(128) unsigned char smem[];
    float4 *sj = reinterpret_cast<float4 *>(smem);
    float4 *sr = reinterpret_cast<float4 *>(smem + NS * BYTES_J);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * (BYTES_J + BYTES_R));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    const int64_t cta = blockIdx.x;
    const int64_t u0 = cta * a.units / G;
    const int64_t u1 = (cta + 1) * a.units / G;
    const int64_t count = u1 - u0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[NS + s]), W);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == W) {
        // ---------------- producer warp: stream j tiles ----------------
        if (lane == 0) {
            int64_t k = 0;
            bool ok = true;
            for (; k < count; ++k) {
                const int s = (int)(k % NS);
                if (k >= NS &&
                    !mbar_wait_bounded(smem_u32(&bars[NS + s]), (uint32_t)(((k / NS) - 1) & 1),
                                       a.wait_ns)) {
                    ok = false;
                    break;
                }
                const int64_t jt = (u0 + k) % a.ntile;
                const uint32_t full = smem_u32(&bars[s]);
                mbar_arrive_expect_tx(full, BYTES_J + BYTES_R);
                bulk_g2s(smem_u32(sj + (size_t)s * 2 * T), a.jdup + jt * 2 * T, BYTES_J, full);
                bulk_g2s(smem_u32(sr + (size_t)s * T), a.res + jt * T, BYTES_R, full);
            }
            if (!ok) atomicExch(a.err, (int)STEPS_ETIMEOUT);
            // drain: every copy this thread issued must land before the CTA may exit
            const int64_t first = k > NS ? k - NS : 0;
            for (int64_t q = first; q < k; ++q)
                if (!mbar_wait_bounded(smem_u32(&bars[q % NS]), (uint32_t)((q / NS) & 1), kDrainNs))
                    atomicExch(a.err, (int)STEPS_ETIMEOUT);
        }
        return;
    }

    // ---------------- compute warps ----------------
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    unsigned long long n_near = 0, n_all = 0;
    int64_t u = u0;
    int64_t k = 0;
    int seg = 0;
    while (u < u1) {
        const int64_t blk = u / a.ntile;
        const int64_t seg_end = min(u1, (blk + 1) * a.ntile);
        const int64_t itile = blk * W + warp;
        const float4 ci = a.tbox_c[itile];
        const float4 ei = a.tbox_e[itile];
        const int64_t ibase = itile * T + lane * KI;

        float2 xi[NPAIR], yi[NPAIR], zi[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const float4 p0 = a.jdup[2 * (ibase + 2 * q)];
            const float4 p0z = a.jdup[2 * (ibase + 2 * q) + 1];
            const float4 p1 = a.jdup[2 * (ibase + 2 * q + 1)];
            const float4 p1z = a.jdup[2 * (ibase + 2 * q + 1) + 1];
            xi[q] = make_float2(p0.x, p1.x);
            yi[q] = make_float2(p0.z, p1.z);
            zi[q] = make_float2(p0z.x, p1z.x);
        }
        float2 hx[NPAIR], hy[NPAIR], hz[NPAIR];     // running sums
        float2 cx_[NPAIR], cy_[NPAIR], cz_[NPAIR];  // Kahan terms (negated), COMP only
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            hx[q] = hy[q] = hz[q] = make_float2(0.f, 0.f);
            cx_[q] = cy_[q] = cz_[q] = make_float2(0.f, 0.f);
        }

        for (; u < seg_end; ++u, ++k) {
            const int s = (int)(k % NS);
            if (!mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((k / NS) & 1), a.wait_ns)) {
                if (lane == 0) atomicExch(a.err, (int)STEPS_ETIMEOUT);
                return;
            }
            const int64_t jt = u - blk * a.ntile;
            const float4 cj = a.tbox_c[jt];
            const float4 ej = a.tbox_e[jt];
            const float dcx = ci.x - cj.x, dcy = ci.y - cj.y, dcz = ci.z - cj.z;
            // Warp-uniform classification of the tile pair (conservative margins of
            // 2^-18 cover the FP32 rounding here):
            //  * near if any pair may be closer than h_i + h_j (spline of Eq. 4), or
            //  * near if the boxes are closer than alpha times the offset scale, where
            //    FP32 offsets alone could lose relative precision in d.
            const float gx = fmaxf(0.f, fabsf(dcx) * (1.0f - 0x1p-18f) - (ei.x + ej.x) * (1.0f + 0x1p-18f));
            const float gy = fmaxf(0.f, fabsf(dcy) * (1.0f - 0x1p-18f) - (ei.y + ej.y) * (1.0f + 0x1p-18f));
            const float gz = fmaxf(0.f, fabsf(dcz) * (1.0f - 0x1p-18f) - (ei.z + ej.z) * (1.0f + 0x1p-18f));
            const float gap2 = gx * gx + gy * gy + gz * gz;
            const float hs = (ci.w + cj.w) * (1.0f + 0x1p-18f);
            const float scale = sqrtf(dcx * dcx + dcy * dcy + dcz * dcz) +
                                sqrtf(ei.x * ei.x + ei.y * ei.y + ei.z * ei.z) +
                                sqrtf(ej.x * ej.x + ej.y * ej.y + ej.z * ej.z);
            const bool near = gap2 <= hs * hs || gap2 < a.alpha2 * scale * scale;
            n_near += near;
            n_all += 1;

            // negated target positions in the j tile's frame: -(o_i + (c_I - c_J))
            float2 nx[NPAIR], ny[NPAIR], nz[NPAIR];
            {
                const float2 ndx = make_float2(-dcx, -dcx), ndy = make_float2(-dcy, -dcy),
                             ndz = make_float2(-dcz, -dcz);
#pragma unroll
                for (int q = 0; q < NPAIR; ++q) {
                    nx[q] = __ffma2_rn(xi[q], neg1, ndx);
                    ny[q] = __ffma2_rn(yi[q], neg1, ndy);
                    nz[q] = __ffma2_rn(zi[q], neg1, ndz);
                }
            }
            const float4 *S = sj + (size_t)s * 2 * T;
            const float4 *R = sr + (size_t)s * T;
            if (!near) {
                // Far field.  xs = fl(o_i + dc) loses xs_lo = (o_i + c_I - c_J) - xs, and
                // that loss is the same for every j of the tile: left alone it would act
                // as a coherent shift of the target.  Undo it to first order with the
                // tile's monopole tidal tensor: p -= M (xs_lo/R^3 - 3 D (D.xs_lo)/R^5),
                // D = c_J - x_i ~ -xs.  Fast2Sum (|dc| >= |o_i| off the near field)
                // gives the rounding error of xs; two_diff that of dc.
                float2 ccx[NPAIR], ccy[NPAIR], ccz[NPAIR];
                {
                    float edx, edy, edz;
                    two_diff(ci.x, cj.x, edx);
                    two_diff(ci.y, cj.y, edy);
                    two_diff(ci.z, cj.z, edz);
                    const float2 dcx2 = make_float2(dcx, dcx), dcy2 = make_float2(dcy, dcy),
                                 dcz2 = make_float2(dcz, dcz);
                    const float2 edx2 = make_float2(edx, edx), edy2 = make_float2(edy, edy),
                                 edz2 = make_float2(edz, edz);
                    const float2 M2 = make_float2(ej.w, ej.w);
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        const float2 lx = __fadd2_rn(__fadd2_rn(xi[q], __fadd2_rn(nx[q], dcx2)), edx2);
                        const float2 ly = __fadd2_rn(__fadd2_rn(yi[q], __fadd2_rn(ny[q], dcy2)), edy2);
                        const float2 lz = __fadd2_rn(__fadd2_rn(zi[q], __fadd2_rn(nz[q], dcz2)), edz2);
                        float2 R2 = __fmul2_rn(nx[q], nx[q]);
                        R2 = __ffma2_rn(ny[q], ny[q], R2);
                        R2 = __ffma2_rn(nz[q], nz[q], R2);
                        const float2 Ri = make_float2(rsqrt_approx(R2.x), rsqrt_approx(R2.y));
                        const float2 Ri2 = __fmul2_rn(Ri, Ri);
                        const float2 k1 = __fmul2_rn(__fmul2_rn(M2, Ri), Ri2);
                        float2 proj = __fmul2_rn(nx[q], lx);
                        proj = __ffma2_rn(ny[q], ly, proj);
                        proj = __ffma2_rn(nz[q], lz, proj);
                        const float2 k2 = __fmul2_rn(__fmul2_rn(make_float2(3.f, 3.f), k1), __fmul2_rn(proj, Ri2));
                        const float2 nk1 = __fmul2_rn(k1, neg1);
                        ccx[q] = __ffma2_rn(k2, nx[q], __fmul2_rn(nk1, lx));
                        ccy[q] = __ffma2_rn(k2, ny[q], __fmul2_rn(nk1, ly));
                        ccz[q] = __ffma2_rn(k2, nz[q], __fmul2_rn(nk1, lz));
                    }
                }
#pragma unroll 1
                for (int j0 = 0; j0 < T; j0 += FOLD) {
                    float2 px[NPAIR], py[NPAIR], pz[NPAIR];
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        if (COMP) {
                            if (j0 == 0) {
                                px[q] = ccx[q];
                                py[q] = ccy[q];
                                pz[q] = ccz[q];
                            } else {
                                px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
                            }
                        } else {
                            px[q] = hx[q];
                            py[q] = hy[q];
                            pz[q] = hz[q];
                        }
                    }
#pragma unroll 2
                    for (int j = j0; j < j0 + FOLD; ++j) {
                        const float4 A = S[2 * j];
                        const float4 B = S[2 * j + 1];
                        const float2 xj = make_float2(A.x, A.y);
                        const float2 yj = make_float2(A.z, A.w);
                        const float2 zj = make_float2(B.x, B.y);
                        const float2 mj = make_float2(B.z, B.w);
#pragma unroll
                        for (int q = 0; q < NPAIR; ++q) {
                            const float2 dx = __fadd2_rn(xj, nx[q]);
                            const float2 dy = __fadd2_rn(yj, ny[q]);
                            const float2 dz = __fadd2_rn(zj, nz[q]);
                            float2 r2 = __fmul2_rn(dx, dx);
                            r2 = __ffma2_rn(dy, dy, r2);
                            r2 = __ffma2_rn(dz, dz, r2);
                            const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                            const float2 ri2 = __fmul2_rn(ri, ri);
                            float2 sc = __fmul2_rn(mj, ri);
                            sc = __fmul2_rn(sc, ri2);
                            px[q] = __ffma2_rn(sc, dx, px[q]);
                            py[q] = __ffma2_rn(sc, dy, py[q]);
                            pz[q] = __ffma2_rn(sc, dz, pz[q]);
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
            } else {
                // Near field: separation with the FP32 residuals of both offsets and the
                // exact rounding errors of c_I - c_J and o_i + (c_I - c_J), i.e. d to
                // ~1 ulp of |d| however large the tiles are; full spline kernel.
                float edx, edy, edz;
                two_diff(ci.x, cj.x, edx);
                two_diff(ci.y, cj.y, edy);
                two_diff(ci.z, cj.z, edz);
#pragma unroll
                for (int q = 0; q < NPAIR; ++q) {
                    // per target of this pair: -(r_i + err(c_I - c_J) + err(o_i + dc)), h_i
                    float nrx[2], nry[2], nrz[2], hI[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float4 ri4 = a.res[ibase + 2 * q + e];
                        float esx, esy, esz;
                        two_sum(e ? xi[q].y : xi[q].x, dcx, esx);
                        two_sum(e ? yi[q].y : yi[q].x, dcy, esy);
                        two_sum(e ? zi[q].y : zi[q].x, dcz, esz);
                        nrx[e] = -((ri4.x + edx) + esx);
                        nry[e] = -((ri4.y + edy) + esy);
                        nrz[e] = -((ri4.z + edz) + esz);
                        hI[e] = ri4.w;
                    }
#pragma unroll 1
                    for (int j0 = 0; j0 < T; j0 += FOLD) {
                        float2 px, py, pz;
                        if (COMP) {
                            px = py = pz = make_float2(0.f, 0.f);
                        } else {
                            px = hx[q];
                            py = hy[q];
                            pz = hz[q];
                        }
#pragma unroll 1
                        for (int j = j0; j < j0 + FOLD; ++j) {
                            const float4 A = S[2 * j];
                            const float4 B = S[2 * j + 1];
                            const float4 Rj = R[j];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const float dx = (A.x + (e ? nx[q].y : nx[q].x)) + (Rj.x + nrx[e]);
                                const float dy = (A.z + (e ? ny[q].y : ny[q].x)) + (Rj.y + nry[e]);
                                const float dz = (B.x + (e ? nz[q].y : nz[q].x)) + (Rj.z + nrz[e]);
                                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                if (r2 > 0.f) {  // r2 == 0: the particle itself or a coincident one
                                    const float H = hI[e] + Rj.w;
                                    const float ri = rsqrt_approx(r2);
                                    const float g =
                                        (r2 >= H * H) ? ri * ri * ri : spline_over_r_f32(r2 * ri, H);
                                    const float sc = B.z * g;
                                    if (e) {
                                        px.y = fmaf(sc, dx, px.y);
                                        py.y = fmaf(sc, dy, py.y);
                                        pz.y = fmaf(sc, dz, pz.y);
                                    } else {
                                        px.x = fmaf(sc, dx, px.x);
                                        py.x = fmaf(sc, dy, py.x);
                                        pz.x = fmaf(sc, dz, pz.x);
                                    }
                                }
                            }
                        }
                        if (COMP) {
                            kahan2(hx[q], cx_[q], px);
                            kahan2(hy[q], cy_[q], py);
                            kahan2(hz[q], cz_[q], pz);
                        } else {
                            hx[q] = px;
                            hy[q] = py;
                            hz[q] = pz;
                        }
                    }
                }
            }
            // release the stage so the producer can refill it
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[NS + s]));
        }
        // ---- segment done: write this CTA's partial sums for block blk ----
        double *P = a.partial + ((size_t)(cta * a.smax + seg) * 3) * B_I;
        const int loc = warp * T + lane * KI;
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            P[0 * B_I + loc + 2 * q] = (double)hx[q].x + (double)cx_[q].x;
            P[0 * B_I + loc + 2 * q + 1] = (double)hx[q].y + (double)cx_[q].y;
            P[1 * B_I + loc + 2 * q] = (double)hy[q].x + (double)cy_[q].x;
            P[1 * B_I + loc + 2 * q + 1] = (double)hy[q].y + (double)cy_[q].y;
            P[2 * B_I + loc + 2 * q] = (double)hz[q].x + (double)cz_[q].x;
            P[2 * B_I + loc + 2 * q + 1] = (double)hz[q].y + (double)cz_[q].y;
        }
        ++seg;
    }
    if (a.stats && lane == 0) {
        atomicAdd(&a.stats[0], n_near);
        atomicAdd(&a.stats[1], n_all);
    }
}

__device__ __forceinline__ int64_t cta_start(int64_t c, int64_t units, int64_t G) {
    return c * units / G;
}

// Sum the per-CTA partials of each target in CTA order; apply G; sorted order.
__global__ void fixup_kernel(const double *__restrict__ partial, int64_t n, int64_t ntile,
                             int64_t units, int64_t G, int smax, int B_I, double Gc,
                             double *__restrict__ ax, double *__restrict__ ay,
                             double *__restrict__ az) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t blk = p / B_I;
    const int loc = (int)(p - blk * B_I);
    const int64_t ufirst = blk * ntile;
    const int64_t ulast = ufirst + ntile - 1;
    auto cta_of = [&](int64_t uu) {
        int64_t c = uu * G / units;
        while (c + 1 < G && cta_start(c + 1, units, G) <= uu) ++c;
        while (c > 0 && cta_start(c, units, G) > uu) --c;
        return c;
    };
    const int64_t clo = cta_of(ufirst), chi = cta_of(ulast);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t c = clo; c <= chi; ++c) {
        const int64_t seg = blk - cta_start(c, units, G) / ntile;
        const double *P = partial + ((size_t)(c * smax + seg) * 3) * B_I;
        sx += P[loc];
        sy += P[B_I + loc];
        sz += P[2 * B_I + loc];
    }
    ax[p] = Gc * sx;
    ay[p] = Gc * sy;
    az[p] = Gc * sz;
}

using KernelFn = void (*)(const ForceArgs);

template <int KI, int NS>
constexpr size_t smem_of() {
    return (size_t)NS * (32 * KI) * 48 + 2 * NS * sizeof(uint64_t);
}

struct VariantImpl {
    Variant v;
    KernelFn fn;
    size_t smem;
};

#define STEPS_VARIANT(KI, W, NS, COMP, FOLD, MINB, NAME)                                  \
    {{KI, W, NS, COMP, NAME}, force_f32_kernel<KI, W, NS, COMP, FOLD, MINB>, smem_of<KI, NS>()}

const VariantImpl kVariants[] = {
    STEPS_VARIANT(4, 8, 4, true, 32, 2, "comp_ki4_w8_ns4_f32"),
    STEPS_VARIANT(4, 4, 4, true, 32, 3, "comp_ki4_w4_ns4_f32"),
    STEPS_VARIANT(8, 4, 3, true, 32, 1, "comp_ki8_w4_ns3_f32"),
    STEPS_VARIANT(2, 8, 4, true, 32, 3, "comp_ki2_w8_ns4_f32"),
    STEPS_VARIANT(4, 8, 4, false, 32, 2, "naive_ki4_w8_ns4"),
    STEPS_VARIANT(4, 4, 4, false, 32, 3, "naive_ki4_w4_ns4"),
    STEPS_VARIANT(8, 4, 3, false, 32, 1, "naive_ki8_w4_ns3"),
    STEPS_VARIANT(2, 8, 4, false, 32, 3, "naive_ki2_w8_ns4"),
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int num_variants() { return kNumVariants; }
const Variant &variant(int k) { return kVariants[k].v; }
size_t force_smem_bytes(int k) { return kVariants[k].smem; }

ForcePlan plan_force(const Staging &s, int k, int num_sms) {
    const VariantImpl &vi = kVariants[k];
    ForcePlan p;
    p.variant = k;
    p.B_I = vi.v.W * 32 * vi.v.KI;
    p.niblk = s.np / p.B_I;
    p.units = p.niblk * s.ntile;
    int per_sm = 1;
    cudaFuncSetAttribute(vi.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vi.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vi.fn, (vi.v.W + 1) * 32, vi.smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > p.units) grid = p.units;
    if (grid < 1) grid = 1;
    p.grid = (int)grid;
    const int64_t per_cta = (p.units + grid - 1) / grid;
    p.smax = (int)((per_cta + s.ntile - 1) / s.ntile + 1);
    p.partial_elems = (size_t)p.grid * p.smax * 3 * p.B_I;
    return p;
}

cudaError_t launch_force_f32(const ForcePlan &p, const Staging &s, double *partial, int *err,
                             unsigned long long *stats, float alpha, long long wait_ns,
                             cudaStream_t st) {
    const VariantImpl &vi = kVariants[p.variant];
    ForceArgs a;
    a.jdup = s.jdup;
    a.res = s.res;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.partial = partial;
    a.err = err;
    a.stats = stats;
    a.ntile = s.ntile;
    a.units = p.units;
    a.smax = p.smax;
    a.alpha2 = alpha * alpha;
    a.wait_ns = wait_ns;
    vi.fn<<<p.grid, (vi.v.W + 1) * 32, vi.smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fixup(const ForcePlan &p, const Staging &s, const double *partial, double G,
                         double *ax, double *ay, double *az, cudaStream_t st) {
    const int tb = 256;
    const int64_t blocks = (s.n + tb - 1) / tb;
    fixup_kernel<<<(unsigned)blocks, tb, 0, st>>>(partial, s.n, s.ntile, p.units, p.grid, p.smax,
                                                  p.B_I, G, ax, ay, az);
    return cudaGetLastError();
}

}  // namespace steps

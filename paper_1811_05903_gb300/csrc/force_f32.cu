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
//  * A producer warp streams j tiles into an NS-stage shared-memory ring with
//    cp.async.bulk (TMA bulk copies) completing on mbarriers, and classifies
//    every tile pair: far pairs (provably Newtonian, r >= h_i + h_j, and far
//    enough for the FP32 arithmetic below) stay in this kernel; near pairs
//    (neighbours, self pairs, pairs that may lie inside the softening) are
//    marked in a bitmap and summed by the near-field kernel with exact
//    separations and the full spline of Eq. 4.
//  * Compute warps hold KI targets per thread as KI/2 packed pairs and use
//    Blackwell's packed FP32x2 FMA/ADD/MUL (FFMA2).  Explicit form: 12 FP32
//    lane operations + 1 MUFU rsqrt per interaction from a 32-byte-per-source
//    duplicated layout.  Expansion form (the tuned default): |o_j - s|^2
//    expanded about the source tile's centre with the mass folded in, 10 lane
//    operations + 1 MUFU from a 64-byte layout.  Each source is a few
//    broadcast shared-memory loads shared by all of a thread's target pairs.
//  * STEPS_F32_COMP: per-tile FP32 partial sums are folded into a per-target
//    (hi, lo) pair with TwoSum (compensated summation) every FOLD sources.
//    STEPS_F32_NAIVE: a single FP32 running sum per target.
//  * Every mbarrier wait is bounded by a %globaltimer deadline; a wait that
//    runs out records STEPS_ETIMEOUT, the producer drains its own copies and
//    the CTA exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "async_copy.cuh"
#include "pair_terms.cuh"
#include "systems.cuh"
#include "steps_internal.h"

namespace steps {

namespace {

// Far tile pair by expansion about the source tile's centre (EXP variants).
// With s = fl(o_i + (c_I - c_J)) the target relative to the source tile's
// centre, n = -s and k_j = m_j^(-2/3) rounded to FP32,
//     k_j |o_j - s|^2 = k_j |n|^2 + k_j |o_j|^2 + (2 k_j o_j) . n,
// a four-step FMA chain on the staged coefficients (k_j, k_j |o_j|^2, 2 k_j o_j).
// Its reciprocal square root w gives w^3 = m_j / r^3 with no mass product, and
//     sum_j m_j (o_j - s) / r^3 = sum_j w^3 o_j + n sum_j w^3,
// so an interaction costs 4 (squared distance) + 2 (w^3) + 4 (the two sums)
// = 10 FP32 lane operations and one MUFU rsqrt, against 12 for the explicit
// separation.  The rounding of the chain is relative to (|s| + |o_j|)^2
// instead of r^2; far pairs are never closer than 1/32 of the tiles' distance
// plus extents (the near-field criterion), which bounds that growth.  Every
// FOLD sources the sums are combined (S + n S0) and folded into the Kahan
// state.  The coherent rounding of s is undone to first order with the
// source tile's monopole tidal tensor, as in the explicit form.
template <int KI, int T, int FOLD, int UNR, bool SMK, int W>
__device__ __forceinline__ void far_tile_expansion(
    const float4 *__restrict__ S, const float4 m0, const float4 m1, const float4 *myipos, int lane,
    int tid, float2 *skah, float2 (&hx)[KI / 2], float2 (&hy)[KI / 2], float2 (&hz)[KI / 2],
    float2 (&cx_)[KI / 2], float2 (&cy_)[KI / 2], float2 (&cz_)[KI / 2]) {
    constexpr int NPAIR = KI / 2;
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    float2 nx[NPAIR], ny[NPAIR], nz[NPAIR], ss[NPAIR];
    float2 px[NPAIR], py[NPAIR], pz[NPAIR];  // sum of w^3 o_j (starts at the shift correction)
    {
        const float2 dcx2 = make_float2(m0.x, m0.x), dcy2 = make_float2(m0.y, m0.y),
                     dcz2 = make_float2(m0.z, m0.z);
        const float2 edx2 = make_float2(m1.x, m1.x), edy2 = make_float2(m1.y, m1.y),
                     edz2 = make_float2(m1.z, m1.z);
        const float2 ndx = make_float2(-m0.x, -m0.x), ndy = make_float2(-m0.y, -m0.y),
                     ndz = make_float2(-m0.z, -m0.z);
        const float2 M2 = make_float2(m0.w, m0.w);
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const float4 i0 = myipos[lane * KI + 2 * q];
            const float4 i1 = myipos[lane * KI + 2 * q + 1];
            const float2 xi = make_float2(i0.x, i1.x), yi = make_float2(i0.y, i1.y),
                         zi = make_float2(i0.z, i1.z);
            nx[q] = __ffma2_rn(xi, neg1, ndx);
            ny[q] = __ffma2_rn(yi, neg1, ndy);
            nz[q] = __ffma2_rn(zi, neg1, ndz);
            // rounding error of s (exact: Fast2Sum) plus that of c_I - c_J
            const float2 lx = __fadd2_rn(__fadd2_rn(xi, __fadd2_rn(nx[q], dcx2)), edx2);
            const float2 ly = __fadd2_rn(__fadd2_rn(yi, __fadd2_rn(ny[q], dcy2)), edy2);
            const float2 lz = __fadd2_rn(__fadd2_rn(zi, __fadd2_rn(nz[q], dcz2)), edz2);
            float2 R2 = __fmul2_rn(nx[q], nx[q]);
            R2 = __ffma2_rn(ny[q], ny[q], R2);
            R2 = __ffma2_rn(nz[q], nz[q], R2);
            ss[q] = R2;
            const float2 Ri = make_float2(rsqrt_approx(R2.x), rsqrt_approx(R2.y));
            const float2 Ri2 = __fmul2_rn(Ri, Ri);
            const float2 k1 = __fmul2_rn(__fmul2_rn(M2, Ri), Ri2);
            float2 proj = __fmul2_rn(nx[q], lx);
            proj = __ffma2_rn(ny[q], ly, proj);
            proj = __ffma2_rn(nz[q], lz, proj);
            const float2 k2 = __fmul2_rn(__fmul2_rn(make_float2(3.f, 3.f), k1), __fmul2_rn(proj, Ri2));
            const float2 nk1 = __fmul2_rn(k1, neg1);
            px[q] = __ffma2_rn(k2, nx[q], __fmul2_rn(nk1, lx));
            py[q] = __ffma2_rn(k2, ny[q], __fmul2_rn(nk1, ly));
            pz[q] = __ffma2_rn(k2, nz[q], __fmul2_rn(nk1, lz));
        }
    }
#pragma unroll 1
    for (int j0 = 0; j0 < T; j0 += FOLD) {
        float2 p0[NPAIR];  // sum of w^3
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) p0[q] = make_float2(0.f, 0.f);
#pragma unroll UNR
        for (int j = j0; j < j0 + FOLD; ++j) {
            const float4 A = S[4 * j];
            const float4 B = S[4 * j + 1];
            const float4 C = S[4 * j + 2];
            const float4 D = S[4 * j + 3];
            const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
            const float2 zj = make_float2(B.x, B.y), kj = make_float2(B.z, B.w);
            const float2 axj = make_float2(C.x, C.y), ayj = make_float2(C.z, C.w);
            const float2 azj = make_float2(D.x, D.y), bj = make_float2(D.z, D.w);
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                float2 t = __ffma2_rn(kj, ss[q], bj);
                t = __ffma2_rn(axj, nx[q], t);
                t = __ffma2_rn(ayj, ny[q], t);
                t = __ffma2_rn(azj, nz[q], t);
                const float2 w = make_float2(rsqrt_approx(t.x), rsqrt_approx(t.y));
                const float2 sc = __fmul2_rn(__fmul2_rn(w, w), w);
                px[q] = __ffma2_rn(sc, xj, px[q]);
                py[q] = __ffma2_rn(sc, yj, py[q]);
                pz[q] = __ffma2_rn(sc, zj, pz[q]);
                p0[q] = __fadd2_rn(p0[q], sc);
            }
        }
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const float2 qx = __ffma2_rn(nx[q], p0[q], px[q]);
            const float2 qy = __ffma2_rn(ny[q], p0[q], py[q]);
            const float2 qz = __ffma2_rn(nz[q], p0[q], pz[q]);
            if (SMK) {
                float2 *K = skah + q * 32 * W + tid;
                constexpr int CS = NPAIR * 32 * W;  // component stride
                float2 h0 = K[0], h1 = K[CS], h2 = K[2 * CS];
                float2 c0 = K[3 * CS], c1 = K[4 * CS], c2 = K[5 * CS];
                kahan2(h0, c0, qx);
                kahan2(h1, c1, qy);
                kahan2(h2, c2, qz);
                K[0] = h0;
                K[CS] = h1;
                K[2 * CS] = h2;
                K[3 * CS] = c0;
                K[4 * CS] = c1;
                K[5 * CS] = c2;
            } else {
                kahan2(hx[q], cx_[q], qx);
                kahan2(hy[q], cy_[q], qy);
                kahan2(hz[q], cz_[q], qz);
            }
            px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
        }
    }
}

struct ForceArgs {
    const float4 *__restrict__ jdup;   // [2 np] (ox, ox, oy, oy), (oz, oz, m, m)
    const float4 *__restrict__ rdup;   // [2 np] (rx, rx, ry, ry), (rz, rz, h, h): offset residual, softening
    const float4 *__restrict__ fdup;   // [4 np] expansion layout (Staging::fdup), expansion variants only
    const float4 *__restrict__ tbox_c; // [ntile] (cx, cy, cz, hmax)
    const float4 *__restrict__ tbox_e; // [ntile] (ex, ey, ez, tile mass)
    double *__restrict__ partial;      // far field: per-CTA, per-segment partial sums
    double *__restrict__ item_part;    // near field: [items][3][T] partial sums
    uint32_t *__restrict__ nearbits;   // [ntile][words]: tile pair (I, J) is near
    // per tile pair, the near 128 x 128 sub-blocks (bit 2 hI + hJ), or null:
    // the near field then takes whole tile pairs
    const uint8_t *__restrict__ submask;
    const int *__restrict__ near_cnt;  // [ntile] near tiles per target tile
    const int64_t *__restrict__ item_off;  // [ntile + 1] first work item of each target tile
    int64_t *near_meta;                // {chunk, items, work counter}
    int *err;
    unsigned long long *stats;         // [2]: near tile pairs, all tile pairs (may be null)
    const SimDesc *__restrict__ sims;  // independent systems (one for a single simulation)
    int nsims;
    int64_t ntile;                     // tiles, all systems
    int64_t units;                     // tile pairs, all systems
    int smax;
    float alpha2;                      // near-field criterion, squared
    long long wait_ns;
};

// Far field of the pair term over this CTA's stream-K range of tile pairs.
//   KI    targets per thread (KI/2 packed pairs), T = 32 KI particles per tile
//   W     compute warps; warp w owns target tile (block * W + w)
//   NS    shared-memory stages of j tiles
//   COMP  compensated (Kahan, every FOLD j) or naive FP32 running sums
// The producer warp streams j tiles with TMA bulk copies and, per tile and
// compute warp, classifies the tile pair, records near pairs in the bitmap
// (summed later by near_f32_kernel) and stages c_I - c_J (split exactly into
// a float and its rounding error) and the tile mass in shared memory.  The
// compute warps then only see far tile pairs, all of equal cost.
//   KSM   keep the Kahan state (touched once per FOLD sources) in shared memory
//         instead of registers, trading LSU work for occupancy
//   EXP   far-field arithmetic by expansion about the source tile centre (see
//         the far-tile branch below): 10 FP32 lane operations per interaction
//         instead of 12, from the 64-byte-per-source layout Staging::fdup
template <int KI, int W, int NS, bool COMP, int FOLD, int MINB, int UNR, bool KSM, bool EXP>
__global__ void __launch_bounds__((W + 1) * 32, MINB) force_f32_kernel(const ForceArgs a) {
    constexpr int T = 32 * KI;
    constexpr int NPAIR = KI / 2;
    constexpr int B_I = W * T;
    constexpr int V = EXP ? 4 : 2;  // float4 per source in shared memory
    constexpr uint32_t BYTES_J = T * 16u * V;
    constexpr bool SMK = COMP && KSM;
    static_assert(T % FOLD == 0, "fold length must divide the tile");
    static_assert(W <= 32, "one producer lane per compute warp");
    static_assert(!EXP || COMP, "the expansion form is built for compensated sums");

    extern __shared__ __align__(128) unsigned char smem[];
    float4 *sj = reinterpret_cast<float4 *>(smem);                                // [NS][V T]
    float4 *smeta = reinterpret_cast<float4 *>(smem + NS * BYTES_J);              // [NS][W][2]
    float4 *sipos = smeta + NS * W * 2;                                           // [W][T]
    float2 *skah = reinterpret_cast<float2 *>(sipos + W * T);                     // [6][NPAIR][32 W] (SMK)
    uint64_t *bars = reinterpret_cast<uint64_t *>(skah + (SMK ? 6 * NPAIR * 32 * W : 0));  // full, empty

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
        // ---------------- producer warp ----------------
        // walk (system, target block, source tile) through the unit range
        int64_t k = 0;
        bool ok = true;
        int sidx = sim_of_unit(a.sims, a.nsims, u0);
        SimDesc d = a.sims[sidx];
        int64_t blk = (u0 - d.unit_off) / d.ntile;
        int64_t jt = (u0 - d.unit_off) - blk * d.ntile;
        bool reload = true;
        float4 ci = make_float4(0.f, 0.f, 0.f, 0.f), ei = ci;
        unsigned long long n_near = 0;
        for (; k < count; ++k) {
            const int s = (int)(k % NS);
            if (reload) {
                reload = false;
                if (lane < W) {
                    ci = a.tbox_c[d.tile_off + blk * W + lane];
                    ei = a.tbox_e[d.tile_off + blk * W + lane];
                }
            }
            const int64_t gjt = d.tile_off + jt;
            const float4 cj = a.tbox_c[gjt];
            const float4 ej = a.tbox_e[gjt];
            bool near = false;
            float dcx = 0.f, dcy = 0.f, dcz = 0.f, edx = 0.f, edy = 0.f, edz = 0.f;
            if (lane < W) {
                near = tile_pair_near(ci, ei, cj, ej, a.alpha2);
                dcx = two_diff(ci.x, cj.x, edx);
                dcy = two_diff(ci.y, cj.y, edy);
                dcz = two_diff(ci.z, cj.z, edz);
                if (near) {
                    atomicOr(&a.nearbits[d.bits_off + (blk * W + lane) * d.words + (jt >> 5)],
                             1u << (jt & 31));
                    ++n_near;
                }
            }
            if (k >= NS) {
                bool got = true;
                if (lane == 0)
                    got = mbar_wait_bounded(smem_u32(&bars[NS + s]), (uint32_t)(((k / NS) - 1) & 1),
                                            a.wait_ns);
                if (!__shfl_sync(0xffffffffu, got, 0)) {
                    ok = false;
                    break;
                }
            }
            if (lane < W) {
                smeta[(s * W + lane) * 2] = make_float4(dcx, dcy, dcz, ej.w);
                smeta[(s * W + lane) * 2 + 1] = make_float4(edx, edy, edz, near ? 1.f : 0.f);
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();  // the other lanes' metadata before the release-arrive
                const uint32_t full = smem_u32(&bars[s]);
                mbar_arrive_expect_tx(full, BYTES_J);
                const float4 *src = EXP ? a.fdup + gjt * 4 * T : a.jdup + gjt * 2 * T;
                bulk_g2s(smem_u32(sj + (size_t)s * V * T), src, BYTES_J, full);
            }
            // next unit
            if (++jt == d.ntile) {
                jt = 0;
                reload = true;
                if (++blk * W == d.ntile) {
                    blk = 0;
                    if (++sidx < a.nsims) d = a.sims[sidx];
                }
            }
        }
        if (lane == 0) {
            if (!ok) atomicExch(a.err, (int)STEPS_ETIMEOUT);
            // drain: every copy this warp issued must land before the CTA may exit
            const int64_t first = k > NS ? k - NS : 0;
            for (int64_t q = first; q < k; ++q)
                if (!mbar_wait_bounded(smem_u32(&bars[q % NS]), (uint32_t)((q / NS) & 1), kDrainNs))
                    atomicExch(a.err, (int)STEPS_ETIMEOUT);
        }
        if (a.stats) {
            for (int o = 16; o > 0; o >>= 1) n_near += __shfl_xor_sync(0xffffffffu, n_near, o);
            if (lane == 0) {
                atomicAdd(&a.stats[0], n_near);
                atomicAdd(&a.stats[1], (unsigned long long)(count * W));
            }
        }
        return;
    }

    // ---------------- compute warps ----------------
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    float4 *myipos = sipos + warp * T;
    const int tid = warp * 32 + lane;
    int64_t u = u0;
    int64_t k = 0;
    int seg = 0;
    int sidx = sim_of_unit(a.sims, a.nsims, u0);
    SimDesc d = a.sims[sidx];
    int64_t blk = (u0 - d.unit_off) / d.ntile;
    while (u < u1) {
        const int64_t seg_end = min(u1, d.unit_off + (blk + 1) * d.ntile);
        const int64_t ibase = (d.tile_off + blk * W + warp) * T + lane * KI;
        // stash this lane's target offsets in shared memory (read again per tile)
        __syncwarp();
#pragma unroll
        for (int t = 0; t < KI; ++t) {
            const float4 p = a.jdup[2 * (ibase + t)];
            const float4 pz = a.jdup[2 * (ibase + t) + 1];
            myipos[lane * KI + t] = make_float4(p.x, p.z, pz.x, 0.f);
        }
        float2 hx[NPAIR], hy[NPAIR], hz[NPAIR];     // running sums
        float2 cx_[NPAIR], cy_[NPAIR], cz_[NPAIR];  // Kahan terms (negated), COMP only
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            hx[q] = hy[q] = hz[q] = make_float2(0.f, 0.f);
            cx_[q] = cy_[q] = cz_[q] = make_float2(0.f, 0.f);
            if (SMK) {
#pragma unroll
                for (int c = 0; c < 6; ++c) skah[(c * NPAIR + q) * 32 * W + tid] = make_float2(0.f, 0.f);
            }
        }

        for (; u < seg_end; ++u, ++k) {
            const int s = (int)(k % NS);
            if (!mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((k / NS) & 1), a.wait_ns)) {
                if (lane == 0) atomicExch(a.err, (int)STEPS_ETIMEOUT);
                return;
            }
            const float4 m0 = smeta[(s * W + warp) * 2];
            const float4 m1 = smeta[(s * W + warp) * 2 + 1];
            if (EXP && m1.w == 0.f) {
                far_tile_expansion<KI, T, FOLD, UNR, SMK, W>(sj + (size_t)s * V * T, m0, m1, myipos, lane, tid,
                                                              skah, hx, hy, hz, cx_, cy_, cz_);
            } else if (!EXP && m1.w == 0.f) {
                // Far tile pair.  xs = fl(o_i + dc) loses xs_lo = (o_i + c_I - c_J) - xs,
                // and that loss is the same for every j of the tile: left alone it would
                // act as a coherent shift of the target.  Undo it to first order with
                // the tile's monopole tidal tensor, p -= M (xs_lo/R^3 - 3 D (D.xs_lo)/R^5),
                // D = c_J - x_i ~ -xs.  Fast2Sum (|dc| >= |o_i| off the near field)
                // gives the rounding error of xs; the producer split dc exactly.
                float2 nx[NPAIR], ny[NPAIR], nz[NPAIR];
                float2 px[NPAIR], py[NPAIR], pz[NPAIR];
                {
                    const float2 dcx2 = make_float2(m0.x, m0.x), dcy2 = make_float2(m0.y, m0.y),
                                 dcz2 = make_float2(m0.z, m0.z);
                    const float2 edx2 = make_float2(m1.x, m1.x), edy2 = make_float2(m1.y, m1.y),
                                 edz2 = make_float2(m1.z, m1.z);
                    const float2 ndx = make_float2(-m0.x, -m0.x), ndy = make_float2(-m0.y, -m0.y),
                                 ndz = make_float2(-m0.z, -m0.z);
                    const float2 M2 = make_float2(m0.w, m0.w);
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        const float4 i0 = myipos[lane * KI + 2 * q];
                        const float4 i1 = myipos[lane * KI + 2 * q + 1];
                        const float2 xi = make_float2(i0.x, i1.x), yi = make_float2(i0.y, i1.y),
                                     zi = make_float2(i0.z, i1.z);
                        nx[q] = __ffma2_rn(xi, neg1, ndx);
                        ny[q] = __ffma2_rn(yi, neg1, ndy);
                        nz[q] = __ffma2_rn(zi, neg1, ndz);
                        const float2 lx = __fadd2_rn(__fadd2_rn(xi, __fadd2_rn(nx[q], dcx2)), edx2);
                        const float2 ly = __fadd2_rn(__fadd2_rn(yi, __fadd2_rn(ny[q], dcy2)), edy2);
                        const float2 lz = __fadd2_rn(__fadd2_rn(zi, __fadd2_rn(nz[q], dcz2)), edz2);
                        float2 R2 = __fmul2_rn(nx[q], nx[q]);
                        R2 = __ffma2_rn(ny[q], ny[q], R2);
                        R2 = __ffma2_rn(nz[q], nz[q], R2);
                        const float2 Ri = make_float2(rsqrt_approx(R2.x), rsqrt_approx(R2.y));
                        const float2 Ri2 = __fmul2_rn(Ri, Ri);
                        const float2 k1 = __fmul2_rn(__fmul2_rn(M2, Ri), Ri2);
                        float2 proj = __fmul2_rn(nx[q], lx);
                        proj = __ffma2_rn(ny[q], ly, proj);
                        proj = __ffma2_rn(nz[q], lz, proj);
                        const float2 k2 =
                            __fmul2_rn(__fmul2_rn(make_float2(3.f, 3.f), k1), __fmul2_rn(proj, Ri2));
                        const float2 nk1 = __fmul2_rn(k1, neg1);
                        const float2 cxq = __ffma2_rn(k2, nx[q], __fmul2_rn(nk1, lx));
                        const float2 cyq = __ffma2_rn(k2, ny[q], __fmul2_rn(nk1, ly));
                        const float2 czq = __ffma2_rn(k2, nz[q], __fmul2_rn(nk1, lz));
                        if (COMP) {
                            px[q] = cxq;
                            py[q] = cyq;
                            pz[q] = czq;
                        } else {
                            px[q] = __fadd2_rn(hx[q], cxq);
                            py[q] = __fadd2_rn(hy[q], cyq);
                            pz[q] = __fadd2_rn(hz[q], czq);
                        }
                    }
                }
                const float4 *S = sj + (size_t)s * V * T;
#pragma unroll 1
                for (int j0 = 0; j0 < T; j0 += FOLD) {
#pragma unroll UNR
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
                    if (SMK) {
#pragma unroll
                        for (int q = 0; q < NPAIR; ++q) {
                            float2 *K = skah + q * 32 * W + tid;
                            constexpr int CS = NPAIR * 32 * W;  // component stride
                            float2 h0 = K[0], h1 = K[CS], h2 = K[2 * CS];
                            float2 c0 = K[3 * CS], c1 = K[4 * CS], c2 = K[5 * CS];
                            kahan2(h0, c0, px[q]);
                            kahan2(h1, c1, py[q]);
                            kahan2(h2, c2, pz[q]);
                            K[0] = h0;
                            K[CS] = h1;
                            K[2 * CS] = h2;
                            K[3 * CS] = c0;
                            K[4 * CS] = c1;
                            K[5 * CS] = c2;
                            px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
                        }
                    } else if (COMP) {
#pragma unroll
                        for (int q = 0; q < NPAIR; ++q) {
                            kahan2(hx[q], cx_[q], px[q]);
                            kahan2(hy[q], cy_[q], py[q]);
                            kahan2(hz[q], cz_[q], pz[q]);
                            px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
                        }
                    }
                }
                if (!COMP) {
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        hx[q] = px[q];
                        hy[q] = py[q];
                        hz[q] = pz[q];
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
            if (SMK) {
                const float2 *K = skah + q * 32 * W + tid;
                constexpr int CS = NPAIR * 32 * W;
                hx[q] = K[0];
                hy[q] = K[CS];
                hz[q] = K[2 * CS];
                cx_[q] = K[3 * CS];
                cy_[q] = K[4 * CS];
                cz_[q] = K[5 * CS];
            }
            P[0 * B_I + loc + 2 * q] = (double)hx[q].x + (double)cx_[q].x;
            P[0 * B_I + loc + 2 * q + 1] = (double)hx[q].y + (double)cx_[q].y;
            P[1 * B_I + loc + 2 * q] = (double)hy[q].x + (double)cy_[q].x;
            P[1 * B_I + loc + 2 * q + 1] = (double)hy[q].y + (double)cy_[q].y;
            P[2 * B_I + loc + 2 * q] = (double)hz[q].x + (double)cz_[q].x;
            P[2 * B_I + loc + 2 * q + 1] = (double)hz[q].y + (double)cz_[q].y;
        }
        ++seg;
        if (++blk * W == d.ntile) {
            blk = 0;
            if (++sidx < a.nsims) d = a.sims[sidx];
        }
    }
}

// Index of the first set bit >= pos in a bitmap row of `words` words, or -1.
// Warp-cooperative (32 words per probe); every lane returns the same value.
__device__ __forceinline__ int64_t next_near(const uint32_t *__restrict__ row, int64_t words,
                                             int64_t pos, int lane) {
    for (int64_t w0 = pos >> 5; w0 < words; w0 += 32) {
        const int64_t wi = w0 + lane;
        uint32_t v = (wi < words) ? row[wi] : 0u;
        if (wi == (pos >> 5)) v &= ~0u << (pos & 31);
        const unsigned any = __ballot_sync(0xffffffffu, v != 0u);
        if (any) {
            const int l = __ffs(any) - 1;
            const uint32_t vv = __shfl_sync(0xffffffffu, v, l);
            return (w0 + l) * 32 + (__ffs(vv) - 1);
        }
    }
    return -1;
}

constexpr int kNearWarps = 4;   // warps per CTA of the near-field kernel
constexpr int kNearChunk = 32;  // near tiles per work item (raised on device if needed)
// Near-field sources per compensated fold.  Neighbouring tiles contribute
// nearly parallel pair forces whose FP32 partial sums grow coherently; the
// rounding error of such a sum grows with its length, so the near field folds
// more often than the far field (it is a small share of the work).
constexpr int kNearFold = 8;

// Rank-th set bit (0-based) of a bitmap row, or -1; warp-cooperative.
__device__ __forceinline__ int64_t select_near(const uint32_t *__restrict__ row, int64_t words,
                                               int64_t rank, int lane) {
    int64_t seen = 0;
    for (int64_t w0 = 0; w0 < words; w0 += 32) {
        const int64_t wi = w0 + lane;
        const uint32_t v = (wi < words) ? row[wi] : 0u;
        int c = __popc(v), incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (seen + total > rank) {
            const unsigned hit = __ballot_sync(0xffffffffu, seen + incl > rank);
            const int l = __ffs(hit) - 1;
            uint32_t vv = __shfl_sync(0xffffffffu, v, l);
            int r = (int)(rank - seen - (__shfl_sync(0xffffffffu, incl, l) - __popc(vv)));
            for (; r > 0; --r) vv &= vv - 1;
            return (w0 + l) * 32 + (__ffs(vv) - 1);
        }
        seen += total;
    }
    return -1;
}

// Per target tile: number of near source tiles (one warp per row).
__global__ void near_count_kernel(const uint32_t *__restrict__ bits, const SimDesc *__restrict__ sims,
                                  int nsims, int64_t ntile, int *__restrict__ cnt) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= ntile) return;
    const SimDesc d = sims[sim_of_tile(sims, nsims, row)];
    const uint32_t *r = bits + d.bits_off + (row - d.tile_off) * d.words;
    int c = 0;
    for (int64_t w = lane; w < d.words; w += 32) c += __popc(r[w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[row] = c;
}

// Work items: row r contributes halves x ceil(cnt[r] / chunk) items (halves:
// the parts of the target tile one warp takes at a time); item_off is the
// exclusive scan.  chunk starts at kNearChunk and grows if the item buffer
// (cap items) would overflow.  meta = {chunk, items, work counter}.  One CTA.
__global__ void near_scan_kernel(const int *__restrict__ cnt, int64_t ntile, int64_t cap, int halves,
                                 int64_t *__restrict__ item_off, int64_t *__restrict__ meta) {
    __shared__ int64_t part[1024];
    __shared__ int64_t s_chunk;
    const int t = threadIdx.x;
    const int64_t per = (ntile + blockDim.x - 1) / blockDim.x;
    const int64_t r0 = t * per, r1 = min(ntile, r0 + per);
    int64_t tot = 0;
    for (int64_t r = r0; r < r1; ++r) tot += cnt[r];
    part[t] = tot;
    __syncthreads();
    if (t == 0) {
        int64_t all = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) all += part[k];
        int64_t chunk = kNearChunk;
        while (halves * (ntile + (all + chunk - 1) / chunk) > cap) chunk *= 2;
        s_chunk = chunk;
    }
    __syncthreads();
    const int64_t chunk = s_chunk;
    int64_t items = 0;
    for (int64_t r = r0; r < r1; ++r) items += halves * ((cnt[r] + chunk - 1) / chunk);
    __syncthreads();
    part[t] = items;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const int64_t v = part[k];
            part[k] = run;
            run += v;
        }
        meta[0] = chunk;
        meta[1] = run;
        meta[2] = 0;
        item_off[ntile] = run;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t r = r0; r < r1; ++r) {
        item_off[r] = run;
        run += halves * ((cnt[r] + chunk - 1) / chunk);
    }
}

// Near field of the pair term.  Work items are chunks of the near tiles of one
// target tile (row of the bitmap); persistent warps claim items from a
// counter, so rows with many near tiles spread over many warps.  Each item
// writes its own partial sums (item_part[item][c][T]), which the fixup adds
// in item order: deterministic.  Within an item the j tiles are
// double-buffered with TMA bulk copies.  The separation carries the FP32
// residuals of both offsets and the exact rounding errors of c_I - c_J and
// o_i + (c_I - c_J): d to ~1 ulp of |d| however large the tiles are.  Pairs
// are summed in packed FP32x2 on the Newtonian branch; where some lane of the
// warp meets a pair inside h_i + h_j the full spline of Eq. 4 is taken for
// that source.  Self pairs (d == 0 exactly) contribute nothing.
// NB source buffers per warp: 2 (the next tile's copy overlaps this tile's
// terms) up to 128-particle tiles; 256-particle tiles take 1 so that three
// CTAs fit on an SM (other warps cover the copy latency).
template <int KI>
constexpr int near_buffers() { return KI >= 8 ? 1 : 2; }
// Targets per lane in one work item: a 256-particle tile is taken in two
// halves of 128 targets (separate items), which keeps the register footprint
// of the 128-particle kernel.
template <int KI>
constexpr int near_ti() { return KI == 8 ? 4 : KI; }

template <int KI, bool COMP, int FOLD>
__global__ void __launch_bounds__(32 * kNearWarps) near_f32_kernel(const ForceArgs a) {
    constexpr int T = 32 * KI;
    constexpr int TI = near_ti<KI>();
    constexpr int H = KI / TI;      // items per (row, chunk)
    constexpr int NPAIR = TI / 2;
    constexpr int NB = near_buffers<KI>();
    constexpr uint32_t BYTES = T * 64u;  // jdup + rdup of one tile
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float4 *buf = reinterpret_cast<float4 *>(smem) + (size_t)warp * NB * 4 * T;  // [NB][jdup 2T | rdup 2T]
    uint64_t *bars =
        reinterpret_cast<uint64_t *>(reinterpret_cast<float4 *>(smem) + kNearWarps * NB * 4 * T) + 2 * warp;
    if (lane == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t chunk = a.near_meta[0];
    const int64_t items = a.near_meta[1];
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(&a.near_meta[2]);
    int64_t uses[2] = {0, 0};  // completed uses of each buffer (phase parity)
    auto issue = [&](int64_t jt, int b) {
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t bar = smem_u32(&bars[b]);
            float4 *dst = buf + (size_t)b * 4 * T;
            mbar_arrive_expect_tx(bar, BYTES);
            bulk_g2s(smem_u32(dst), a.jdup + jt * 2 * T, T * 32u, bar);
            bulk_g2s(smem_u32(dst + 2 * T), a.rdup + jt * 2 * T, T * 32u, bar);
        }
    };
    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = (int64_t)atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= items) break;
        // row = last r with item_off[r] <= item
        int64_t lo = 0, hi_r = a.ntile;  // item_off[lo] <= item < item_off[hi_r]
        while (hi_r - lo > 1) {
            const int64_t mid = (lo + hi_r) >> 1;
            if (a.item_off[mid] <= item) lo = mid; else hi_r = mid;
        }
        const int64_t itile = lo;
        const int half = (int)((item - a.item_off[itile]) % H);
        const int64_t first = ((item - a.item_off[itile]) / H) * chunk;
        const int64_t last = min((int64_t)a.near_cnt[itile], first + chunk);
        const SimDesc d = a.sims[sim_of_tile(a.sims, a.nsims, itile)];
        const uint32_t *row = a.nearbits + d.bits_off + (itile - d.tile_off) * d.words;

        const float4 ci = a.tbox_c[itile];
        const float4 ei = a.tbox_e[itile];
        const int64_t ibase = itile * T + half * 32 * TI + lane * TI;
        float2 xi[NPAIR], yi[NPAIR], zi[NPAIR], rxi[NPAIR], ryi[NPAIR], rzi[NPAIR];
        const float4 *RI = a.rdup + 2 * ibase;  // this lane's targets: residuals and h
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const float4 p0 = a.jdup[2 * (ibase + 2 * q)], p0z = a.jdup[2 * (ibase + 2 * q) + 1];
            const float4 p1 = a.jdup[2 * (ibase + 2 * q + 1)], p1z = a.jdup[2 * (ibase + 2 * q + 1) + 1];
            const float4 r0 = a.rdup[2 * (ibase + 2 * q)], r0z = a.rdup[2 * (ibase + 2 * q) + 1];
            const float4 r1 = a.rdup[2 * (ibase + 2 * q + 1)], r1z = a.rdup[2 * (ibase + 2 * q + 1) + 1];
            xi[q] = make_float2(p0.x, p1.x);
            yi[q] = make_float2(p0.z, p1.z);
            zi[q] = make_float2(p0z.x, p1z.x);
            rxi[q] = make_float2(r0.x, r1.x);
            ryi[q] = make_float2(r0.z, r1.z);
            rzi[q] = make_float2(r0z.x, r1z.x);
        }
        float2 hx[NPAIR], hy[NPAIR], hz[NPAIR], cx_[NPAIR], cy_[NPAIR], cz_[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            hx[q] = hy[q] = hz[q] = make_float2(0.f, 0.f);
            cx_[q] = cy_[q] = cz_[q] = make_float2(0.f, 0.f);
        }
        int64_t jt = select_near(row, d.words, first, lane);
        int b = 0;
        if (jt >= 0) issue(d.tile_off + jt, b);
        for (int64_t rk = first; rk < last && jt >= 0; ++rk) {
            const int64_t jn = (rk + 1 < last) ? next_near(row, d.words, jt + 1, lane) : -1;
            if (NB == 2 && jn >= 0) issue(d.tile_off + jn, b ^ 1);
            bool got = true;
            if (lane == 0) got = mbar_wait_bounded(smem_u32(&bars[b]), (uint32_t)(uses[b] & 1), a.wait_ns);
            if (!__shfl_sync(0xffffffffu, got, 0)) {
                if (lane == 0) {
                    atomicExch(a.err, (int)STEPS_ETIMEOUT);
                    // drain the copies still in flight before the warp exits
                    mbar_wait_bounded(smem_u32(&bars[b]), (uint32_t)(uses[b] & 1), kDrainNs);
                    if (NB == 2 && jn >= 0)
                        mbar_wait_bounded(smem_u32(&bars[b ^ 1]), (uint32_t)(uses[b ^ 1] & 1), kDrainNs);
                }
                return;
            }
            uses[b] += 1;
            const float4 *S = buf + (size_t)b * 4 * T;  // jdup tile
            const float4 *Rr = S + 2 * T;               // rdup tile
            const float4 cj = a.tbox_c[d.tile_off + jt];
            float edx, edy, edz;
            const float dcx = two_diff(ci.x, cj.x, edx);
            const float dcy = two_diff(ci.y, cj.y, edy);
            const float dcz = two_diff(ci.z, cj.z, edz);
            // -(xs), xs = fl(o_i + dc), and -(r_i + err(dc) + err(xs)), per target pair
            float2 nxs[NPAIR], nys[NPAIR], nzs[NPAIR], nrx[NPAIR], nry[NPAIR], nrz[NPAIR];
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                float e0, e1;
                nxs[q].x = -two_sum(xi[q].x, dcx, e0);
                nxs[q].y = -two_sum(xi[q].y, dcx, e1);
                nrx[q] = make_float2(-((rxi[q].x + edx) + e0), -((rxi[q].y + edx) + e1));
                nys[q].x = -two_sum(yi[q].x, dcy, e0);
                nys[q].y = -two_sum(yi[q].y, dcy, e1);
                nry[q] = make_float2(-((ryi[q].x + edy) + e0), -((ryi[q].y + edy) + e1));
                nzs[q].x = -two_sum(zi[q].x, dcz, e0);
                nzs[q].y = -two_sum(zi[q].y, dcz, e1);
                nrz[q] = make_float2(-((rzi[q].x + edz) + e0), -((rzi[q].y + edz) + e1));
            }
            // Can any pair of the two tiles lie inside h_i + h_j?  (the softening test of
            // tile_pair_near; the tile itself always can, it holds the self pairs)
            const float4 ej = a.tbox_e[d.tile_off + jt];
            bool soft = d.tile_off + jt == itile;
            {
                const float up = 1.0f + 0x1p-18f, dn = 1.0f - 0x1p-18f;
                const float gx = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcx), dn), __fmul_rn(__fadd_rn(ei.x, ej.x), up)));
                const float gy = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcy), dn), __fmul_rn(__fadd_rn(ei.y, ej.y), up)));
                const float gz = fmaxf(0.f, __fsub_rn(__fmul_rn(fabsf(dcz), dn), __fmul_rn(__fadd_rn(ei.z, ej.z), up)));
                const float gap2 = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
                const float hs = __fmul_rn(__fadd_rn(ci.w, cj.w), up);
                soft = soft || gap2 <= __fmul_rn(hs, hs);
            }
            // with sub-block masks only the near source halves of this target
            // half (the far kernel took the others)
            int j_begin = 0, j_end = T;
            if (KI == 8 && a.submask) {
                const int mk = a.submask[(d.bits_off + (itile - d.tile_off) * d.words) * 32 + jt] >> (2 * half);
                j_begin = (mk & 1) ? 0 : T / 2;
                j_end = (mk & 2) ? T : T / 2;
            }
            if (j_begin < j_end) {
                if (soft) {
                    // (h_i + the source tile's largest h)^2: at least (h_i + h_j)^2 for
                    // every source (rounding is monotone, the tile's h is rounded up)
                    float2 hT2[NPAIR];
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        const float h0 = __fadd_rn(RI[2 * (2 * q) + 1].z, cj.w);
                        const float h1 = __fadd_rn(RI[2 * (2 * q + 1) + 1].z, cj.w);
                        hT2[q] = make_float2(__fmul_rn(h0, h0), __fmul_rn(h1, h1));
                    }
                    near_tile_terms<TI, COMP, FOLD, true, T>(S, Rr, nxs, nys, nzs, nrx, nry, nrz, hT2, RI, hx, hy,
                                                          hz, cx_, cy_, cz_, j_begin, j_end);
                } else {
                    const float2 none[NPAIR] = {};
                    near_tile_terms<TI, COMP, FOLD, false, T>(S, Rr, nxs, nys, nzs, nrx, nry, nrz, none, RI, hx,
                                                           hy, hz, cx_, cy_, cz_, j_begin, j_end);
                }
            }
            __syncwarp();  // every lane is done with buffer b before it is refilled
            jt = jn;
            if (NB == 2)
                b ^= 1;
            else if (jn >= 0)
                issue(d.tile_off + jn, b);
        }
        double *P = a.item_part + (size_t)item * 3 * T;
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int li = half * 32 * TI + lane * TI + 2 * q + e;
                P[li] = (double)(e ? hx[q].y : hx[q].x) + (double)(e ? cx_[q].y : cx_[q].x);
                P[T + li] = (double)(e ? hy[q].y : hy[q].x) + (double)(e ? cy_[q].y : cy_[q].x);
                P[2 * T + li] = (double)(e ? hz[q].y : hz[q].x) + (double)(e ? cz_[q].y : cz_[q].x);
            }
        }
        // the other halves of the tile are another item's: zero here
#pragma unroll
        for (int hh = 0; hh < H; ++hh) {
            if (hh == half) continue;
#pragma unroll
            for (int t = 0; t < TI; ++t) {
                const int li = hh * 32 * TI + lane * TI + t;
                P[li] = 0.0;
                P[T + li] = 0.0;
                P[2 * T + li] = 0.0;
            }
        }
    }
}

__device__ __forceinline__ int64_t cta_start(int64_t c, int64_t units, int64_t G) {
    return c * units / G;
}

// Sum the per-CTA far-field partials of each target in CTA order, then its
// near-field work items in item order; apply G (sorted order, all systems).
__global__ void fixup_kernel(const double *__restrict__ partial, const double *__restrict__ item_part,
                             const int64_t *__restrict__ item_off, const SimDesc *__restrict__ sims,
                             int nsims, int T, int W, int64_t n, int64_t units, int64_t G, int smax,
                             double Gc, double *__restrict__ ax, double *__restrict__ ay,
                             double *__restrict__ az) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int B_I = W * T;
    const int64_t row = p / T;
    const SimDesc d = sims[sim_of_tile(sims, nsims, row)];
    const int64_t blk = (row - d.tile_off) / W;
    const int loc = (int)(p - (d.tile_off + blk * W) * T);
    const int64_t ufirst = d.unit_off + blk * d.ntile;
    const int64_t ulast = ufirst + d.ntile - 1;
    const int64_t gblk = d.blk_off + blk;
    auto cta_of = [&](int64_t uu) {
        int64_t c = uu * G / units;
        while (c + 1 < G && cta_start(c + 1, units, G) <= uu) ++c;
        while (c > 0 && cta_start(c, units, G) > uu) --c;
        return c;
    };
    double sx = 0.0, sy = 0.0, sz = 0.0;
    {
        const int li = (int)(p - row * T);
        for (int64_t it = item_off[row]; it < item_off[row + 1]; ++it) {
            const double *Q = item_part + (size_t)it * 3 * T;
            sx += Q[li];
            sy += Q[T + li];
            sz += Q[2 * T + li];
        }
    }
    const int64_t clo = cta_of(ufirst), chi = cta_of(ulast);
    for (int64_t c = clo; c <= chi; ++c) {
        const int64_t us = cta_start(c, units, G);
        const SimDesc dc = sims[sim_of_unit(sims, nsims, us)];
        const int64_t seg = gblk - (dc.blk_off + (us - dc.unit_off) / dc.ntile);
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

template <int KI, int W, int NS, bool SMK, bool EXP>
constexpr size_t smem_of() {
    return (size_t)NS * (32 * KI) * (EXP ? 64 : 32) + (size_t)NS * W * 32 + (size_t)W * (32 * KI) * 16 +
           (SMK ? (size_t)6 * (KI / 2) * 32 * W * 8 : 0) + 2 * NS * sizeof(uint64_t);
}

template <int KI>
constexpr size_t near_smem_of() {
    return (size_t)kNearWarps * near_buffers<KI>() * (32 * KI) * 64 + 2 * kNearWarps * sizeof(uint64_t);
}

struct VariantImpl {
    Variant v;
    KernelFn fn;       // far field (stream-K, TMA pipeline)
    KernelFn near_fn;  // near field (balanced work items)
    size_t smem;
    size_t near_smem;
};

#define STEPS_VARIANT(KI, W, NS, COMP, FOLD, MINB, UNR, KSM, EXP, NAME)                        \
    {{KI, W, NS, COMP, NAME, EXP ? 1 : 0},                                                     \
     force_f32_kernel<KI, W, NS, COMP, FOLD, MINB, UNR, KSM, EXP>, near_f32_kernel<KI, COMP, kNearFold>, \
     smem_of<KI, W, NS, COMP && KSM, EXP>(), near_smem_of<KI>()}

// Compensated variants first (expansion form, then explicit separation), then
// the naive-sum comparison variants.  The autotuner times every variant of the
// requested summation mode; systems whose staging has no expansion layout
// only use the explicit form.
const VariantImpl kVariants[] = {
    STEPS_VARIANT(4, 4, 4, true, 32, 3, 8, false, true, "exp_ki4_w4_u8"),
    STEPS_VARIANT(6, 4, 4, true, 32, 2, 4, false, true, "exp_ki6_w4_u4"),
    STEPS_VARIANT(4, 4, 4, true, 32, 3, 4, false, false, "comp_ki4_w4_u4"),
    STEPS_VARIANT(4, 8, 4, true, 32, 2, 2, false, false, "comp_ki4_w8_u2"),
    STEPS_VARIANT(6, 8, 4, true, 32, 2, 2, false, false, "comp_ki6_w8_u2"),
    STEPS_VARIANT(2, 8, 4, true, 32, 4, 4, false, false, "comp_ki2_w8_u4"),
    STEPS_VARIANT(4, 4, 4, false, 32, 3, 4, false, false, "naive_ki4_w4_u4"),
    STEPS_VARIANT(4, 8, 4, false, 32, 2, 2, false, false, "naive_ki4_w8_u2"),
    STEPS_VARIANT(2, 8, 4, false, 32, 4, 4, false, false, "naive_ki2_w8_u4"),
    // symmetric far field (force_sym.cu): 256-particle tiles, 4 compute warps
    {{8, 4, 4, true, "sym_ki8_w4", 2, 3}, nullptr, near_f32_kernel<8, true, kNearFold>, 0, near_smem_of<8>()},
    {{4, 4, 4, true, "sym_ki4_w4", 2, 4}, nullptr, near_f32_kernel<4, true, kNearFold>, 0, near_smem_of<4>()},
    {{8, 4, 4, true, "sym_ki8s_w4", 2, 3, true}, nullptr, near_f32_kernel<8, true, kNearFold>, 0,
     near_smem_of<8>()},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int num_variants() { return kNumVariants; }
const Variant &variant(int k) { return kVariants[k].v; }
size_t force_smem_bytes(int k) {
    return kVariants[k].v.form == 2 ? sym_smem_bytes(kVariants[k].v.KI, kVariants[k].v.W) : kVariants[k].smem;
}

ForcePlan plan_force_multi(int k, int num_sms, SimDesc *descs, int nsims, const SimDesc *dev_sims,
                           int64_t *bits_words) {
    const VariantImpl &vi = kVariants[k];
    const int W = vi.v.W;
    ForcePlan p;
    p.variant = k;
    p.B_I = W * 32 * vi.v.KI;
    p.sims = dev_sims;
    p.nsims = nsims;
    int64_t units = 0, blocks = 0, bits = 0;
    const bool sym = vi.v.form == 2;
    std::vector<int64_t> starts;  // unit at which every target block starts
    for (int s = 0; s < nsims; ++s) {
        SimDesc &d = descs[s];
        d.unit_off = units;
        d.blk_off = blocks;
        d.words = (d.ntile + 31) / 32;
        d.bits_off = bits;

        if (!sym)
            for (int64_t b = 0; b < d.ntile / W; ++b) starts.push_back(units + b * d.ntile);
        units += sym ? sym_units(d.ntile, W) : (d.ntile / W) * d.ntile;
        blocks += d.ntile / W;
        bits += d.ntile * d.words;
    }
    if (bits_words) *bits_words = bits;
    p.mask_bytes = bits * 32;  // one byte per bit of the near bitmap
    p.niblk = blocks;
    p.units = units;
    cudaFuncSetAttribute(vi.near_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vi.near_smem);
    if (sym) {
        // persistent grid; every unit adds to fixed-point sums, no per-CTA partials
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * sym_blocks_per_sm(vi.v.KI, W, vi.v.ctas, vi.v.sub),
                                                                    units));
        p.grid = (int)grid;
        p.smax = 0;
        p.partial_elems = 0;
        return p;
    }
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
    // segments per CTA = target blocks its unit range touches
    int smax = 1;
    for (int64_t c = 0; c < grid; ++c) {
        const int64_t a0 = c * units / grid, a1 = (c + 1) * units / grid;
        const auto lo = std::upper_bound(starts.begin(), starts.end(), a0);
        const auto hi = std::lower_bound(starts.begin(), starts.end(), a1);
        const int segs = 1 + (int)std::max<int64_t>(0, hi - lo);
        smax = std::max(smax, segs);
    }
    p.smax = smax;
    p.partial_elems = (size_t)p.grid * p.smax * 3 * p.B_I;
    return p;
}

ForcePlan plan_force(const Staging &s, int k, int num_sms) {
    SimDesc d{};
    d.tile_off = 0;
    d.ntile = s.ntile;
    return plan_force_multi(k, num_sms, &d, 1, nullptr, nullptr);
}

cudaError_t launch_force_f32(const ForcePlan &p, const Staging &s, double *partial,
                             const NearScratch &nr, int *err, unsigned long long *stats,
                             float alpha, long long wait_ns, int num_sms, cudaStream_t st,
                             cudaEvent_t far_begin, cudaEvent_t far_end) {
    const VariantImpl &vi = kVariants[p.variant];
    ForceArgs a;
    a.jdup = s.jdup;
    a.rdup = s.rdup;
    a.fdup = s.fdup;
    a.tbox_c = s.tbox_c;
    a.tbox_e = s.tbox_e;
    a.partial = partial;
    a.item_part = nr.item_part;
    a.nearbits = nr.bits;
    a.submask = (vi.v.form == 2 && vi.v.KI == 8 && s.tbox_hc) ? nr.submask : nullptr;
    a.near_cnt = nr.cnt;
    a.item_off = nr.item_off;
    a.near_meta = nr.meta;
    a.sims = p.sims;
    a.nsims = p.nsims;
    a.err = err;
    a.stats = stats;
    a.ntile = s.ntile;
    a.units = p.units;
    a.smax = p.smax;
    a.alpha2 = alpha * alpha;
    a.wait_ns = wait_ns;
    cudaError_t e;
    if (vi.v.form == 2) {
        // classification pass (whole bitmap, fixed-point scales), then the symmetric far field
        if ((e = cudaMemsetAsync(nr.sym_acc, 0, sizeof(unsigned long long) * 3 * (size_t)s.np, st)) != cudaSuccess)
            return e;
        if ((e = launch_sym_classify(s, p, nr, alpha, stats, st)) != cudaSuccess) return e;
        if (far_begin && (e = cudaEventRecord(far_begin, st)) != cudaSuccess) return e;
        if ((e = launch_sym_far(s, p, nr, err, wait_ns, st)) != cudaSuccess) return e;
        if (far_end && (e = cudaEventRecord(far_end, st)) != cudaSuccess) return e;
    } else {
        e = cudaMemsetAsync(nr.bits, 0, sizeof(uint32_t) * (size_t)nr.bits_words, st);
        if (e != cudaSuccess) return e;
        if (far_begin && (e = cudaEventRecord(far_begin, st)) != cudaSuccess) return e;
        vi.fn<<<p.grid, (vi.v.W + 1) * 32, vi.smem, st>>>(a);
        if (far_end && (e = cudaEventRecord(far_end, st)) != cudaSuccess) return e;
    }
    near_count_kernel<<<(unsigned)((s.ntile * 32 + 255) / 256), 256, 0, st>>>(nr.bits, p.sims, p.nsims,
                                                                             s.ntile, nr.cnt);
    near_scan_kernel<<<1, 1024, 0, st>>>(nr.cnt, s.ntile, nr.cap_items, vi.v.KI == 8 ? 2 : 1,
                                         nr.item_off, nr.meta);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vi.near_fn, 32 * kNearWarps, vi.near_smem) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    vi.near_fn<<<(unsigned)(num_sms * per_sm), 32 * kNearWarps, vi.near_smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fixup(const ForcePlan &p, const Staging &s, const double *partial,
                         const NearScratch &nr, double G, double *ax, double *ay, double *az,
                         cudaStream_t st) {
    if (kVariants[p.variant].v.form == 2) return launch_sym_fixup(s, p, nr, G, ax, ay, az, st);
    const int tb = 256;
    const int64_t blocks = (s.n + tb - 1) / tb;
    fixup_kernel<<<(unsigned)blocks, tb, 0, st>>>(partial, nr.item_part, nr.item_off, p.sims, p.nsims, s.T,
                                                  kVariants[p.variant].v.W, s.n, p.units, p.grid, p.smax,
                                                  G, ax, ay, az);
    return cudaGetLastError();
}

}  // namespace steps

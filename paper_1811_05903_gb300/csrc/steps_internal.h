// Internal declarations shared by the libsteps translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/steps.h"

namespace steps {

// ---------------------------------------------------------------------------
// Error handling: thread-local last-error string, status helpers.
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
steps_status cuda_status(cudaError_t e, const char *what);
// Device allocation counted against the process-wide steps_set_memory_limit cap.
steps_status counted_malloc(void **p, size_t bytes);
void counted_free(void *p, size_t bytes);

#define STEPS_CUDA(call)                                                  \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::steps::cuda_status(_e, #call);    \
    } while (0)

#define STEPS_TRY(expr)                         \
    do {                                        \
        steps_status _s = (expr);               \
        if (_s != STEPS_OK) return _s;          \
    } while (0)

// ---------------------------------------------------------------------------
// Force-kernel variants (FP32 pair arithmetic).
//   KI   targets per thread (even; handled as KI/2 packed pairs)
//   W    compute warps per CTA (one extra producer warp issues the copies)
//   NS   shared-memory stages of j tiles
// A tile is T = 32*KI consecutive (sorted) particles sharing one FP32 centre;
// a warp owns one tile of targets, a CTA owns W tiles (B_I = W*T targets).
// ---------------------------------------------------------------------------
struct Variant {
    int KI, W, NS;
    bool comp;
    const char *name;
    // far-field arithmetic: 0 = explicit separation d = o_j - s (12 FP32 lane
    // operations per interaction), 1 = expansion of |o_j - s|^2 about the
    // source tile centre with the mass folded into the squared distance
    // (10 lane operations; reads Staging::fdup), 2 = symmetric: every far pair
    // of tiles (I < J) is evaluated once and its force is added to both
    // particles (explicit separation, 8 lane operations and half an MUFU per
    // interaction; reads Staging::sdup, accumulates in fixed point)
    int form;
    // symmetric kernel: CTAs of 4 warps per SM it is compiled for (3 for
    // 256-particle tiles: up to 168 registers per thread; 4 for 128: up to 128)
    int ctas = 0;
    // symmetric 256-particle tiles: classify 128 x 128 sub-blocks, so that only
    // the near sub-blocks of a tile pair go to the near-field kernel
    bool sub = false;
};

int num_variants();
const Variant &variant(int k);

// Device views used by the FP32 force path.
struct Staging {
    int64_t n = 0;        // real particles
    int64_t np = 0;       // padded to a multiple of B_I
    int T = 0;            // tile size (particles)
    int64_t ntile = 0;    // np / T
    float4 *jdup = nullptr;   // [2 np] (ox, ox, oy, oy), (oz, oz, m, m): FP32 offsets from the tile centre
    float4 *rdup = nullptr;   // [2 np] (rx, rx, ry, ry), (rz, rz, h, h): FP32 residual x - c - o, softening
    // [4 np] far-field expansion layout, or null when no expansion variant runs:
    // (ox, ox, oy, oy), (oz, oz, k, k), (2k ox, 2k ox, 2k oy, 2k oy), (2k oz, 2k oz, k |o|^2, k |o|^2)
    // with k = fl(m^(-2/3)); padding: o = 1e15, k = 1e10, 2k o = 0, k |o|^2 = +inf
    float4 *fdup = nullptr;
    // [2 np] symmetric-kernel layout, or null: per 32-particle chunk of a tile,
    // 32 x (ox, ox, oy, oy) then 32 x (oz, oz, m, m); padding: o = 1e15, m = 0
    float4 *sdup = nullptr;
    // device word for the largest |coordinate| (bit pattern of a non-negative
    // double), or null.  When set, tile centres are rounded to multiples of
    // 2^(e-22) with max|x| < 2^e, so that every difference of two centres is
    // exact in FP32.
    unsigned long long *qmax = nullptr;
    // positions and softenings are multiplied by pscale before staging (1 / L
    // in periodic mode: box units); with qmax the centre grid is at least
    // 2^(qemin - 22)
    double pscale = 1.0;
    int qemin = -1000;
    float4 *tbox_c = nullptr; // [ntile] (cx, cy, cz, hmax)
    float4 *tbox_e = nullptr; // [ntile] (ex, ey, ez, M) half extents (rounded up), tile mass
    // [2 ntile] the same for the two halves of every tile, or null (the
    // 256-particle symmetric variant classifies 128 x 128 sub-blocks)
    float4 *tbox_hc = nullptr;
    float4 *tbox_he = nullptr;
};

// One independent system inside the concatenated staging arrays.  A single
// simulation is a table of one; an ensemble concatenates its members, each
// padded to a whole number of target blocks (W tiles).
struct SimDesc {
    int64_t tile_off;  // first global tile of the system
    int64_t ntile;     // its tiles (a multiple of the block's W)
    int64_t unit_off;  // its first far-field unit (one-sided: (ntile / W) * ntile units; symmetric: sym_units)
    int64_t blk_off;   // its first target block in the global block order
    int64_t bits_off;  // first word of its near bitmap, [ntile][words]
    int64_t words;     // bitmap words per row, (ntile + 31) / 32
};

// Launch the staging kernel: FP64 sorted SoA -> FP32 tile-relative arrays.
// A particle with a negative softening is padding (ensembles).
void launch_stage(const Staging &s, const double *x, const double *y, const double *z,
                  const double *m, const double *h, cudaStream_t st);

// Near-field scratch: bitmap of near tile pairs, per-row counts, work items.
struct NearScratch {
    uint32_t *bits = nullptr;     // [ntile][(ntile + 31) / 32]
    int *cnt = nullptr;           // [ntile]
    int64_t *item_off = nullptr;  // [ntile + 1]
    int64_t *meta = nullptr;      // [3] {chunk, items, work counter}
    double *item_part = nullptr;  // [cap_items][3][T]
    int64_t cap_items = 0;
    int64_t bits_words = 0;       // words of `bits` in use (cleared per evaluation)
    // symmetric kernel (Variant::form == 2) only:
    unsigned long long *sym_acc = nullptr;  // [3][np] fixed-point far-field sums
    float *tscale = nullptr;                // [ntile] 2^(62 - E_t): FP32 value -> fixed point
    double *tinv = nullptr;                 // [ntile] 2^(E_t - 62)
    int *nonfinite = nullptr;               // set to 1 when a far-field partial is not finite
    unsigned long long *sym_next = nullptr; // chunk counter of the symmetric far kernel
    // per ordered tile pair, bit 2 hI + hJ: the sub-block (half hI of I, half hJ
    // of J) is near, laid out like the near bitmap with a byte per bit (row I
    // of a system at (bits_off + I words) 32), or null
    uint8_t *submask = nullptr;
    int64_t mask_bytes = 0;                 // bytes of submask in use
};

// Stream-K plan for one FP32 force evaluation over one or more systems.
struct ForcePlan {
    int variant = 0;
    int grid = 0;       // persistent CTAs
    int smax = 0;       // max segments (target blocks touched) per CTA
    int64_t niblk = 0;  // target blocks, all systems
    int64_t units = 0;  // tile pairs, all systems
    int B_I = 0;
    size_t partial_elems = 0;  // grid * smax * 3 * B_I doubles
    int64_t mask_bytes = 0;    // sub-block near masks of all systems (32 bytes per bitmap word)
    const SimDesc *sims = nullptr;  // device table
    int nsims = 1;
};

ForcePlan plan_force(const Staging &s, int variant, int num_sms);

// Symmetric far field (force_sym.cu).  Units are (target block b of W tiles,
// source tile J) with J > b W, per system; warp w of the block takes tile
// b W + w when it precedes J.
int64_t sym_units(int64_t ntile, int W);
size_t sym_smem_bytes(int KI, int W);
// ctas: the variant's Variant::ctas (which compiled kernel)
int sym_blocks_per_sm(int KI, int W, int ctas, bool sub);
// Near bitmap (all ordered tile pairs; each tile with itself is near),
// per-tile fixed-point scales from a bound on the far-field sums, near/all counts.
cudaError_t launch_sym_classify(const Staging &s, const ForcePlan &p, const NearScratch &nr, float alpha,
                                unsigned long long *stats, cudaStream_t st);
cudaError_t launch_sym_far(const Staging &s, const ForcePlan &p, const NearScratch &nr, int *err,
                           long long wait_ns, cudaStream_t st);
// acc = G (fixed-point far field + near-field items), sorted order.
cudaError_t launch_sym_fixup(const Staging &s, const ForcePlan &p, const NearScratch &nr, double G,
                             double *ax, double *ay, double *az, cudaStream_t st);
// Plan for several systems: descs is the host copy of the table (its unit_off,
// blk_off and bits_off are filled in here); dev_sims the device copy to use.
ForcePlan plan_force_multi(int variant, int num_sms, SimDesc *descs, int nsims,
                           const SimDesc *dev_sims, int64_t *bits_words);
size_t force_smem_bytes(int variant);
// alpha: tile pairs whose boxes are closer than alpha * (|c_I - c_J| + |e_I| + |e_J|)
// take the compensated near-field path.  stats (may be null) counts near/all tile pairs.
// Launches the far field and then the near-field work items.  One-sided
// variants: stream-K over all tile pairs, marking near pairs in nr.bits
// (cleared here); symmetric variants: the classification kernel (near bitmap,
// sub-block masks, fixed-point scales), then the far units in chunks from a
// global counter.  Then the near-field count, scan and item kernels.
// far_begin / far_end (may be null): events recorded on st around the far-field launch.
cudaError_t launch_force_f32(const ForcePlan &p, const Staging &s, double *partial,
                             const NearScratch &nr, int *err, unsigned long long *stats,
                             float alpha, long long wait_ns, int num_sms, cudaStream_t st,
                             cudaEvent_t far_begin = nullptr, cudaEvent_t far_end = nullptr);
cudaError_t launch_fixup(const ForcePlan &p, const Staging &s, const double *partial,
                         const NearScratch &nr, double G, double *ax, double *ay, double *az,
                         cudaStream_t st);

// Periodic pair term (Eq. 2 with Eq. 5).  The staging is in box units
// (Staging::pscale = 1 / L, tile centres on a grid of 2^-21 or coarser), so
// every image shift c_I - c_J - n is exact in FP32.
//
// Per-target FP32 kernel (periodic.cu): work items (target tile, chunk of
// source tiles) write FP64 partials item_part [ntile * nchunk][3][T]
// (nchunk = periodic_chunks(ntile, num_sms)), then a reduction applies G / L^2
// into ax, ay, az (sorted order).  It takes every image of the quasi-periodic
// sum and of the cut sum on staging without the symmetric layout; with the
// symmetric kernel (cut sum, 128-particle tiles) it takes only the images that
// may hold a softened pair ("residual" mode), and the reduction adds the
// symmetric kernel's fixed-point sums.
struct PeriodicArgs {
    const float4 *jdup, *rdup, *fdup, *tbox_c, *tbox_e;
    const double *x, *y, *z;  // FP64 sorted positions: decisions near the cut / half-box faces
    double *item_part;
    int64_t ntile, nchunk, n;
    double L;   // box length of x, y, z (FP64 decisions)
    double Ls;  // box length in staging units (1)
    int images;
    int residual;  // 1: only the images the symmetric kernel leaves out
    // residual mode: items are the entries of the soft partner lists (target
    // tile by soff, source tile slist[item]) when soff[ntile] <= cap_items,
    // else (target tile, chunk of source tiles) as in the full mode
    const int64_t *soff;
    const int *slist;
    int64_t cap_items;
};
// Scratch of the symmetric periodic kernel (periodic_sym.cu).
struct PeriodicSymScratch {
    unsigned long long *acc = nullptr;  // [3][np] fixed-point sums
    float *tscale = nullptr;            // [ntile] 2^(62 - E_t)
    double *tinv = nullptr;             // [ntile] 2^(E_t - 62)
    int64_t *off = nullptr;             // [npairs + 2] work-unit offsets of the tile pairs (I <= J), counter
    float2 *bnd = nullptr;              // [npairs] bound contributions (to I, to J)
    int *nonfinite = nullptr;
    // tiles sharing a softened image (the per-target kernel's work items)
    int *soft = nullptr;                // [npairs] softened images of the pair
    int64_t *soff = nullptr;            // [ntile + 1] per target tile, into slist
    int *slist = nullptr;               // [cap_items] source tiles
    int64_t cap_items = 0;              // list entries (and item partials) that fit
};
int64_t periodic_chunks(int64_t ntile, int num_sms);
// Largest item_part size (doubles) any tile size needs for np padded particles.
size_t periodic_part_elems(int64_t np, int num_sms);
// Tile pairs I <= J of ntile tiles, and the tile size the symmetric kernel needs.
int64_t periodic_sym_pairs(int64_t ntile);
int periodic_sym_tile();
// Symmetric kernel alone: fixed-point sums of every non-soft image of the cut
// sum (images 0) or the quasi-periodic sum (images 1) into ps.acc (box units,
// without G / L^2), scales into ps.tscale / ps.tinv.
cudaError_t launch_periodic_sym(const Staging &s, const double *x, const double *y, const double *z, double L,
                                int images, const PeriodicSymScratch &ps, int num_sms, cudaStream_t st);
// The whole FP32 periodic evaluation into ax, ay, az.  ps: symmetric scratch,
// or null for the per-target kernel alone.  far_begin / far_end (optional)
// bracket the symmetric kernel.
cudaError_t launch_periodic_f32(const Staging &s, const double *x, const double *y, const double *z, double L,
                                int images, double G, double *item_part, const PeriodicSymScratch *ps,
                                int num_sms, double *ax, double *ay, double *az, cudaStream_t st,
                                cudaEvent_t far_begin = nullptr, cudaEvent_t far_end = nullptr);
cudaError_t launch_periodic_f64(int64_t n, const double *x, const double *y, const double *z, const double *m,
                                const double *h, double G, double L, int images, double *ax, double *ay,
                                double *az, cudaStream_t st);

// FP64 comparison path: direct sum over sorted FP64 SoA, targets [i0, i1).
cudaError_t launch_force_f64(int64_t n, const double *x, const double *y, const double *z,
                             const double *m, const double *h, double G, int64_t i0, int64_t i1,
                             double *ax, double *ay, double *az, cudaStream_t st);
// FP64 pair term for a list of sorted target indices; out3 is [nt][3] in list order.
cudaError_t launch_force_f64_list(int64_t n, const double *x, const double *y, const double *z,
                                  const double *m, const double *h, double G, int64_t nt,
                                  const int64_t *idx, double *out3, cudaStream_t st);
// inv[perm[k]] = k, then out[t] = inv[caller[t]]; *bad |= 1 for an index outside [0, n).
cudaError_t launch_map_targets(int64_t n, const int64_t *perm, int64_t *inv, int64_t nt,
                               const int64_t *caller, int64_t *out, int *bad, cudaStream_t st);
// FP64 pair potential per particle, row[i] = sum_{j != i} G m_i m_j W(r_ij, h_i + h_j).
cudaError_t launch_potential_f64(int64_t n, const double *x, const double *y, const double *z,
                                 const double *m, const double *h, double G, double *row,
                                 cudaStream_t st);

// ---------------------------------------------------------------------------
// Spatial sort (Morton order of FP64 positions).
// ---------------------------------------------------------------------------
struct SortScratch {
    int64_t npow2 = 0;
    unsigned long long *keys = nullptr;
    unsigned int *vals = nullptr;
    double *bbox = nullptr;   // [6] min xyz, max xyz (morton_sort: [8 + 6 x 256], partials after the box)
    double *tmp = nullptr;    // [n] gather buffer
    int64_t *tmpi = nullptr;  // [n]
};
// Sorts (key, index) pairs; *launches receives the number of kernels issued.
cudaError_t morton_sort(int64_t n, const double *x, const double *y, const double *z,
                        SortScratch &s, cudaStream_t st, int *launches);
// Sort an ensemble by (system, Morton code within the system's own box);
// off[nsims + 1] are the systems' first indices, sim[p] the system of p, and
// padding (h < 0) sorts to the end of its system.
cudaError_t ensemble_sort(int nsims, const int64_t *off, int64_t np_total, const int *sim,
                          const double *x, const double *y, const double *z, const double *h,
                          SortScratch &s, cudaStream_t st, int *launches);
// out[k] = in[vals[k]] for k < n
cudaError_t gather_f64(int64_t n, const unsigned int *vals, const double *in, double *out,
                       cudaStream_t st);
cudaError_t gather_i64(int64_t n, const unsigned int *vals, const int64_t *in, int64_t *out,
                       cudaStream_t st);

// ---------------------------------------------------------------------------
// FP64 integrator on device.  Scalars live in device memory so that a whole
// step can be captured in a CUDA graph.
// ---------------------------------------------------------------------------
enum { SC_T = 0, SC_A = 1, SC_H = 2, SC_DT = 3, SC_STEP = 4, SC_RUN = 5, SC_COUNT = 8 };

struct Cosmo {
    double G, H0, Om, OL, Or, Ok;  // G is the pair term's constant: -G when gravity is reversed
    int comoving;
    int reversed;                  // 1: the background term of Eq. 8 changes sign too
    int periodic;                  // 1: Eq. 2 (no background term), positions wrapped into [0, box)
    double box;
};

cudaError_t launch_kick(int64_t n, const double *x, const double *y, const double *z, double *vx,
                        double *vy, double *vz, const double *ax, const double *ay,
                        const double *az, const double *sc, const Cosmo &c, cudaStream_t st);
// Drift and wrap into [0, box)^3 (periodic mode): x += v dt; x -= box floor(x / box).
cudaError_t launch_drift_wrap(int64_t n, double *x, double *y, double *z, const double *vx,
                              const double *vy, const double *vz, const double *sc, double box,
                              cudaStream_t st);
// x -= box floor(x / box) for k < 3 n interleaved or n SoA values.
cudaError_t launch_wrap(int64_t n, double *v, double box, cudaStream_t st);
cudaError_t launch_drift(int64_t n, double *x, double *y, double *z, const double *vx,
                         const double *vy, const double *vz, const double *sc, cudaStream_t st);
cudaError_t launch_rk4(double *sc, const Cosmo &c, cudaStream_t st);
cudaError_t launch_set_dt(double *sc, const double *dts, cudaStream_t st);
// Eq. 12: sc[SC_DT] = min(dt_max, min_i sqrt(2 (2.8 h_i) eps / |A_i|)), limited to
// t_end - sc[SC_T] when t_end is finite; part holds nblk doubles of scratch.
cudaError_t launch_timestep(int64_t n, const double *x, const double *y, const double *z,
                            const double *vx, const double *vy, const double *vz, const double *ax,
                            const double *ay, const double *az, const double *h, double *sc,
                            const Cosmo &c, double eps, double dt_max, double t_end, double *part,
                            int nblk, cudaStream_t st);

// Deterministic FP64 reductions: out[0] = sum w*v^2/2, out[1..3] = sum w*v
cudaError_t launch_kinetic(int64_t n, const double *vx, const double *vy, const double *vz,
                           const double *m, double *block_buf, int nblk, double *out,
                           cudaStream_t st);
cudaError_t launch_sum(int64_t n, const double *v, double *block_buf, int nblk, double *out,
                       cudaStream_t st);

// Scatter sorted-order FP64 SoA into caller order [n][3].
cudaError_t launch_scatter3(int64_t n, const int64_t *perm, const double *a, const double *b,
                            const double *c, double *out3, cudaStream_t st);
// Gather caller order [n][3] into sorted SoA through perm (sorted k <- caller perm[k]).
cudaError_t launch_gather3(int64_t n, const int64_t *perm, const double *in3, double *a, double *b,
                           double *c, cudaStream_t st);
cudaError_t launch_split3(int64_t n, const double *in3, double *a, double *b, double *c,
                          cudaStream_t st);
cudaError_t launch_iota(int64_t n, int64_t *perm, cudaStream_t st);
// Eq. 7 on device: h = cbrt(m / m_min) * h_min, with m_min reduced on device.
cudaError_t launch_softening(int64_t n, const double *m, double h_min, double *h, double *scratch,
                             cudaStream_t st);
// Input check: *flag |= 1 if a holds NaN/Inf, |= 2 if positive != 0 and some a[i] <= 0.
cudaError_t launch_check_finite(int64_t n, const double *a, int positive, int *flag,
                                cudaStream_t st);
// *flag = 1 if some a[i], b[i] or c[i], i < n, is NaN or Inf (the non-finite result check);
// with h given, slots with h[i] < 0 (padding) are skipped.
cudaError_t launch_check_finite3(int64_t n, const double *a, const double *b, const double *c, int *flag,
                                 cudaStream_t st, const double *h = nullptr);
cudaError_t launch_set_scalar(double *sc, int slot, double v, cudaStream_t st);

}  // namespace steps

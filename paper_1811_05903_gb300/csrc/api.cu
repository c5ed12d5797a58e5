// C ABI of libsteps: simulation contexts, force evaluation, the KDK step
// (Eq. 9-11) and diagnostics.  Host-side runtime only; all arithmetic of the
// method runs in the kernels of force_f32.cu, force_f64.cu, stage.cu and
// integrate.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "steps_internal.h"

namespace steps {

static thread_local char g_last_error[512] = "";
static size_t g_mem_limit = 0;  // process-wide cap on this library's device allocations (0: none)
static size_t g_mem_used = 0;
static std::mutex g_mem_mu;

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

steps_status cuda_status(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? STEPS_ENOMEM : STEPS_ECUDA;
}

steps_status counted_malloc(void **p, size_t bytes) {
    *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (g_mem_limit && g_mem_used + bytes > g_mem_limit) {
            set_error("device allocation of %zu bytes exceeds the library memory limit (%zu of %zu used)",
                      bytes, g_mem_used, g_mem_limit);
            return STEPS_ENOMEM;
        }
        g_mem_used += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        g_mem_used -= bytes;
        *p = nullptr;
        return cuda_status(e, "cudaMalloc");
    }
    return STEPS_OK;
}

void counted_free(void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_used -= bytes;
}

}  // namespace steps

using namespace steps;

struct steps_ctx {
    int64_t n = 0;
    steps_config cfg{};
    Cosmo cosmo{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;
    // FP64 master state, sorted order (SoA)
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *vx = nullptr, *vy = nullptr, *vz = nullptr;
    double *m = nullptr, *h = nullptr;
    double *ax = nullptr, *ay = nullptr, *az = nullptr;
    int64_t *perm = nullptr;  // sorted index -> caller index
    double *sc = nullptr;     // device scalars SC_*
    double *red = nullptr;    // reduction scratch
    int nred = 0;
    double *tmp3 = nullptr;   // [n][3] caller-order staging for boundary copies
    double *dts = nullptr;    // per-step dt for runs
    int dts_cap = 0;
    // FP32 staging
    Staging stg;
    float4 *jdup_buf = nullptr, *rdup_buf = nullptr, *fdup_buf = nullptr, *tbc_buf = nullptr, *tbe_buf = nullptr;
    float4 *sdup_buf = nullptr;           // symmetric-kernel layout
    float4 *hbc_buf = nullptr, *hbe_buf = nullptr;  // half-tile boxes (256-particle symmetric variant)
    uint8_t *submask_buf = nullptr;       // its sub-block near masks
    int64_t submask_cap = 0;
    unsigned long long *qmax = nullptr;   // largest |coordinate| (centre grid of the staging)
    NearScratch nr;                       // near-field bitmap and work items
    double *per_part = nullptr;           // periodic mode: FP64 partials per work item
    PeriodicSymScratch ps;                // periodic cut sum: symmetric kernel scratch
    SimDesc *dsim = nullptr;              // device table of one system
    unsigned long long *stats = nullptr;  // near / all tile pairs, accumulated
    float alpha = 0.03125f;
    int64_t np = 0, ntile_cap = 0;
    int variant = -1;
    ForcePlan plan;
    double *partial = nullptr;
    size_t partial_cap = 0;
    SortScratch srt;
    int *err = nullptr;       // device error word
    int *flag = nullptr;      // device validation flags
    int *nonfinite = nullptr; // device word: a force or state value was NaN or Inf (err + 2)
    long long wait_ns = 2000000000LL;
    int64_t since_sort = 0;
    // benchmark hooks
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> force_events;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> far_events;  // far-field kernel alone
    int64_t force_launches = 0;
    int64_t kernel_launches = 0;
    int64_t *inv = nullptr;   // inverse permutation scratch (subset forces)
    int64_t *tgt = nullptr;   // mapped target indices
    int64_t tgt_cap = 0;
    std::vector<void *> allocs;
    std::vector<size_t> sizes;
};

namespace {

steps_status dev_alloc(steps_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (g_mem_limit && g_mem_used + bytes > g_mem_limit) {
            set_error("device allocation of %zu bytes exceeds the library memory limit (%zu of %zu used)",
                      bytes, g_mem_used, g_mem_limit);
            return STEPS_ENOMEM;
        }
        g_mem_used += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        g_mem_used -= bytes;
        return cuda_status(e, "cudaMalloc");
    }
    c->allocs.push_back(*p);
    c->sizes.push_back(bytes);
    return STEPS_OK;
}

template <typename T>
steps_status alloc_n(steps_ctx *c, T **p, size_t count) {
    return dev_alloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

void dev_free(steps_ctx *c, void *p) {
    if (!p) return;
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (c->allocs[k] == p) {
            cudaFree(p);
            std::lock_guard<std::mutex> lk(g_mem_mu);
            g_mem_used -= c->sizes[k];
            c->allocs.erase(c->allocs.begin() + k);
            c->sizes.erase(c->sizes.begin() + k);
            return;
        }
    }
}

// Check the device error word and clear it.
steps_status sync_and_check(steps_ctx *c) {
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    int w[3] = {0, 0, 0};  // error word, validation flags, non-finite word
    STEPS_CUDA(cudaMemcpy(w, c->err, sizeof(w), cudaMemcpyDeviceToHost));
    if (w[0]) {
        STEPS_CUDA(cudaMemset(c->err, 0, sizeof(int)));
        set_error("a bounded device-side wait ran out (error word %d); the kernel exited early", w[0]);
        return (steps_status)w[0];
    }
    if (w[2]) {
        STEPS_CUDA(cudaMemset(c->nonfinite, 0, sizeof(int)));
        set_error("a computed force, position or velocity is NaN or Inf (FP32 overflow of the inputs' scale?)");
        return STEPS_ENONFINITE;
    }
    return STEPS_OK;
}

// Default variant before tuning (and the choice below 2^17 particles): the
// first built variant of the requested summation mode with 4 targets per
// thread; systems below 32,768 particles use 64-particle tiles (2 targets per
// thread) to limit padding and near-field work.  Periodic mode (both the cut
// image sum and the quasi-periodic sum) runs on the symmetric periodic
// kernel's 128-particle tiles.
int pick_variant(const steps_ctx *c) {
    const bool comp = c->cfg.prec != STEPS_F32_NAIVE;
    if (c->cfg.tile_override > 0 && c->cfg.tile_override <= num_variants())
        return c->cfg.tile_override - 1;
    if (c->cosmo.periodic && comp) {
        // the symmetric periodic kernel's 128-particle tiles
        for (int k = 0; k < num_variants(); ++k)
            if (variant(k).form == 2 && 32 * variant(k).KI == periodic_sym_tile()) return k;
    }
    const int ki = (c->n >= 32768 && !c->cosmo.periodic) ? 4 : 2;
    for (int k = 0; k < num_variants(); ++k) {
        const Variant &v = variant(k);
        if (v.comp == comp && v.KI == ki) return k;
    }
    return 0;
}

// Tuned variant per (size bucket, compensated?) for this process.
std::mutex g_tune_mu;
std::vector<std::pair<std::pair<int, int>, int>> g_tuned;

steps_status configure_variant(steps_ctx *c, int k) {
    const Variant &v = variant(k);
    c->variant = k;
    const int64_t bi = (int64_t)v.W * 32 * v.KI;
    c->stg.n = c->n;
    c->stg.np = (c->n + bi - 1) / bi * bi;  // <= c->np, the allocated padding
    c->stg.T = 32 * v.KI;
    c->stg.ntile = c->stg.np / c->stg.T;
    c->stg.jdup = c->jdup_buf;
    c->stg.rdup = c->rdup_buf;
    // the per-target periodic kernel reads the expansion layout unless the
    // symmetric periodic kernel takes the far images
    const bool per_sym = c->cosmo.periodic && v.form == 2 && 32 * v.KI == periodic_sym_tile();
    c->stg.fdup = (v.form == 1 || (c->cosmo.periodic && !per_sym)) ? c->fdup_buf : nullptr;
    c->stg.sdup = v.form == 2 ? c->sdup_buf : nullptr;
    c->stg.qmax = c->qmax;
    // periodic mode stages box units with a centre grid of at least 2^-21, so
    // that every image shift c_I - c_J - n is exact in FP32
    c->stg.pscale = c->cosmo.periodic ? 1.0 / c->cosmo.box : 1.0;
    c->stg.qemin = c->cosmo.periodic ? 1 : -1000;
    c->stg.tbox_c = c->tbc_buf;
    c->stg.tbox_e = c->tbe_buf;
    SimDesc d{};
    d.tile_off = 0;
    d.ntile = c->stg.ntile;
    c->plan = plan_force_multi(k, c->num_sms, &d, 1, c->dsim, &c->nr.bits_words);
    // the 256-particle symmetric variant classifies 128 x 128 sub-blocks
    const bool sub = v.form == 2 && v.sub;
    if (sub) {
        if (!c->hbc_buf) {
            STEPS_TRY(alloc_n(c, &c->hbc_buf, 2 * (c->np / 256) + 2));
            STEPS_TRY(alloc_n(c, &c->hbe_buf, 2 * (c->np / 256) + 2));
        }
        if (c->plan.mask_bytes > c->submask_cap) {
            dev_free(c, c->submask_buf);
            c->submask_buf = nullptr;
            c->submask_cap = 0;
            STEPS_TRY(alloc_n(c, &c->submask_buf, (size_t)c->plan.mask_bytes));
            c->submask_cap = c->plan.mask_bytes;
        }
    }
    c->stg.tbox_hc = sub ? c->hbc_buf : nullptr;
    c->stg.tbox_he = sub ? c->hbe_buf : nullptr;
    c->nr.submask = sub ? c->submask_buf : nullptr;
    STEPS_CUDA(cudaMemcpyAsync(c->dsim, &d, sizeof(d), cudaMemcpyHostToDevice, c->st));
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    c->nr.cap_items = 8 * (c->np / c->stg.T);
    if (c->plan.partial_elems > c->partial_cap) {
        dev_free(c, c->partial);
        c->partial = nullptr;
        c->partial_cap = 0;
        STEPS_TRY(alloc_n(c, &c->partial, c->plan.partial_elems));
        c->partial_cap = c->plan.partial_elems;
    }
    return STEPS_OK;
}

// Re-sort the FP64 state into Morton order; the permutation follows.
steps_status resort(steps_ctx *c) {
    const int64_t n = c->n;
    int launches = 0;
    STEPS_CUDA(morton_sort(n, c->x, c->y, c->z, c->srt, c->st, &launches));
    c->kernel_launches += launches + 12;
    double **arrs[] = {&c->x, &c->y, &c->z, &c->vx, &c->vy, &c->vz, &c->m, &c->h, &c->ax, &c->ay, &c->az};
    for (double **a : arrs) {
        STEPS_CUDA(gather_f64(n, c->srt.vals, *a, c->srt.tmp, c->st));
        std::swap(*a, c->srt.tmp);
    }
    STEPS_CUDA(gather_i64(n, c->srt.vals, c->perm, c->srt.tmpi, c->st));
    std::swap(c->perm, c->srt.tmpi);
    c->since_sort = 0;
    return STEPS_OK;
}

bool capturing(const steps_ctx *c) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

// Pair term at the current positions into ax, ay, az (sorted order).
steps_status compute_forces(steps_ctx *c) {
    const bool prof = c->profiling && !capturing(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr, f0 = nullptr, f1 = nullptr;
    if (prof) {
        STEPS_CUDA(cudaEventCreate(&e0));
        STEPS_CUDA(cudaEventCreate(&e1));
        if (c->cfg.prec != STEPS_F64) {
            STEPS_CUDA(cudaEventCreate(&f0));
            STEPS_CUDA(cudaEventCreate(&f1));
        }
    }
    if (c->cosmo.periodic) {
        // Eq. 2 with the image sum of Eq. 5
        if (c->cfg.prec == STEPS_F64) {
            if (prof) STEPS_CUDA(cudaEventRecord(e0, c->st));
            STEPS_CUDA(launch_periodic_f64(c->n, c->x, c->y, c->z, c->m, c->h, c->cosmo.G, c->cosmo.box,
                                           c->cfg.images, c->ax, c->ay, c->az, c->st));
            c->kernel_launches += 1;
        } else {
            launch_stage(c->stg, c->x, c->y, c->z, c->m, c->h, c->st);
            STEPS_CUDA(cudaGetLastError());
            if (prof) STEPS_CUDA(cudaEventRecord(e0, c->st));
            const bool sym = c->stg.sdup && c->stg.T == periodic_sym_tile();
            STEPS_CUDA(launch_periodic_f32(c->stg, c->x, c->y, c->z, c->cosmo.box, c->cfg.images, c->cosmo.G,
                                           c->per_part, sym ? &c->ps : nullptr, c->num_sms, c->ax, c->ay, c->az,
                                           c->st, f0, f1));
            // absmax, stage, (count, scan, symmetric), per-target, reduce
            c->kernel_launches += sym ? 7 : 4;
        }
        if (prof) STEPS_CUDA(cudaEventRecord(e1, c->st));
    } else if (c->cfg.prec == STEPS_F64) {
        if (prof) STEPS_CUDA(cudaEventRecord(e0, c->st));
        STEPS_CUDA(launch_force_f64(c->n, c->x, c->y, c->z, c->m, c->h, c->cosmo.G, 0, c->n, c->ax,
                                    c->ay, c->az, c->st));
        if (prof) STEPS_CUDA(cudaEventRecord(e1, c->st));
        c->kernel_launches += 1;
    } else {
        launch_stage(c->stg, c->x, c->y, c->z, c->m, c->h, c->st);
        STEPS_CUDA(cudaGetLastError());
        if (prof) STEPS_CUDA(cudaEventRecord(e0, c->st));
        STEPS_CUDA(launch_force_f32(c->plan, c->stg, c->partial, c->nr, c->err, c->stats, c->alpha,
                                    c->wait_ns, c->num_sms, c->st, f0, f1));
        if (prof) STEPS_CUDA(cudaEventRecord(e1, c->st));
        STEPS_CUDA(launch_fixup(c->plan, c->stg, c->partial, c->nr, c->cosmo.G, c->ax, c->ay,
                                c->az, c->st));
        // absmax, stage, (classify,) far, near count, near scan, near, fixup
        c->kernel_launches += variant(c->variant).form == 2 ? 8 : 7;
    }
    // non-finite result check (read at the next synchronising call: STEPS_ENONFINITE)
    STEPS_CUDA(launch_check_finite3(c->n, c->ax, c->ay, c->az, c->nonfinite, c->st));
    c->kernel_launches += 1;
    c->force_launches += 1;
    if (prof) c->force_events.push_back({e0, e1});
    if (prof && f0) c->far_events.push_back({f0, f1});
    return STEPS_OK;
}

// Autotuner: for systems of >= 2^14 particles, time every built variant of
// the requested summation mode (one warm-up evaluation, then the median of
// three timed ones) and keep the fastest; the choice is cached per
// (floor(log2 n), mode) for the process.  Below 2^14 particles an evaluation
// is dominated by launch latency and the default is kept.
steps_status autotune(steps_ctx *c) {
    const bool comp = c->cfg.prec != STEPS_F32_NAIVE;
    if (c->n < (1 << 14)) return STEPS_OK;
    int bucket = 0;
    while ((int64_t(1) << (bucket + 1)) <= c->n) ++bucket;
    const std::pair<int, int> key(bucket, comp ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &e : g_tuned)
            if (e.first == key) return configure_variant(c, e.second);
    }
    const bool prof = c->profiling;
    c->profiling = false;
    constexpr int kReps = 3;
    cudaEvent_t ev[kReps + 1];
    for (auto &e : ev) STEPS_CUDA(cudaEventCreate(&e));
    int best = c->variant;
    float best_ms = 1e30f;
    steps_status st = STEPS_OK;
    for (int k = 0; k < num_variants() && st == STEPS_OK; ++k) {
        if (variant(k).comp != comp) continue;
        st = configure_variant(c, k);
        if (st == STEPS_OK) st = compute_forces(c);  // warm-up (first launch of the variant)
        for (int r = 0; r < kReps && st == STEPS_OK; ++r) {
            if (cudaEventRecord(ev[r], c->st) != cudaSuccess) st = STEPS_ECUDA;
            if (st == STEPS_OK) st = compute_forces(c);
        }
        if (st == STEPS_OK && cudaEventRecord(ev[kReps], c->st) != cudaSuccess) st = STEPS_ECUDA;
        if (st == STEPS_OK) st = sync_and_check(c);
        float t[kReps];
        bool ok = st == STEPS_OK;
        for (int r = 0; r < kReps && ok; ++r) ok = cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]) == cudaSuccess;
        if (ok) {
            std::sort(t, t + kReps);
            if (t[kReps / 2] < best_ms) {
                best_ms = t[kReps / 2];
                best = k;
            }
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    c->profiling = prof;
    STEPS_TRY(st);
    cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), c->st);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned.push_back({key, best});
    }
    return configure_variant(c, best);
}

// One KDK step with dt already in sc[SC_DT] (Eq. 11).
steps_status issue_step(steps_ctx *c, bool do_sort) {
    c->kernel_launches += 4;  // kick, drift, rk4, kick
    STEPS_CUDA(launch_kick(c->n, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->ax, c->ay, c->az, c->sc,
                           c->cosmo, c->st));
    if (c->cosmo.periodic)
        STEPS_CUDA(launch_drift_wrap(c->n, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->sc, c->cosmo.box, c->st));
    else
        STEPS_CUDA(launch_drift(c->n, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->sc, c->st));
    STEPS_CUDA(launch_rk4(c->sc, c->cosmo, c->st));
    if (do_sort) STEPS_TRY(resort(c));
    STEPS_TRY(compute_forces(c));
    STEPS_CUDA(launch_kick(c->n, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->ax, c->ay, c->az, c->sc,
                           c->cosmo, c->st));
    return STEPS_OK;
}

int resort_every(const steps_ctx *c) { return c->cfg.resort_every > 0 ? c->cfg.resort_every : 8; }

steps_status validate(steps_ctx *c, const double *d, int64_t count, bool positive, const char *name) {
    STEPS_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), c->st));
    STEPS_CUDA(launch_check_finite(count, d, positive ? 1 : 0, c->flag, c->st));
    int f = 0;
    STEPS_CUDA(cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    if (f & 1) {
        set_error("%s contains NaN or Inf", name);
        return STEPS_EINVAL;
    }
    if (f & 2) {
        set_error("%s must be > 0", name);
        return STEPS_EINVAL;
    }
    return STEPS_OK;
}

// Copy a caller [n][3] array (host or device) into sorted SoA via perm (or identity).
steps_status load3(steps_ctx *c, const double *src, double *a, double *b, double *cc, bool via_perm) {
    STEPS_CUDA(cudaMemcpyAsync(c->tmp3, src, sizeof(double) * 3 * c->n, cudaMemcpyDefault, c->st));
    STEPS_TRY(validate(c, c->tmp3, 3 * c->n, false, "a position/velocity array"));
    if (via_perm)
        STEPS_CUDA(launch_gather3(c->n, c->perm, c->tmp3, a, b, cc, c->st));
    else
        STEPS_CUDA(launch_split3(c->n, c->tmp3, a, b, cc, c->st));
    return STEPS_OK;
}

steps_status store3(steps_ctx *c, double *dst, const double *a, const double *b, const double *cc) {
    STEPS_CUDA(launch_scatter3(c->n, c->perm, a, b, cc, c->tmp3, c->st));
    STEPS_CUDA(cudaMemcpyAsync(dst, c->tmp3, sizeof(double) * 3 * c->n, cudaMemcpyDefault, c->st));
    return STEPS_OK;
}

steps_status init_impl(steps_ctx *c, const double *pos, const double *vel, const double *mass,
                       const double *soft, double h_min, double t0, double a0) {
    const int64_t n = c->n;
    STEPS_CUDA(cudaGetDevice(&c->device));
    STEPS_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    double **soa[] = {&c->x, &c->y, &c->z, &c->vx, &c->vy, &c->vz, &c->m, &c->h, &c->ax, &c->ay, &c->az};
    for (double **a : soa) STEPS_TRY(alloc_n(c, a, n));
    STEPS_TRY(alloc_n(c, &c->perm, n));
    STEPS_TRY(alloc_n(c, &c->sc, SC_COUNT));
    c->nred = 256;
    STEPS_TRY(alloc_n(c, &c->red, 4 * c->nred + 8));
    STEPS_TRY(alloc_n(c, &c->tmp3, 3 * n));
    STEPS_TRY(alloc_n(c, &c->err, 4));
    c->flag = c->err + 1;
    c->nonfinite = c->err + 2;
    STEPS_CUDA(cudaMemsetAsync(c->err, 0, 4 * sizeof(int), c->st));
    // staging: padded to the largest multiple any variant's i-block (W x 32 KI
    // targets) needs, so that every variant fits; each pads to its own multiple
    c->np = 0;
    for (int k = 0; k < num_variants(); ++k) {
        const int64_t bi = (int64_t)variant(k).W * 32 * variant(k).KI;
        c->np = std::max<int64_t>(c->np, (n + bi - 1) / bi * bi);
    }
    c->ntile_cap = c->np / 64;
    STEPS_TRY(alloc_n(c, &c->jdup_buf, 2 * c->np));
    STEPS_TRY(alloc_n(c, &c->rdup_buf, 2 * c->np));
    STEPS_TRY(alloc_n(c, &c->fdup_buf, 4 * c->np));
    STEPS_TRY(alloc_n(c, &c->sdup_buf, 2 * c->np));
    STEPS_TRY(alloc_n(c, &c->qmax, 1));
    STEPS_TRY(alloc_n(c, &c->nr.sym_acc, 3 * c->np));
    STEPS_TRY(alloc_n(c, &c->nr.sym_next, 1));
    STEPS_TRY(alloc_n(c, &c->nr.tscale, c->ntile_cap));
    STEPS_TRY(alloc_n(c, &c->nr.tinv, c->ntile_cap));
    c->nr.nonfinite = c->nonfinite;
    STEPS_TRY(alloc_n(c, &c->nr.bits, (size_t)c->ntile_cap * ((c->ntile_cap + 31) / 32)));
    STEPS_TRY(alloc_n(c, &c->nr.cnt, c->ntile_cap));
    STEPS_TRY(alloc_n(c, &c->nr.item_off, c->ntile_cap + 1));
    STEPS_TRY(alloc_n(c, &c->nr.meta, 4));
    STEPS_TRY(alloc_n(c, &c->dsim, 1));
    // near-field work-item partials: up to 8 items per target tile (the chunk
    // size adapts on the device), 3 doubles per particle per item
    STEPS_TRY(alloc_n(c, &c->nr.item_part, (size_t)24 * c->np));
    if (c->cosmo.periodic && c->cfg.prec != STEPS_F64) {
        STEPS_TRY(alloc_n(c, &c->per_part, periodic_part_elems(c->np, c->num_sms)));
        {
            const int64_t np_sym = c->np / periodic_sym_tile();
            const int64_t npairs = periodic_sym_pairs(np_sym);
            c->ps.acc = c->nr.sym_acc;
            c->ps.tscale = c->nr.tscale;
            c->ps.tinv = c->nr.tinv;
            c->ps.nonfinite = c->nonfinite;
            STEPS_TRY(alloc_n(c, &c->ps.off, npairs + 2));  // offsets and the work counter
            STEPS_TRY(alloc_n(c, &c->ps.bnd, npairs));
            STEPS_TRY(alloc_n(c, &c->ps.soft, npairs));
            STEPS_TRY(alloc_n(c, &c->ps.soff, np_sym + 1));
            // the soft partner lists share the item partials of the per-target kernel
            c->ps.cap_items = (int64_t)(periodic_part_elems(c->np, c->num_sms) / (3 * periodic_sym_tile()));
            STEPS_TRY(alloc_n(c, &c->ps.slist, c->ps.cap_items));
        }
    }
    STEPS_TRY(alloc_n(c, &c->stats, 2));
    STEPS_CUDA(cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), c->st));
    STEPS_TRY(alloc_n(c, &c->tbc_buf, c->ntile_cap));
    STEPS_TRY(alloc_n(c, &c->tbe_buf, c->ntile_cap));
    // sort scratch
    int64_t p2 = 1;
    while (p2 < n) p2 <<= 1;
    c->srt.npow2 = std::max<int64_t>(p2, 2);
    STEPS_TRY(alloc_n(c, &c->srt.keys, c->srt.npow2));
    STEPS_TRY(alloc_n(c, &c->srt.vals, c->srt.npow2));
    STEPS_TRY(alloc_n(c, &c->srt.bbox, 8 + 6 * 256));  // the box, then the per-CTA partials of morton_sort
    STEPS_TRY(alloc_n(c, &c->srt.tmp, n));
    STEPS_TRY(alloc_n(c, &c->srt.tmpi, n));

    // upload (caller order == initial internal order)
    STEPS_TRY(load3(c, pos, c->x, c->y, c->z, false));
    if (c->cosmo.periodic) {
        for (double *v : {c->x, c->y, c->z}) STEPS_CUDA(launch_wrap(n, v, c->cosmo.box, c->st));
    }
    if (vel) {
        STEPS_TRY(load3(c, vel, c->vx, c->vy, c->vz, false));
    } else {
        STEPS_CUDA(cudaMemsetAsync(c->vx, 0, sizeof(double) * n, c->st));
        STEPS_CUDA(cudaMemsetAsync(c->vy, 0, sizeof(double) * n, c->st));
        STEPS_CUDA(cudaMemsetAsync(c->vz, 0, sizeof(double) * n, c->st));
    }
    STEPS_CUDA(cudaMemcpyAsync(c->m, mass, sizeof(double) * n, cudaMemcpyDefault, c->st));
    STEPS_TRY(validate(c, c->m, n, true, "mass"));
    if (soft) {
        STEPS_CUDA(cudaMemcpyAsync(c->h, soft, sizeof(double) * n, cudaMemcpyDefault, c->st));
    } else {
        if (!(h_min > 0.0) || !std::isfinite(h_min)) {
            set_error("h_min must be finite and > 0 when soft is NULL");
            return STEPS_EINVAL;
        }
        STEPS_CUDA(launch_softening(n, c->m, h_min, c->h, c->red, c->st));  // Eq. 7
    }
    STEPS_TRY(validate(c, c->h, n, true, "softening"));
    STEPS_CUDA(cudaMemsetAsync(c->ax, 0, sizeof(double) * n, c->st));
    STEPS_CUDA(cudaMemsetAsync(c->ay, 0, sizeof(double) * n, c->st));
    STEPS_CUDA(cudaMemsetAsync(c->az, 0, sizeof(double) * n, c->st));
    STEPS_CUDA(launch_iota(n, c->perm, c->st));
    double sc[SC_COUNT] = {0};
    sc[SC_T] = t0;
    sc[SC_A] = c->cosmo.comoving ? a0 : 1.0;
    if (c->cosmo.comoving) {
        const double ia = 1.0 / a0;
        sc[SC_H] = c->cosmo.H0 * std::sqrt(c->cosmo.Om * ia * ia * ia + c->cosmo.Or * ia * ia * ia * ia +
                                           c->cosmo.OL + c->cosmo.Ok * ia * ia);
    }
    STEPS_CUDA(cudaMemcpyAsync(c->sc, sc, sizeof(sc), cudaMemcpyHostToDevice, c->st));
    STEPS_TRY(configure_variant(c, pick_variant(c)));
    STEPS_TRY(resort(c));
    if (c->cfg.prec != STEPS_F64 && c->cfg.tile_override == 0 && !c->cosmo.periodic) STEPS_TRY(autotune(c));
    STEPS_TRY(compute_forces(c));
    return sync_and_check(c);
}

}  // namespace

extern "C" {

steps_config steps_default_config(void) {
    steps_config c;
    std::memset(&c, 0, sizeof(c));
    c.G = 1.0;
    c.H0 = 1.0;
    c.Om = 0.3;
    c.OL = 0.7;
    c.mode = STEPS_STATIC;
    c.prec = STEPS_F32_COMP;
    c.resort_every = 8;
    c.tile_override = 0;
    return c;
}

steps_status steps_init(steps_ctx **out, int64_t n, const double *pos, const double *vel,
                        const double *mass, const double *soft, double h_min, double t0, double a0,
                        const steps_config *cfg, void *cuda_stream) {
    if (!out) {
        set_error("out is NULL");
        return STEPS_EINVAL;
    }
    *out = nullptr;
    if (n <= 0 || n > (int64_t)1 << 31) {
        set_error("n must be in [1, 2^31], got %lld", (long long)n);
        return STEPS_EINVAL;
    }
    if (!pos || !mass) {
        set_error("pos and mass are required");
        return STEPS_EINVAL;
    }
    steps_config c = cfg ? *cfg : steps_default_config();
    if (c.mode != STEPS_STATIC && c.mode != STEPS_COMOVING && c.mode != STEPS_COMOVING_REVERSED &&
        c.mode != STEPS_PERIODIC) {
        set_error("unknown mode %d", c.mode);
        return STEPS_EINVAL;
    }
    if (c.mode == STEPS_PERIODIC) {
        if (!(c.box > 0.0) || !std::isfinite(c.box) || (c.images != 0 && c.images != 1)) {
            set_error("periodic mode needs a finite box > 0 and images 0 (cut at 2.6 L) or 1 (quasi-periodic)");
            return STEPS_EINVAL;
        }
        if (c.prec == STEPS_F32_NAIVE) {
            set_error("periodic mode runs with STEPS_F32_COMP or STEPS_F64");
            return STEPS_EUNSUPPORTED;
        }
    }
    if (c.prec < STEPS_F32_COMP || c.prec > STEPS_F64) {
        set_error("unknown precision %d", c.prec);
        return STEPS_EINVAL;
    }
    if (c.tile_override < 0 || c.tile_override > num_variants()) {
        set_error("tile_override %d out of range [0, %d]", c.tile_override, num_variants());
        return STEPS_EINVAL;
    }
    if (c.tile_override > 0 && variant(c.tile_override - 1).comp != (c.prec == STEPS_F32_COMP) &&
        c.prec != STEPS_F64) {
        set_error("tile_override %d does not match the precision mode", c.tile_override);
        return STEPS_EINVAL;
    }
    if (!std::isfinite(c.G) || !std::isfinite(t0) ||
        (c.mode != STEPS_STATIC && (!(a0 > 0.0) || !std::isfinite(a0) || !std::isfinite(c.H0)))) {
        set_error("G, t0, H0 and a0 must be finite (a0 > 0 in comoving mode)");
        return STEPS_EINVAL;
    }
    steps_ctx *ctx = new (std::nothrow) steps_ctx();
    if (!ctx) {
        set_error("host allocation failed");
        return STEPS_ENOMEM;
    }
    ctx->n = n;
    ctx->cfg = c;
    const bool rev = c.mode == STEPS_COMOVING_REVERSED;
    const bool per = c.mode == STEPS_PERIODIC;
    ctx->cosmo = Cosmo{rev ? -c.G : c.G, c.H0, c.Om, c.OL, c.Or, c.Ok, c.mode != STEPS_STATIC ? 1 : 0, rev ? 1 : 0,
                       per ? 1 : 0, per ? c.box : 0.0};
    if (cuda_stream) {
        ctx->st = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return cuda_status(e, "cudaStreamCreate");
        }
        ctx->own_stream = true;
    }
    steps_status s = init_impl(ctx, pos, vel, mass, soft, h_min, t0, a0);
    if (s != STEPS_OK) {
        steps_free(ctx);
        return s;
    }
    *out = ctx;
    return STEPS_OK;
}

steps_status steps_forces(steps_ctx *c, double *acc_out) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    STEPS_TRY(compute_forces(c));
    if (acc_out) STEPS_TRY(store3(c, acc_out, c->ax, c->ay, c->az));
    return sync_and_check(c);
}

steps_status steps_kdk_step(steps_ctx *c, double dt, double *a_out) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    if (!std::isfinite(dt)) {
        set_error("dt must be finite");
        return STEPS_EINVAL;
    }
    STEPS_CUDA(launch_set_scalar(c->sc, SC_DT, dt, c->st));
    c->kernel_launches += 1;
    const bool do_sort = ++c->since_sort >= resort_every(c);
    STEPS_TRY(issue_step(c, do_sort));
    if (a_out) {
        STEPS_CUDA(cudaMemcpyAsync(a_out, c->sc + SC_A, sizeof(double), cudaMemcpyDefault, c->st));
        return sync_and_check(c);
    }
    return STEPS_OK;
}

steps_status steps_kdk_run(steps_ctx *c, int nsteps, const double *dts) {
    if (!c || nsteps < 0 || (nsteps > 0 && !dts)) {
        set_error("bad arguments to steps_kdk_run");
        return STEPS_EINVAL;
    }
    if (nsteps == 0) return STEPS_OK;
    for (int k = 0; k < nsteps; ++k) {
        if (!std::isfinite(dts[k])) {
            set_error("dts[%d] is not finite", k);
            return STEPS_EINVAL;
        }
    }
    if (nsteps > c->dts_cap) {
        dev_free(c, c->dts);
        c->dts = nullptr;
        c->dts_cap = 0;
        STEPS_TRY(alloc_n(c, &c->dts, nsteps));
        c->dts_cap = nsteps;
    }
    STEPS_CUDA(cudaMemcpyAsync(c->dts, dts, sizeof(double) * nsteps, cudaMemcpyDefault, c->st));
    STEPS_CUDA(launch_set_scalar(c->sc, SC_RUN, 0.0, c->st));
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    // Capture one plain step and one step with a re-sort; replay per step.
    // The re-sort swaps buffer pointers, so the sorting graph is re-captured
    // (and the plain one with it) after every sort.
    cudaGraphExec_t plain = nullptr;
    steps_status s = STEPS_OK;
    auto capture = [&](bool do_sort, cudaGraphExec_t *exec) -> steps_status {
        cudaGraph_t g = nullptr;
        STEPS_CUDA(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        steps_status si = STEPS_OK;
        if (launch_set_dt(c->sc, c->dts, c->st) != cudaSuccess) si = STEPS_ECUDA;
        if (si == STEPS_OK) si = issue_step(c, do_sort);
        cudaError_t e = cudaStreamEndCapture(c->st, &g);
        if (si != STEPS_OK) {
            if (g) cudaGraphDestroy(g);
            return si;
        }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
        return STEPS_OK;
    };
    for (int k = 0; k < nsteps && s == STEPS_OK; ++k) {
        const bool do_sort = ++c->since_sort >= resort_every(c);
        if (do_sort) {
            // a sorting step changes the buffer roles: run it directly
            if (plain) {
                cudaGraphExecDestroy(plain);
                plain = nullptr;
            }
            if (launch_set_dt(c->sc, c->dts, c->st) != cudaSuccess) s = STEPS_ECUDA;
            if (s == STEPS_OK) s = issue_step(c, true);
            continue;
        }
        if (!plain) s = capture(false, &plain);
        if (s == STEPS_OK) {
            cudaError_t e = cudaGraphLaunch(plain, c->st);
            if (e != cudaSuccess) s = cuda_status(e, "cudaGraphLaunch");
        }
    }
    if (plain) cudaGraphExecDestroy(plain);
    if (s != STEPS_OK) return s;
    return sync_and_check(c);
}

namespace {

steps_status check_timestep_args(const steps_ctx *c, double eps, double dt_max, double t_end) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    if (!(eps > 0.0) || !std::isfinite(eps) || !(dt_max > 0.0) || !std::isfinite(dt_max) ||
        std::isnan(t_end)) {
        set_error("eps and dt_max must be finite and > 0, t_end a number (+inf: no limit)");
        return STEPS_EINVAL;
    }
    return STEPS_OK;
}

cudaError_t issue_timestep(steps_ctx *c, double eps, double dt_max, double t_end) {
    c->kernel_launches += 2;
    return launch_timestep(c->n, c->x, c->y, c->z, c->vx, c->vy, c->vz, c->ax, c->ay, c->az, c->h, c->sc,
                           c->cosmo, eps, dt_max, t_end, c->red, c->nred, c->st);
}

}  // namespace

steps_status steps_timestep(steps_ctx *c, double eps, double dt_max, double t_end, double *dt_out) {
    STEPS_TRY(check_timestep_args(c, eps, dt_max, t_end));
    STEPS_CUDA(issue_timestep(c, eps, dt_max, t_end));
    if (dt_out) {
        STEPS_CUDA(cudaMemcpyAsync(dt_out, c->sc + SC_DT, sizeof(double), cudaMemcpyDefault, c->st));
        return sync_and_check(c);
    }
    return STEPS_OK;
}

steps_status steps_kdk_run_adaptive(steps_ctx *c, int nsteps, double eps, double dt_max, double t_end,
                                    double *t_out) {
    STEPS_TRY(check_timestep_args(c, eps, dt_max, t_end));
    if (nsteps < 0) {
        set_error("nsteps must be >= 0");
        return STEPS_EINVAL;
    }
    // Each step: Eq. 12 on the device at the step's start, then Eq. 11 with
    // that length.  Steps without a re-sort replay one captured graph.
    cudaGraphExec_t plain = nullptr;
    steps_status s = STEPS_OK;
    for (int k = 0; k < nsteps && s == STEPS_OK; ++k) {
        const bool do_sort = ++c->since_sort >= resort_every(c);
        if (do_sort) {
            if (plain) {
                cudaGraphExecDestroy(plain);
                plain = nullptr;
            }
            if (issue_timestep(c, eps, dt_max, t_end) != cudaSuccess) s = STEPS_ECUDA;
            if (s == STEPS_OK) s = issue_step(c, true);
            continue;
        }
        if (!plain) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                s = cuda_status(e, "cudaStreamBeginCapture");
                break;
            }
            steps_status si = issue_timestep(c, eps, dt_max, t_end) == cudaSuccess ? STEPS_OK : STEPS_ECUDA;
            if (si == STEPS_OK) si = issue_step(c, false);
            e = cudaStreamEndCapture(c->st, &g);
            if (si != STEPS_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                s = si != STEPS_OK ? si : cuda_status(e, "cudaStreamEndCapture");
                break;
            }
            e = cudaGraphInstantiate(&plain, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                plain = nullptr;
                s = cuda_status(e, "cudaGraphInstantiate");
                break;
            }
        }
        cudaError_t e = cudaGraphLaunch(plain, c->st);
        if (e != cudaSuccess) s = cuda_status(e, "cudaGraphLaunch");
    }
    if (plain) cudaGraphExecDestroy(plain);
    if (s != STEPS_OK) return s;
    if (t_out) STEPS_CUDA(cudaMemcpyAsync(t_out, c->sc + SC_T, sizeof(double), cudaMemcpyDefault, c->st));
    return sync_and_check(c);
}

steps_status steps_get_state(steps_ctx *c, double *pos, double *vel, double *acc, double *t,
                             double *a) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    STEPS_CUDA(launch_check_finite3(c->n, c->x, c->y, c->z, c->nonfinite, c->st));
    STEPS_CUDA(launch_check_finite3(c->n, c->vx, c->vy, c->vz, c->nonfinite, c->st));
    if (pos) {
        STEPS_TRY(store3(c, pos, c->x, c->y, c->z));
        STEPS_CUDA(cudaStreamSynchronize(c->st));
    }
    if (vel) {
        STEPS_TRY(store3(c, vel, c->vx, c->vy, c->vz));
        STEPS_CUDA(cudaStreamSynchronize(c->st));
    }
    if (acc) {
        STEPS_TRY(store3(c, acc, c->ax, c->ay, c->az));
        STEPS_CUDA(cudaStreamSynchronize(c->st));
    }
    double sc[SC_COUNT];
    STEPS_CUDA(cudaMemcpyAsync(sc, c->sc, sizeof(sc), cudaMemcpyDeviceToHost, c->st));
    STEPS_TRY(sync_and_check(c));
    if (t) *t = sc[SC_T];
    if (a) *a = sc[SC_A];
    return STEPS_OK;
}

steps_status steps_set_state(steps_ctx *c, const double *pos, const double *vel, double t, double a) {
    if (!c || !pos || !vel) {
        set_error("ctx, pos and vel are required");
        return STEPS_EINVAL;
    }
    if (!std::isfinite(t) || (c->cosmo.comoving && !(a > 0.0 && std::isfinite(a)))) {
        set_error("t must be finite and a > 0");
        return STEPS_EINVAL;
    }
    STEPS_TRY(load3(c, pos, c->x, c->y, c->z, true));
    if (c->cosmo.periodic) {
        for (double *v : {c->x, c->y, c->z}) STEPS_CUDA(launch_wrap(c->n, v, c->cosmo.box, c->st));
    }
    STEPS_TRY(load3(c, vel, c->vx, c->vy, c->vz, true));
    double sc[SC_COUNT];
    STEPS_CUDA(cudaMemcpyAsync(sc, c->sc, sizeof(sc), cudaMemcpyDeviceToHost, c->st));
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    sc[SC_T] = t;
    if (c->cosmo.comoving) {
        const double ia = 1.0 / a;
        sc[SC_A] = a;
        sc[SC_H] = c->cosmo.H0 * std::sqrt(c->cosmo.Om * ia * ia * ia + c->cosmo.Or * ia * ia * ia * ia +
                                           c->cosmo.OL + c->cosmo.Ok * ia * ia);
    }
    STEPS_CUDA(cudaMemcpyAsync(c->sc, sc, sizeof(sc), cudaMemcpyHostToDevice, c->st));
    STEPS_TRY(resort(c));
    STEPS_TRY(compute_forces(c));
    return sync_and_check(c);
}

// Checkpoint layout: int64 header[4] = {magic, n, since_sort, variant}, then
// double sc[SC_COUNT], 11 sorted FP64 arrays (x..az incl. m, h), int64 perm[n].
static const int64_t kCkptMagic = 0x5354655053434b31LL;  // "STePSCK1"

steps_status steps_checkpoint_size(steps_ctx *c, size_t *bytes) {
    if (!c || !bytes) {
        set_error("ctx and bytes are required");
        return STEPS_EINVAL;
    }
    *bytes = 4 * sizeof(int64_t) + SC_COUNT * sizeof(double) + 11 * sizeof(double) * c->n +
             sizeof(int64_t) * c->n;
    return STEPS_OK;
}

steps_status steps_checkpoint_save(steps_ctx *c, void *buf) {
    if (!c || !buf) {
        set_error("ctx and buf are required");
        return STEPS_EINVAL;
    }
    char *p = (char *)buf;
    int64_t hdr[4] = {kCkptMagic, c->n, c->since_sort, c->variant};
    std::memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    STEPS_CUDA(cudaMemcpyAsync(p, c->sc, SC_COUNT * sizeof(double), cudaMemcpyDefault, c->st));
    p += SC_COUNT * sizeof(double);
    const double *arrs[] = {c->x, c->y, c->z, c->vx, c->vy, c->vz, c->m, c->h, c->ax, c->ay, c->az};
    for (const double *a : arrs) {
        STEPS_CUDA(cudaMemcpyAsync(p, a, sizeof(double) * c->n, cudaMemcpyDefault, c->st));
        p += sizeof(double) * c->n;
    }
    STEPS_CUDA(cudaMemcpyAsync(p, c->perm, sizeof(int64_t) * c->n, cudaMemcpyDefault, c->st));
    return sync_and_check(c);
}

steps_status steps_checkpoint_load(steps_ctx *c, const void *buf) {
    if (!c || !buf) {
        set_error("ctx and buf are required");
        return STEPS_EINVAL;
    }
    const char *p = (const char *)buf;
    int64_t hdr[4];
    std::memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != kCkptMagic || hdr[1] != c->n) {
        set_error("checkpoint does not match this context (magic or n)");
        return STEPS_EINVAL;
    }
    if (hdr[3] < 0 || hdr[3] >= num_variants()) {
        set_error("checkpoint names an unknown force variant");
        return STEPS_EINVAL;
    }
    p += sizeof(hdr);
    STEPS_CUDA(cudaMemcpyAsync(c->sc, p, SC_COUNT * sizeof(double), cudaMemcpyDefault, c->st));
    p += SC_COUNT * sizeof(double);
    double *arrs[] = {c->x, c->y, c->z, c->vx, c->vy, c->vz, c->m, c->h, c->ax, c->ay, c->az};
    for (double *a : arrs) {
        STEPS_CUDA(cudaMemcpyAsync(a, p, sizeof(double) * c->n, cudaMemcpyDefault, c->st));
        p += sizeof(double) * c->n;
    }
    STEPS_CUDA(cudaMemcpyAsync(c->perm, p, sizeof(int64_t) * c->n, cudaMemcpyDefault, c->st));
    c->since_sort = hdr[2];
    if (hdr[3] != c->variant) STEPS_TRY(configure_variant(c, (int)hdr[3]));
    return sync_and_check(c);
}

steps_status steps_diagnostics(steps_ctx *c, double *ekin, double *epot, double p[3]) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    double *out = c->red + 4 * c->nred;  // 4 result slots after the block partials
    double host[5] = {0, 0, 0, 0, 0};
    if (ekin || p) {
        STEPS_CUDA(launch_kinetic(c->n, c->vx, c->vy, c->vz, c->m, c->red, c->nred, out, c->st));
        STEPS_CUDA(cudaMemcpyAsync(host, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        STEPS_CUDA(cudaStreamSynchronize(c->st));
    }
    if (epot && c->cosmo.periodic) {
        set_error("the pair potential is not available in periodic mode");
        return STEPS_EUNSUPPORTED;
    }
    if (epot) {
        STEPS_CUDA(launch_potential_f64(c->n, c->x, c->y, c->z, c->m, c->h, c->cosmo.G, c->tmp3,
                                        c->st));
        STEPS_CUDA(launch_sum(c->n, c->tmp3, c->red, c->nred, out, c->st));
        STEPS_CUDA(cudaMemcpyAsync(&host[4], out, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
    STEPS_TRY(sync_and_check(c));
    if (ekin) *ekin = host[0];
    if (p) {
        p[0] = host[1];
        p[1] = host[2];
        p[2] = host[3];
    }
    if (epot) *epot = 0.5 * host[4];
    return STEPS_OK;
}

steps_status steps_forces_subset(steps_ctx *c, int64_t nt, const int64_t *targets, double *acc_out) {
    if (!c || nt < 0 || (nt > 0 && (!targets || !acc_out))) {
        set_error("bad arguments to steps_forces_subset");
        return STEPS_EINVAL;
    }
    if (c->cosmo.periodic) {
        set_error("steps_forces_subset computes the open-boundary sum; not available in periodic mode");
        return STEPS_EUNSUPPORTED;
    }
    if (nt == 0) return STEPS_OK;
    if (nt > c->tgt_cap) {
        dev_free(c, c->tgt);
        c->tgt = nullptr;
        c->tgt_cap = 0;
        STEPS_TRY(alloc_n(c, &c->tgt, 2 * nt));
        c->tgt_cap = nt;
    }
    if (!c->inv) STEPS_TRY(alloc_n(c, &c->inv, c->n));
    double *out3 = nullptr;
    STEPS_TRY(alloc_n(c, &out3, 3 * nt));
    int64_t *caller = c->tgt + nt;
    steps_status s = STEPS_OK;
    int bad = 0;
    do {
        cudaError_t e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(caller, targets, sizeof(int64_t) * nt, cudaMemcpyDefault, c->st);
        if (e == cudaSuccess) e = launch_map_targets(c->n, c->perm, c->inv, nt, caller, c->tgt, c->flag, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) {
            s = cuda_status(e, "steps_forces_subset (targets)");
            break;
        }
        if (bad) {
            set_error("a target index is outside [0, n)");
            s = STEPS_EINVAL;
            break;
        }
        e = launch_force_f64_list(c->n, c->x, c->y, c->z, c->m, c->h, c->cosmo.G, nt, c->tgt, out3, c->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(acc_out, out3, sizeof(double) * 3 * nt, cudaMemcpyDefault, c->st);
        if (e != cudaSuccess) {
            s = cuda_status(e, "steps_forces_subset");
            break;
        }
        c->kernel_launches += 3;
        s = sync_and_check(c);
    } while (0);
    cudaStreamSynchronize(c->st);
    dev_free(c, out3);
    return s;
}

steps_status steps_set_near_alpha(steps_ctx *c, double alpha) {
    if (!c || !(alpha >= 0.0) || !std::isfinite(alpha)) {
        set_error("ctx is NULL or alpha is negative or not finite");
        return STEPS_EINVAL;
    }
    c->alpha = (float)alpha;
    return STEPS_OK;
}

steps_status steps_profile_enable(steps_ctx *c, int on) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    c->profiling = on != 0;
    return STEPS_OK;
}

steps_status steps_profile_read(steps_ctx *c, double *force_ms, int64_t *force_launches,
                                int64_t *kernel_launches, int reset) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    double ms = 0.0;
    for (auto &ev : c->force_events) {
        float t = 0.f;
        STEPS_CUDA(cudaEventElapsedTime(&t, ev.first, ev.second));
        ms += t;
    }
    if (force_ms) *force_ms = ms;
    if (force_launches) *force_launches = (int64_t)c->force_events.size();
    if (kernel_launches) *kernel_launches = c->kernel_launches;
    if (reset) {
        for (auto *list : {&c->force_events, &c->far_events}) {
            for (auto &ev : *list) {
                cudaEventDestroy(ev.first);
                cudaEventDestroy(ev.second);
            }
            list->clear();
        }
        c->force_launches = 0;
        c->kernel_launches = 0;
    }
    return STEPS_OK;
}

steps_status steps_profile_read_far(steps_ctx *c, double *far_ms, int64_t *far_launches) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    double ms = 0.0;
    for (auto &ev : c->far_events) {
        float t = 0.f;
        STEPS_CUDA(cudaEventElapsedTime(&t, ev.first, ev.second));
        ms += t;
    }
    if (far_ms) *far_ms = ms;
    if (far_launches) *far_launches = (int64_t)c->far_events.size();
    return STEPS_OK;
}

steps_status steps_force_stats(steps_ctx *c, uint64_t *near_pairs, uint64_t *all_pairs) {
    if (!c) {
        set_error("ctx is NULL");
        return STEPS_EINVAL;
    }
    unsigned long long h[2] = {0, 0};
    STEPS_CUDA(cudaMemcpyAsync(h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    STEPS_CUDA(cudaMemsetAsync(c->stats, 0, sizeof(h), c->st));
    STEPS_CUDA(cudaStreamSynchronize(c->st));
    if (near_pairs) *near_pairs = h[0];
    if (all_pairs) *all_pairs = h[1];
    return STEPS_OK;
}

int64_t steps_size(const steps_ctx *c) { return c ? c->n : 0; }

void steps_free(steps_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    for (auto &ev : c->force_events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    while (!c->allocs.empty()) dev_free(c, c->allocs.back());
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
}

const char *steps_strerror(steps_status s) {
    switch (s) {
        case STEPS_OK: return "ok";
        case STEPS_EINVAL: return "invalid argument";
        case STEPS_ENOMEM: return "out of device memory";
        case STEPS_ECUDA: return "CUDA error";
        case STEPS_ETIMEOUT: return "device-side wait timed out";
        case STEPS_ENONFINITE: return "non-finite result";
        case STEPS_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *steps_last_error(void) { return g_last_error; }

steps_status steps_set_wait_limit(steps_ctx *c, int64_t ns) {
    if (!c || ns < 0) {
        set_error("ctx is NULL or ns < 0");
        return STEPS_EINVAL;
    }
    c->wait_ns = ns;
    return STEPS_OK;
}

steps_status steps_set_memory_limit(size_t bytes) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_limit = bytes;
    return STEPS_OK;
}

int steps_num_variants(void) { return num_variants(); }

steps_status steps_get_variant(steps_ctx *c, int *k) {
    if (!c || !k) {
        set_error("ctx and k are required");
        return STEPS_EINVAL;
    }
    *k = c->cfg.prec == STEPS_F64 ? -1 : c->variant;
    return STEPS_OK;
}

const char *steps_variant_name(int k) {
    if (k < 0 || k >= num_variants()) return nullptr;
    return variant(k).name;
}

}  // extern "C"

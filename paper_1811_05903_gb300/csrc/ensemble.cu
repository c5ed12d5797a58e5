// Batched ensembles: many independent StePS simulations of uneven N and
// different cosmologies advanced together.  The members are concatenated
// (each padded to whole target blocks) and every force evaluation is ONE
// far-field launch whose stream-K unit space is the union of the members' own
// tile pairs, plus one near-field launch; the FP64 integrator kernels carry a
// per-member cosmology, scale factor and step length.  A step is captured once
// as a CUDA graph and replayed (re-sorting steps run directly).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "steps_internal.h"

using namespace steps;

struct steps_ens {
    int nsims = 0;
    std::vector<int64_t> n, off;  // real particles, first padded index of each member (+ total)
    int64_t NP = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int variant = 0;
    int resort_every = 8;
    int64_t since_sort = 0;
    long long wait_ns = 2000000000LL;
    // device state (sorted within each member)
    double *x = nullptr, *y = nullptr, *z = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr;
    double *m = nullptr, *h = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    int64_t *perm = nullptr;   // caller index inside the member
    int *sim = nullptr;        // member of each slot
    int64_t *doff = nullptr;   // [nsims + 1]
    double *sc = nullptr;      // [nsims][SC_COUNT]
    Cosmo *cosmo = nullptr;    // [nsims]
    double *dts = nullptr;     // [nsims][dts_cap]
    int dts_cap = 0;
    double *tmp3 = nullptr;    // caller-layout staging of one member
    int64_t tmp3_cap = 0;
    // FP32 path: staging buffers for every candidate variant, the chosen plan
    Staging stg;
    NearScratch nr;
    SimDesc *dsims = nullptr;
    ForcePlan plan;
    double *partial = nullptr;
    float4 *fdup_buf = nullptr, *sdup_buf = nullptr;
    float4 *hbox_c = nullptr, *hbox_e = nullptr;  // half-tile boxes (256-particle symmetric variant)
    uint8_t *submask = nullptr;                   // its sub-block near masks
    unsigned long long *qmax = nullptr;
    int *nonfinite = nullptr;
    int64_t pad = 0;                     // members are padded to multiples of this
    std::vector<int> candidates;         // variants the autotuner times
    SortScratch srt;
    int *err = nullptr;
    unsigned long long *stats = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;
};

namespace {

constexpr float kAlpha = 0.03125f;
// Members are padded to a multiple of this many particles: a whole number of
// target blocks (W x 32 KI) for every variant whose block divides it, so that
// all of them can run on one layout and the autotuner can compare them.
constexpr int64_t kEnsPad = 1024;

template <typename T>
steps_status ens_alloc(steps_ens *e, T **p, size_t count) {
    void *q = nullptr;
    STEPS_TRY(counted_malloc(&q, count * sizeof(T)));
    e->allocs.push_back({q, count * sizeof(T)});
    *p = static_cast<T *>(q);
    return STEPS_OK;
}

inline unsigned blocks_for(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

__device__ __forceinline__ double hubble_e(double a, const Cosmo &c) {
    const double ia = 1.0 / a;
    return c.H0 * sqrt(c.Om * ia * ia * ia + c.Or * ia * ia * ia * ia + c.OL + c.Ok * ia * ia);
}

// Padding slots: h = -1 marks them, zero mass and state.
__global__ void ens_pad_kernel(int nsims, const int64_t *__restrict__ off, const int64_t *__restrict__ nreal,
                               int *__restrict__ sim, int64_t *__restrict__ perm, double *x, double *y,
                               double *z, double *vx, double *vy, double *vz, double *m, double *h,
                               double *ax, double *ay, double *az) {
    const int s = blockIdx.y;
    const int64_t i = off[s] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= off[s + 1]) return;
    sim[i] = s;
    const int64_t local = i - off[s];
    perm[i] = local;
    if (local < nreal[s]) return;
    x[i] = y[i] = z[i] = vx[i] = vy[i] = vz[i] = 0.0;
    ax[i] = ay[i] = az[i] = 0.0;
    m[i] = 0.0;
    h[i] = -1.0;
}

// Eq. 7 per member: h = cbrt(m / m_min) h_min with the member's own m_min.
__global__ void ens_softening_kernel(const int64_t *__restrict__ off, const int64_t *__restrict__ nreal,
                                     const double *__restrict__ hmin, const double *__restrict__ m,
                                     double *__restrict__ h) {
    __shared__ double red[256];
    const int s = blockIdx.x;
    double v = 1e300;
    for (int64_t i = off[s] + threadIdx.x; i < off[s] + nreal[s]; i += blockDim.x) v = fmin(v, m[i]);
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const double mmin = red[0];
    if (hmin[s] <= 0.0) return;  // caller-supplied softening for this member
    for (int64_t i = off[s] + threadIdx.x; i < off[s] + nreal[s]; i += blockDim.x)
        h[i] = cbrt(m[i] / mmin) * hmin[s];
}

// Half kick with the member's cosmology (Eq. 8 comoving, or static).
__global__ void ens_kick_kernel(int64_t NP, const int *__restrict__ sim, const double *__restrict__ h,
                                const double *__restrict__ x, const double *__restrict__ y,
                                const double *__restrict__ z, double *__restrict__ vx,
                                double *__restrict__ vy, double *__restrict__ vz,
                                const double *__restrict__ ax, const double *__restrict__ ay,
                                const double *__restrict__ az, const double *__restrict__ sc,
                                const Cosmo *__restrict__ cos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP || h[i] < 0.0) return;
    const int s = sim[i];
    const Cosmo c = cos[s];
    const double *S = sc + s * SC_COUNT;
    const double hdt = 0.5 * S[SC_DT];
    if (!c.comoving) {
        vx[i] += hdt * ax[i];
        vy[i] += hdt * ay[i];
        vz[i] += hdt * az[i];
        return;
    }
    const double a = S[SC_A], H = S[SC_H];
    const double ia3 = 1.0 / (a * a * a);
    const double bg = 0.5 * c.Om * c.H0 * c.H0;
    const double Ax = ax[i] * ia3 - 2.0 * H * vx[i] + bg * x[i] * ia3;
    const double Ay = ay[i] * ia3 - 2.0 * H * vy[i] + bg * y[i] * ia3;
    const double Az = az[i] * ia3 - 2.0 * H * vz[i] + bg * z[i] * ia3;
    vx[i] += hdt * Ax;
    vy[i] += hdt * Ay;
    vz[i] += hdt * Az;
}

__global__ void ens_drift_kernel(int64_t NP, const int *__restrict__ sim, const double *__restrict__ h,
                                 double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                                 const double *__restrict__ vx, const double *__restrict__ vy,
                                 const double *__restrict__ vz, const double *__restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP || h[i] < 0.0) return;
    const double dt = sc[sim[i] * SC_COUNT + SC_DT];
    x[i] += vx[i] * dt;
    y[i] += vy[i] * dt;
    z[i] += vz[i] * dt;
}

// Per member: RK4 step of da/dt = a H(a) (Eq. 1), then t, step counters.
__global__ void ens_rk4_kernel(int nsims, double *__restrict__ sc, const Cosmo *__restrict__ cos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsims) return;
    double *S = sc + s * SC_COUNT;
    const Cosmo c = cos[s];
    const double dt = S[SC_DT];
    if (c.comoving) {
        double a = S[SC_A];
        const double k1 = a * hubble_e(a, c);
        const double a2 = a + 0.5 * dt * k1;
        const double k2 = a2 * hubble_e(a2, c);
        const double a3 = a + 0.5 * dt * k2;
        const double k3 = a3 * hubble_e(a3, c);
        const double a4 = a + dt * k3;
        const double k4 = a4 * hubble_e(a4, c);
        a = a + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
        S[SC_A] = a;
        S[SC_H] = hubble_e(a, c);
    }
    S[SC_T] += dt;
    S[SC_STEP] += 1.0;
    S[SC_RUN] += 1.0;
}

__global__ void ens_set_dt_kernel(int nsims, double *__restrict__ sc, const double *__restrict__ dts,
                                  int cap) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsims) return;
    double *S = sc + s * SC_COUNT;
    S[SC_DT] = dts[(int64_t)s * cap + (int64_t)S[SC_RUN]];
}

__global__ void ens_reset_run_kernel(int nsims, double *__restrict__ sc) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsims) sc[s * SC_COUNT + SC_RUN] = 0.0;
}

steps_status ens_sync(steps_ens *e) {
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    int w[3] = {0, 0, 0};  // error word, validation flags, non-finite word
    STEPS_CUDA(cudaMemcpy(w, e->err, sizeof(w), cudaMemcpyDeviceToHost));
    if (w[0]) {
        STEPS_CUDA(cudaMemset(e->err, 0, sizeof(int)));
        set_error("a bounded device-side wait ran out (error word %d); the kernel exited early", w[0]);
        return (steps_status)w[0];
    }
    if (w[2]) {
        STEPS_CUDA(cudaMemset(e->nonfinite, 0, sizeof(int)));
        set_error("a computed force is NaN or Inf (FP32 overflow of the inputs' scale?)");
        return STEPS_ENONFINITE;
    }
    return STEPS_OK;
}

// Make variant k the active one: tile size, staging views, the system table
// and the stream-K plan (buffers were sized for every candidate at init).
steps_status ens_configure(steps_ens *e, int k) {
    const Variant &v = variant(k);
    const int64_t T = 32 * v.KI;
    e->variant = k;
    e->stg.T = (int)T;
    e->stg.ntile = e->NP / T;
    e->stg.fdup = v.form == 1 ? e->fdup_buf : nullptr;
    e->stg.sdup = v.form == 2 ? e->sdup_buf : nullptr;
    const bool sub = v.form == 2 && v.sub;
    e->stg.tbox_hc = sub ? e->hbox_c : nullptr;
    e->stg.tbox_he = sub ? e->hbox_e : nullptr;
    e->nr.submask = sub ? e->submask : nullptr;
    e->stg.qmax = e->qmax;
    std::vector<SimDesc> descs(e->nsims);
    for (int s = 0; s < e->nsims; ++s) {
        descs[s] = SimDesc{};
        descs[s].tile_off = e->off[s] / T;
        descs[s].ntile = (e->off[s + 1] - e->off[s]) / T;
    }
    int64_t bits_words = 0;
    e->plan = plan_force_multi(k, e->num_sms, descs.data(), e->nsims, e->dsims, &bits_words);
    e->nr.bits_words = bits_words;
    e->nr.cap_items = 8 * e->stg.ntile;
    STEPS_CUDA(cudaMemcpyAsync(e->dsims, descs.data(), sizeof(SimDesc) * e->nsims, cudaMemcpyHostToDevice, e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    return STEPS_OK;
}

steps_status ens_resort(steps_ens *e) {
    int launches = 0;
    STEPS_CUDA(ensemble_sort(e->nsims, e->doff, e->NP, e->sim, e->x, e->y, e->z, e->h, e->srt, e->st,
                             &launches));
    double **arrs[] = {&e->x, &e->y, &e->z, &e->vx, &e->vy, &e->vz, &e->m, &e->h, &e->ax, &e->ay, &e->az};
    for (double **a : arrs) {
        STEPS_CUDA(gather_f64(e->NP, e->srt.vals, *a, e->srt.tmp, e->st));
        std::swap(*a, e->srt.tmp);
    }
    STEPS_CUDA(gather_i64(e->NP, e->srt.vals, e->perm, e->srt.tmpi, e->st));
    std::swap(e->perm, e->srt.tmpi);
    e->since_sort = 0;
    return STEPS_OK;
}

steps_status ens_forces(steps_ens *e) {
    launch_stage(e->stg, e->x, e->y, e->z, e->m, e->h, e->st);
    STEPS_CUDA(cudaGetLastError());
    STEPS_CUDA(launch_force_f32(e->plan, e->stg, e->partial, e->nr, e->err, e->stats, kAlpha, e->wait_ns,
                                e->num_sms, e->st));
    STEPS_CUDA(launch_fixup(e->plan, e->stg, e->partial, e->nr, 1.0, e->ax, e->ay, e->az, e->st));
    // non-finite result check (read at the next synchronising call)
    STEPS_CUDA(launch_check_finite3(e->NP, e->ax, e->ay, e->az, e->nonfinite, e->st, e->h));
    return STEPS_OK;
}

// G differs per member in general; the fixup applied G = 1, so scale here.
__global__ void ens_scale_g_kernel(int64_t NP, const int *__restrict__ sim, const Cosmo *__restrict__ cos,
                                   double *ax, double *ay, double *az) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const double G = cos[sim[i]].G;
    ax[i] *= G;
    ay[i] *= G;
    az[i] *= G;
}

steps_status ens_forces_g(steps_ens *e) {
    STEPS_TRY(ens_forces(e));
    ens_scale_g_kernel<<<blocks_for(e->NP, 256), 256, 0, e->st>>>(e->NP, e->sim, e->cosmo, e->ax, e->ay,
                                                                    e->az);
    STEPS_CUDA(cudaGetLastError());
    return STEPS_OK;
}

steps_status ens_step(steps_ens *e, bool do_sort) {
    const unsigned b = blocks_for(e->NP, 256);
    const unsigned bs = blocks_for(e->nsims, 64);
    ens_set_dt_kernel<<<bs, 64, 0, e->st>>>(e->nsims, e->sc, e->dts, e->dts_cap);
    ens_kick_kernel<<<b, 256, 0, e->st>>>(e->NP, e->sim, e->h, e->x, e->y, e->z, e->vx, e->vy, e->vz, e->ax,
                                          e->ay, e->az, e->sc, e->cosmo);
    ens_drift_kernel<<<b, 256, 0, e->st>>>(e->NP, e->sim, e->h, e->x, e->y, e->z, e->vx, e->vy, e->vz, e->sc);
    ens_rk4_kernel<<<bs, 64, 0, e->st>>>(e->nsims, e->sc, e->cosmo);
    STEPS_CUDA(cudaGetLastError());
    if (do_sort) STEPS_TRY(ens_resort(e));
    STEPS_TRY(ens_forces_g(e));
    ens_kick_kernel<<<b, 256, 0, e->st>>>(e->NP, e->sim, e->h, e->x, e->y, e->z, e->vx, e->vy, e->vz, e->ax,
                                          e->ay, e->az, e->sc, e->cosmo);
    STEPS_CUDA(cudaGetLastError());
    return STEPS_OK;
}

// Autotuner: time one force evaluation of the whole ensemble (a warm-up,
// then the median of three) with every candidate variant on the members'
// actual initial state and keep the fastest.
steps_status ens_autotune(steps_ens *e) {
    if (e->candidates.size() < 2) return STEPS_OK;
    constexpr int kReps = 3;
    cudaEvent_t ev[kReps + 1];
    for (auto &x : ev) STEPS_CUDA(cudaEventCreate(&x));
    int best = e->candidates[0];
    float best_ms = 1e30f;
    steps_status st = STEPS_OK;
    for (int k : e->candidates) {
        if (st != STEPS_OK) break;
        st = ens_configure(e, k);
        if (st == STEPS_OK) st = ens_forces(e);  // warm-up
        for (int r = 0; r < kReps && st == STEPS_OK; ++r) {
            if (cudaEventRecord(ev[r], e->st) != cudaSuccess) st = STEPS_ECUDA;
            if (st == STEPS_OK) st = ens_forces(e);
        }
        if (st == STEPS_OK && cudaEventRecord(ev[kReps], e->st) != cudaSuccess) st = STEPS_ECUDA;
        if (st == STEPS_OK) st = ens_sync(e);
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
    for (auto &x : ev) cudaEventDestroy(x);
    STEPS_TRY(st);
    STEPS_CUDA(cudaMemsetAsync(e->stats, 0, 2 * sizeof(unsigned long long), e->st));
    return ens_configure(e, best);
}

void ens_release(steps_ens *e) {
    if (!e) return;
    if (e->st) cudaStreamSynchronize(e->st);
    for (auto &a : e->allocs) counted_free(a.first, a.second);
    if (e->own_stream && e->st) cudaStreamDestroy(e->st);
    delete e;
}

steps_status ens_init_impl(steps_ens *e, const double *const *pos, const double *const *vel,
                           const double *const *mass, const double *const *soft, const double *h_min,
                           const double *t0, const double *a0, const steps_config *cfgs) {
    int dev = 0;
    STEPS_CUDA(cudaGetDevice(&dev));
    STEPS_CUDA(cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, dev));
    // candidates: the requested variant, or every variant of the summation mode
    // whose target block divides the common padding
    int64_t BI = kEnsPad;
    if (e->variant >= 0) {
        e->candidates.assign(1, e->variant);
        const Variant &v = variant(e->variant);
        const int64_t bi = (int64_t)v.W * 32 * v.KI;
        BI = kEnsPad % bi == 0 ? kEnsPad : bi;
    } else {
        const bool comp = cfgs[0].prec != STEPS_F32_NAIVE;
        for (int k = 0; k < num_variants(); ++k) {
            const Variant &v = variant(k);
            if (v.comp == comp && kEnsPad % ((int64_t)v.W * 32 * v.KI) == 0) e->candidates.push_back(k);
        }
        if (e->candidates.empty()) {
            set_error("no force variant fits the ensemble layout");
            return STEPS_EUNSUPPORTED;
        }
    }
    e->pad = BI;
    int tmin = 1 << 30;
    bool any_exp = false, any_sym = false;
    for (int k : e->candidates) {
        tmin = std::min(tmin, 32 * variant(k).KI);
        any_exp |= variant(k).form == 1;
        any_sym |= variant(k).form == 2;
    }
    e->off.assign(e->nsims + 1, 0);
    int64_t nmax = 0;
    for (int s = 0; s < e->nsims; ++s) {
        e->off[s + 1] = e->off[s] + (e->n[s] + BI - 1) / BI * BI;
        nmax = std::max(nmax, e->n[s]);
    }
    e->NP = e->off[e->nsims];
    const int64_t NP = e->NP;
    double **soa[] = {&e->x, &e->y, &e->z, &e->vx, &e->vy, &e->vz, &e->m, &e->h, &e->ax, &e->ay, &e->az};
    for (double **a : soa) STEPS_TRY(ens_alloc(e, a, NP));
    STEPS_TRY(ens_alloc(e, &e->perm, NP));
    STEPS_TRY(ens_alloc(e, &e->sim, NP));
    STEPS_TRY(ens_alloc(e, &e->doff, e->nsims + 1));
    STEPS_TRY(ens_alloc(e, &e->sc, (size_t)e->nsims * SC_COUNT));
    STEPS_TRY(ens_alloc(e, &e->cosmo, e->nsims));
    STEPS_TRY(ens_alloc(e, &e->err, 4));
    e->nonfinite = e->err + 2;
    STEPS_TRY(ens_alloc(e, &e->stats, 2));
    e->tmp3_cap = 3 * nmax;
    STEPS_TRY(ens_alloc(e, &e->tmp3, e->tmp3_cap));
    STEPS_CUDA(cudaMemsetAsync(e->err, 0, 4 * sizeof(int), e->st));
    STEPS_CUDA(cudaMemsetAsync(e->stats, 0, 2 * sizeof(unsigned long long), e->st));
    // staging, tables, near field, sort scratch: sized for every candidate
    const int64_t ntile = NP / tmin;  // most tiles any candidate uses
    STEPS_TRY(ens_alloc(e, &e->stg.jdup, 2 * NP));
    STEPS_TRY(ens_alloc(e, &e->stg.rdup, 2 * NP));
    if (any_exp) STEPS_TRY(ens_alloc(e, &e->fdup_buf, 4 * NP));
    if (any_sym) {
        STEPS_TRY(ens_alloc(e, &e->sdup_buf, 2 * NP));
        STEPS_TRY(ens_alloc(e, &e->nr.sym_acc, 3 * NP));
        STEPS_TRY(ens_alloc(e, &e->nr.sym_next, 1));
        STEPS_TRY(ens_alloc(e, &e->nr.tscale, ntile));
        STEPS_TRY(ens_alloc(e, &e->nr.tinv, ntile));
        // sub-blocks of 256-particle tiles: half boxes and a mask per tile pair of a member
        int64_t mbytes = 0;
        for (int s = 0; s < e->nsims; ++s) {
            const int64_t nt = (e->off[s + 1] - e->off[s]) / 256;
            mbytes += nt * ((nt + 31) / 32) * 32;  // a byte per bit of the member's near bitmap
        }
        STEPS_TRY(ens_alloc(e, &e->hbox_c, 2 * (NP / 256) + 2));
        STEPS_TRY(ens_alloc(e, &e->hbox_e, 2 * (NP / 256) + 2));
        STEPS_TRY(ens_alloc(e, &e->submask, mbytes + 16));
    }
    STEPS_TRY(ens_alloc(e, &e->qmax, 1));
    e->nr.nonfinite = e->nonfinite;
    STEPS_TRY(ens_alloc(e, &e->stg.tbox_c, ntile));
    STEPS_TRY(ens_alloc(e, &e->stg.tbox_e, ntile));
    e->stg.n = NP;  // validity comes from h >= 0
    e->stg.np = NP;
    STEPS_TRY(ens_alloc(e, &e->dsims, e->nsims));
    size_t partial_max = 16;
    int64_t bits_max = 1;
    for (int k : e->candidates) {
        const int64_t T = 32 * variant(k).KI;
        std::vector<SimDesc> descs(e->nsims);
        for (int s = 0; s < e->nsims; ++s) {
            descs[s] = SimDesc{};
            descs[s].tile_off = e->off[s] / T;
            descs[s].ntile = (e->off[s + 1] - e->off[s]) / T;
        }
        int64_t bw = 0;
        const ForcePlan pl = plan_force_multi(k, e->num_sms, descs.data(), e->nsims, e->dsims, &bw);
        partial_max = std::max(partial_max, pl.partial_elems);
        bits_max = std::max(bits_max, bw);
    }
    STEPS_TRY(ens_alloc(e, &e->partial, partial_max));
    STEPS_TRY(ens_alloc(e, &e->nr.bits, (size_t)bits_max));
    STEPS_TRY(ens_alloc(e, &e->nr.cnt, ntile));
    STEPS_TRY(ens_alloc(e, &e->nr.item_off, ntile + 1));
    STEPS_TRY(ens_alloc(e, &e->nr.meta, 4));
    STEPS_TRY(ens_alloc(e, &e->nr.item_part, (size_t)24 * NP));
    STEPS_TRY(ens_configure(e, e->candidates[0]));
    int64_t p2 = 2;
    while (p2 < NP) p2 <<= 1;
    e->srt.npow2 = p2;
    STEPS_TRY(ens_alloc(e, &e->srt.keys, p2));
    STEPS_TRY(ens_alloc(e, &e->srt.vals, p2));
    STEPS_TRY(ens_alloc(e, &e->srt.bbox, (size_t)6 * e->nsims));
    STEPS_TRY(ens_alloc(e, &e->srt.tmp, NP));
    STEPS_TRY(ens_alloc(e, &e->srt.tmpi, NP));

    // members' inputs: pad, then copy each member's real particles in
    std::vector<int64_t> nreal(e->n.begin(), e->n.end());
    int64_t *dn = nullptr;
    double *dhmin = nullptr;
    STEPS_TRY(ens_alloc(e, &dn, e->nsims));
    STEPS_TRY(ens_alloc(e, &dhmin, e->nsims));
    STEPS_CUDA(cudaMemcpyAsync(e->doff, e->off.data(), sizeof(int64_t) * (e->nsims + 1), cudaMemcpyHostToDevice, e->st));
    STEPS_CUDA(cudaMemcpyAsync(dn, nreal.data(), sizeof(int64_t) * e->nsims, cudaMemcpyHostToDevice, e->st));
    int64_t maxpad = 0;
    for (int s = 0; s < e->nsims; ++s) maxpad = std::max(maxpad, e->off[s + 1] - e->off[s]);
    ens_pad_kernel<<<dim3(blocks_for(maxpad, 256), e->nsims), 256, 0, e->st>>>(
        e->nsims, e->doff, dn, e->sim, e->perm, e->x, e->y, e->z, e->vx, e->vy, e->vz, e->m, e->h, e->ax,
        e->ay, e->az);
    STEPS_CUDA(cudaGetLastError());
    std::vector<double> hm(e->nsims, 0.0);
    int *flag = e->err + 1;
    for (int s = 0; s < e->nsims; ++s) {
        const int64_t o = e->off[s], ns = e->n[s];
        STEPS_CUDA(cudaMemcpyAsync(e->tmp3, pos[s], sizeof(double) * 3 * ns, cudaMemcpyDefault, e->st));
        STEPS_CUDA(launch_check_finite(3 * ns, e->tmp3, 0, flag, e->st));
        STEPS_CUDA(launch_split3(ns, e->tmp3, e->x + o, e->y + o, e->z + o, e->st));
        if (vel && vel[s]) {
            STEPS_CUDA(cudaMemcpyAsync(e->tmp3, vel[s], sizeof(double) * 3 * ns, cudaMemcpyDefault, e->st));
            STEPS_CUDA(launch_check_finite(3 * ns, e->tmp3, 0, flag, e->st));
            STEPS_CUDA(launch_split3(ns, e->tmp3, e->vx + o, e->vy + o, e->vz + o, e->st));
        }
        STEPS_CUDA(cudaMemcpyAsync(e->m + o, mass[s], sizeof(double) * ns, cudaMemcpyDefault, e->st));
        STEPS_CUDA(launch_check_finite(ns, e->m + o, 1, flag, e->st));
        if (soft && soft[s]) {
            STEPS_CUDA(cudaMemcpyAsync(e->h + o, soft[s], sizeof(double) * ns, cudaMemcpyDefault, e->st));
        } else {
            if (!h_min || !(h_min[s] > 0.0) || !std::isfinite(h_min[s])) {
                set_error("member %d: h_min must be finite and > 0 when its softening is not given", s);
                return STEPS_EINVAL;
            }
            hm[s] = h_min[s];
        }
        // the staging buffer is reused by the next member: finish this one first
        STEPS_CUDA(cudaStreamSynchronize(e->st));
    }
    STEPS_CUDA(cudaMemcpyAsync(dhmin, hm.data(), sizeof(double) * e->nsims, cudaMemcpyHostToDevice, e->st));
    ens_softening_kernel<<<e->nsims, 256, 0, e->st>>>(e->doff, dn, dhmin, e->m, e->h);
    STEPS_CUDA(cudaGetLastError());
    for (int s = 0; s < e->nsims; ++s)
        STEPS_CUDA(launch_check_finite(e->n[s], e->h + e->off[s], 1, flag, e->st));
    int bad = 0;
    STEPS_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    if (bad) {
        set_error("ensemble inputs: positions/velocities must be finite, masses and softening > 0");
        return STEPS_EINVAL;
    }
    // per-member cosmology and scalars
    std::vector<Cosmo> cs(e->nsims);
    std::vector<double> sc((size_t)e->nsims * SC_COUNT, 0.0);
    for (int s = 0; s < e->nsims; ++s) {
        const steps_config &c = cfgs[s];
        cs[s] = Cosmo{c.G, c.H0, c.Om, c.OL, c.Or, c.Ok, c.mode == STEPS_COMOVING ? 1 : 0};
        double *S = sc.data() + (size_t)s * SC_COUNT;
        S[SC_T] = t0 ? t0[s] : 0.0;
        S[SC_A] = cs[s].comoving ? a0[s] : 1.0;
        if (cs[s].comoving) {
            const double ia = 1.0 / a0[s];
            S[SC_H] = c.H0 * std::sqrt(c.Om * ia * ia * ia + c.Or * ia * ia * ia * ia + c.OL + c.Ok * ia * ia);
        }
    }
    STEPS_CUDA(cudaMemcpyAsync(e->cosmo, cs.data(), sizeof(Cosmo) * e->nsims, cudaMemcpyHostToDevice, e->st));
    STEPS_CUDA(cudaMemcpyAsync(e->sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, e->st));
    STEPS_TRY(ens_resort(e));
    STEPS_TRY(ens_autotune(e));
    STEPS_TRY(ens_forces_g(e));
    return ens_sync(e);
}

}  // namespace

extern "C" {

steps_status steps_ensemble_init(steps_ens **out, int nsims, const int64_t *n, const double *const *pos,
                                 const double *const *vel, const double *const *mass,
                                 const double *const *soft, const double *h_min, const double *t0,
                                 const double *a0, const steps_config *cfgs, void *cuda_stream) {
    if (!out) {
        set_error("out is NULL");
        return STEPS_EINVAL;
    }
    *out = nullptr;
    if (nsims <= 0 || nsims > 4096 || !n || !pos || !mass || !cfgs) {
        set_error("nsims must be in [1, 4096] and n, pos, mass, cfgs are required");
        return STEPS_EINVAL;
    }
    for (int s = 0; s < nsims; ++s) {
        if (n[s] <= 0 || !pos[s] || !mass[s]) {
            set_error("member %d: n must be > 0 and pos, mass given", s);
            return STEPS_EINVAL;
        }
        if (cfgs[s].mode != STEPS_STATIC && cfgs[s].mode != STEPS_COMOVING) {
            set_error("member %d: unknown mode", s);
            return STEPS_EINVAL;
        }
        if (cfgs[s].mode == STEPS_COMOVING && (!a0 || !(a0[s] > 0.0) || !std::isfinite(a0[s]))) {
            set_error("member %d: a0 must be finite and > 0 in comoving mode", s);
            return STEPS_EINVAL;
        }
        if (!std::isfinite(cfgs[s].G) || !std::isfinite(cfgs[s].H0)) {
            set_error("member %d: G and H0 must be finite", s);
            return STEPS_EINVAL;
        }
    }
    if (cfgs[0].prec == STEPS_F64) {
        set_error("ensembles run the FP32 path (STEPS_F32_COMP or STEPS_F32_NAIVE)");
        return STEPS_EUNSUPPORTED;
    }
    steps_ens *e = new (std::nothrow) steps_ens();
    if (!e) {
        set_error("host allocation failed");
        return STEPS_ENOMEM;
    }
    e->nsims = nsims;
    e->n.assign(n, n + nsims);
    e->resort_every = cfgs[0].resort_every > 0 ? cfgs[0].resort_every : 8;
    const bool comp = cfgs[0].prec != STEPS_F32_NAIVE;
    e->variant = -1;  // -1: tuned at init among the candidates
    if (cfgs[0].tile_override > 0 && cfgs[0].tile_override <= num_variants()) {
        e->variant = cfgs[0].tile_override - 1;
        if (variant(e->variant).comp != comp) {
            set_error("tile_override %d does not match the precision mode", cfgs[0].tile_override);
            delete e;
            return STEPS_EINVAL;
        }
    }
    if (cuda_stream) {
        e->st = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t ce = cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            delete e;
            return cuda_status(ce, "cudaStreamCreate");
        }
        e->own_stream = true;
    }
    steps_status s = ens_init_impl(e, pos, vel, mass, soft, h_min, t0, a0, cfgs);
    if (s != STEPS_OK) {
        ens_release(e);
        return s;
    }
    *out = e;
    return STEPS_OK;
}

steps_status steps_ensemble_run(steps_ens *e, int nsteps, const double *dts) {
    if (!e || nsteps < 0 || (nsteps > 0 && !dts)) {
        set_error("bad arguments to steps_ensemble_run");
        return STEPS_EINVAL;
    }
    if (nsteps == 0) return STEPS_OK;
    for (int64_t k = 0; k < (int64_t)nsteps * e->nsims; ++k) {
        if (!std::isfinite(dts[k])) {
            set_error("dts[%lld] is not finite", (long long)k);
            return STEPS_EINVAL;
        }
    }
    if (nsteps > e->dts_cap) {
        for (auto it = e->allocs.begin(); it != e->allocs.end(); ++it) {
            if (it->first == e->dts) {
                counted_free(it->first, it->second);
                e->allocs.erase(it);
                break;
            }
        }
        e->dts = nullptr;
        e->dts_cap = 0;
        STEPS_TRY(ens_alloc(e, &e->dts, (size_t)nsteps * e->nsims));
        e->dts_cap = nsteps;
    }
    // dts is [nsims][nsteps]; the device copy uses row stride dts_cap
    STEPS_CUDA(cudaMemcpy2DAsync(e->dts, sizeof(double) * e->dts_cap, dts, sizeof(double) * nsteps,
                                 sizeof(double) * nsteps, e->nsims, cudaMemcpyDefault, e->st));
    ens_reset_run_kernel<<<blocks_for(e->nsims, 64), 64, 0, e->st>>>(e->nsims, e->sc);
    STEPS_CUDA(cudaGetLastError());
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    cudaGraphExec_t plain = nullptr;
    steps_status s = STEPS_OK;
    for (int k = 0; k < nsteps && s == STEPS_OK; ++k) {
        const bool do_sort = ++e->since_sort >= e->resort_every;
        if (do_sort) {
            // a sorting step swaps buffers: run it directly, re-capture after
            if (plain) {
                cudaGraphExecDestroy(plain);
                plain = nullptr;
            }
            s = ens_step(e, true);
            continue;
        }
        if (!plain) {
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal);
            if (ce != cudaSuccess) {
                s = cuda_status(ce, "cudaStreamBeginCapture");
                break;
            }
            steps_status si = ens_step(e, false);
            ce = cudaStreamEndCapture(e->st, &g);
            if (si != STEPS_OK) {
                if (g) cudaGraphDestroy(g);
                s = si;
                break;
            }
            if (ce != cudaSuccess) {
                s = cuda_status(ce, "cudaStreamEndCapture");
                break;
            }
            ce = cudaGraphInstantiate(&plain, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                s = cuda_status(ce, "cudaGraphInstantiate");
                break;
            }
        }
        cudaError_t ce = cudaGraphLaunch(plain, e->st);
        if (ce != cudaSuccess) s = cuda_status(ce, "cudaGraphLaunch");
    }
    if (plain) cudaGraphExecDestroy(plain);
    if (s != STEPS_OK) return s;
    return ens_sync(e);
}

steps_status steps_ensemble_get_state(steps_ens *e, int s, double *pos, double *vel, double *acc,
                                      double *t, double *a) {
    if (!e || s < 0 || s >= e->nsims) {
        set_error("ensemble is NULL or member index out of range");
        return STEPS_EINVAL;
    }
    const int64_t o = e->off[s], ns = e->n[s];
    const double *src[3][3] = {{e->x, e->y, e->z}, {e->vx, e->vy, e->vz}, {e->ax, e->ay, e->az}};
    double *dst[3] = {pos, vel, acc};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        STEPS_CUDA(launch_scatter3(ns, e->perm + o, src[k][0] + o, src[k][1] + o, src[k][2] + o, e->tmp3, e->st));
        STEPS_CUDA(cudaMemcpyAsync(dst[k], e->tmp3, sizeof(double) * 3 * ns, cudaMemcpyDefault, e->st));
        STEPS_CUDA(cudaStreamSynchronize(e->st));
    }
    double S[SC_COUNT];
    STEPS_CUDA(cudaMemcpyAsync(S, e->sc + (size_t)s * SC_COUNT, sizeof(S), cudaMemcpyDeviceToHost, e->st));
    STEPS_TRY(ens_sync(e));
    if (t) *t = S[SC_T];
    if (a) *a = S[SC_A];
    return STEPS_OK;
}

steps_status steps_ensemble_stats(steps_ens *e, int64_t *total_particles, uint64_t *near_pairs,
                                  uint64_t *all_pairs) {
    if (!e) {
        set_error("ensemble is NULL");
        return STEPS_EINVAL;
    }
    unsigned long long h[2] = {0, 0};
    STEPS_CUDA(cudaMemcpyAsync(h, e->stats, sizeof(h), cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaMemsetAsync(e->stats, 0, sizeof(h), e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    if (total_particles) *total_particles = e->NP;
    if (near_pairs) *near_pairs = h[0];
    if (all_pairs) *all_pairs = h[1];
    return STEPS_OK;
}

steps_status steps_ensemble_variant(steps_ens *e, int *k) {
    if (!e || !k) {
        set_error("ensemble and k are required");
        return STEPS_EINVAL;
    }
    *k = e->variant;
    return STEPS_OK;
}

void steps_ensemble_free(steps_ens *e) { ens_release(e); }

}  // extern "C"

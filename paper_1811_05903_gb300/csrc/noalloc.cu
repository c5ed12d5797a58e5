// steps_forces_noalloc: the FP32 compensated pair term for small systems with
// every scratch buffer carved out of one fixed-size device array compiled
// into this library, so the call performs no device allocation.
//
// Who needs this: host code that cannot call cudaMalloc/cudaFree around a
// force evaluation -- for example a caller running inside a larger
// application whose caching allocator already holds the device memory (a
// fresh cudaMalloc could fail or fragment it), or a tight per-step loop of a
// bigger simulation that must not pick up the implicit device-wide
// synchronisation cudaMalloc/cudaFree can cause.  Such a caller still
// provides its own input and output buffers in device memory.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; everything that must start at zero is cleared by the call.
// Calls whose work overlaps on the GPU (two streams, or two host threads on
// one device) race on that array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "steps_internal.h"

namespace steps {

namespace {

// Largest system the static scratch serves, and the scratch size.  The far
// and near kernels use the 64-particle-tile compensated variant; particles
// are tiled in caller order (no spatial sort), which is always correct and
// only moves more tile pairs to the near-field kernel.
constexpr int64_t kMaxN = STEPS_NOALLOC_MAX_N;
constexpr int kKI = 2, kW = 8;
constexpr int64_t kT = 32 * kKI, kBI = kW * kT;
constexpr int64_t kNp = (kMaxN + kBI - 1) / kBI * kBI;
constexpr int64_t kNtile = kNp / kT;
constexpr int64_t kWords = (kNtile + 31) / 32;
constexpr int64_t kPartialDoubles = (int64_t)1 << 19;  // 4 MiB of far-field partial sums

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct Layout {
    size_t soa, acc, perm, jdup, rdup, tbox_c, tbox_e, partial, bits, cnt, item_off, meta, item_part,
        err, stats, mmin, sim, total;
};

constexpr Layout make_layout() {
    Layout L{};
    size_t o = 0;
    L.soa = o;       o = align256(o + sizeof(double) * 5 * kNp);   // x y z m h
    L.acc = o;       o = align256(o + sizeof(double) * 3 * kNp);   // ax ay az
    L.perm = o;      o = align256(o + sizeof(int64_t) * kNp);
    L.jdup = o;      o = align256(o + 16 * 2 * kNp);
    L.rdup = o;      o = align256(o + 16 * 2 * kNp);
    L.tbox_c = o;    o = align256(o + 16 * kNtile);
    L.tbox_e = o;    o = align256(o + 16 * kNtile);
    L.partial = o;   o = align256(o + sizeof(double) * kPartialDoubles);
    L.bits = o;      o = align256(o + sizeof(uint32_t) * kNtile * kWords);
    L.cnt = o;       o = align256(o + sizeof(int) * kNtile);
    L.item_off = o;  o = align256(o + sizeof(int64_t) * (kNtile + 1));
    L.meta = o;      o = align256(o + sizeof(int64_t) * 4);
    L.item_part = o; o = align256(o + sizeof(double) * 24 * kNp);
    L.err = o;       o = align256(o + sizeof(int) * 2);
    L.stats = o;     o = align256(o + sizeof(unsigned long long) * 2);
    L.mmin = o;      o = align256(o + sizeof(double));
    L.sim = o;       o = align256(o + sizeof(SimDesc));
    L.total = o;
    return L;
}

constexpr Layout kLayout = make_layout();

// The scratch array itself.  Its name is only a host-side handle: host code
// obtains the device address with cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kLayout.total];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

steps_status scratch_for_device(unsigned char **out) {
    int dev = 0;
    STEPS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
        return STEPS_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        STEPS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return STEPS_OK;
}

// Device memory of the current device, or managed memory.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

int compensated_small_variant() {
    for (int k = 0; k < num_variants(); ++k)
        if (variant(k).comp && variant(k).form == 0 && variant(k).KI == kKI && variant(k).W == kW) return k;
    return -1;
}

}  // namespace

}  // namespace steps

using namespace steps;

extern "C" steps_status steps_forces_noalloc(int64_t n, const double *pos, const double *mass,
                                             const double *soft, double h_min, double G,
                                             double *acc_out, void *cuda_stream) {
    if (n <= 0 || n > kMaxN) {
        set_error("n = %lld is outside [1, %lld], the size this entry point's fixed scratch serves",
                  (long long)n, (long long)kMaxN);
        return STEPS_EINVAL;
    }
    if (!pos || !mass || !acc_out || !std::isfinite(G)) {
        set_error("pos, mass and acc_out are required and G must be finite");
        return STEPS_EINVAL;
    }
    if (!soft && !(h_min > 0.0 && std::isfinite(h_min))) {
        set_error("h_min must be finite and > 0 when soft is NULL");
        return STEPS_EINVAL;
    }
    int dev = 0;
    STEPS_CUDA(cudaGetDevice(&dev));
    if (!on_device(pos, dev) || !on_device(mass, dev) || !on_device(acc_out, dev) || (soft && !on_device(soft, dev))) {
        set_error("pos, mass, soft and acc_out must be device pointers on the current device");
        return STEPS_EINVAL;
    }
    const int k = compensated_small_variant();
    if (k < 0) {
        set_error("the 64-particle-tile compensated force variant is not built");
        return STEPS_EUNSUPPORTED;
    }
    unsigned char *base = nullptr;
    STEPS_TRY(scratch_for_device(&base));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const Layout &L = kLayout;
    double *soa = reinterpret_cast<double *>(base + L.soa);
    double *x = soa, *y = soa + kNp, *z = soa + 2 * kNp, *m = soa + 3 * kNp, *h = soa + 4 * kNp;
    double *acc = reinterpret_cast<double *>(base + L.acc);
    double *ax = acc, *ay = acc + kNp, *az = acc + 2 * kNp;
    int64_t *perm = reinterpret_cast<int64_t *>(base + L.perm);
    int *err = reinterpret_cast<int *>(base + L.err);
    int *flag = err + 1;
    int num_sms = 0;
    STEPS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

    // inputs into the scratch SoA (caller order), validated like steps_init
    STEPS_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
    STEPS_CUDA(launch_split3(n, pos, x, y, z, st));
    STEPS_CUDA(cudaMemcpyAsync(m, mass, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (soft)
        STEPS_CUDA(cudaMemcpyAsync(h, soft, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    else
        STEPS_CUDA(launch_softening(n, m, h_min, h, reinterpret_cast<double *>(base + L.mmin), st));
    STEPS_CUDA(launch_check_finite(n, x, 0, flag, st));
    STEPS_CUDA(launch_check_finite(n, y, 0, flag, st));
    STEPS_CUDA(launch_check_finite(n, z, 0, flag, st));
    STEPS_CUDA(launch_check_finite(n, m, 1, flag, st));
    STEPS_CUDA(launch_check_finite(n, h, 1, flag, st));
    // the validation flags are read with the error word at the one synchronisation at the end
    STEPS_CUDA(launch_iota(n, perm, st));

    // staging and a stream-K plan whose partial sums fit the fixed scratch
    Staging s;
    s.n = n;
    s.np = (n + kBI - 1) / kBI * kBI;
    s.T = (int)kT;
    s.ntile = s.np / kT;
    s.jdup = reinterpret_cast<float4 *>(base + L.jdup);
    s.rdup = reinterpret_cast<float4 *>(base + L.rdup);
    s.tbox_c = reinterpret_cast<float4 *>(base + L.tbox_c);
    s.tbox_e = reinterpret_cast<float4 *>(base + L.tbox_e);
    SimDesc sd{};
    sd.tile_off = 0;
    sd.ntile = s.ntile;
    sd.unit_off = 0;
    sd.blk_off = 0;
    sd.bits_off = 0;
    sd.words = (s.ntile + 31) / 32;
    SimDesc *dsim = reinterpret_cast<SimDesc *>(base + L.sim);
    STEPS_CUDA(cudaMemcpyAsync(dsim, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    ForcePlan p;
    p.variant = k;
    p.B_I = (int)kBI;
    p.niblk = s.np / kBI;
    p.units = p.niblk * s.ntile;
    p.sims = dsim;
    p.nsims = 1;
    int64_t grid = std::min<int64_t>(p.units, (int64_t)num_sms * 4);
    for (;;) {
        const int64_t per_cta = (p.units + grid - 1) / grid;
        const int64_t smax = (per_cta + s.ntile - 1) / s.ntile + 1;
        if (grid * smax * 3 * kBI <= kPartialDoubles || grid == 1) {
            p.grid = (int)grid;
            p.smax = (int)smax;
            break;
        }
        grid = (grid + 1) / 2;
    }
    p.partial_elems = (size_t)p.grid * p.smax * 3 * kBI;
    NearScratch nr;
    nr.bits = reinterpret_cast<uint32_t *>(base + L.bits);
    nr.cnt = reinterpret_cast<int *>(base + L.cnt);
    nr.item_off = reinterpret_cast<int64_t *>(base + L.item_off);
    nr.meta = reinterpret_cast<int64_t *>(base + L.meta);
    nr.item_part = reinterpret_cast<double *>(base + L.item_part);
    nr.cap_items = 8 * (kNp / kT);
    nr.bits_words = s.ntile * sd.words;
    unsigned long long *stats = reinterpret_cast<unsigned long long *>(base + L.stats);

    launch_stage(s, x, y, z, m, h, st);
    STEPS_CUDA(cudaGetLastError());
    STEPS_CUDA(launch_force_f32(p, s, reinterpret_cast<double *>(base + L.partial), nr, err, stats,
                                0.03125f, 2000000000LL, num_sms, st));
    STEPS_CUDA(launch_fixup(p, s, reinterpret_cast<double *>(base + L.partial), nr, G, ax, ay, az, st));
    STEPS_CUDA(launch_scatter3(n, perm, ax, ay, az, acc_out, st));
    int w[2] = {0, 0};  // error word, validation flags
    STEPS_CUDA(cudaMemcpyAsync(w, err, sizeof(w), cudaMemcpyDeviceToHost, st));
    STEPS_CUDA(cudaStreamSynchronize(st));
    if (w[1]) {
        set_error("positions must be finite and masses and softening lengths finite and > 0 "
                  "(acc_out holds no result)");
        return STEPS_EINVAL;
    }
    if (w[0]) {
        set_error("a bounded device-side wait ran out (error word %d); the kernel exited early", w[0]);
        return (steps_status)w[0];
    }
    return STEPS_OK;
}

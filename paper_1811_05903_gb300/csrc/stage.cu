// Spatial sort and FP32 tile staging for the force kernels.
//
// The FP64 master state is kept in Morton (Z-curve) order so that every tile
// of T consecutive particles is spatially compact.  Each step the staging
// kernel turns the FP64 positions of a tile into FP32 offsets from that
// tile's FP32 centre (positions "relative to tile centres"), plus the tile's
// half-extents and largest softening, which the force kernel uses to prove a
// whole tile pair Newtonian (r >= h_i + h_j for every pair, Eq. 4 branch 3).
#include <algorithm>
#include <cfloat>
#include <cuda_runtime.h>
#include <stdint.h>

#include "steps_internal.h"

namespace steps {

namespace {

constexpr float kPadOffset = 1.0e15f;  // padding particles: far away, zero mass, zero softening

template <typename T, typename Op>
__device__ T block_reduce(T v, T *sbuf, Op op) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    T r = sbuf[0];
    for (int w = 1; w < nw; ++w) r = op(r, sbuf[w]);
    __syncthreads();
    return r;
}

struct MinOp {
    __device__ double operator()(double a, double b) const { return fmin(a, b); }
};
struct MaxOp {
    __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct SumOp {
    __device__ double operator()(double a, double b) const { return a + b; }
};

// Order-preserving integer key of a finite double (a < b <=> key(a) < key(b)):
// the staging kernel takes its minima and maxima on these keys, which is exact
// and runs on the integer pipe instead of GB300's narrow FP64 pipe.
__device__ __forceinline__ long long ord_key(double v) {
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

// Warp partials of K keys (xor tree, the same tree as block_reduce): key k
// takes the minimum when (kmin >> k) & 1, else the maximum.  Lane 0 stores
// the warp's results in red[k][warp]; the caller combines the warps after a
// barrier.
template <int K>
__device__ __forceinline__ void warp_keys(long long (&v)[K], unsigned kmin, long long (*red)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long u = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = ((kmin >> k) & 1) ? (u < v[k] ? u : v[k]) : (u > v[k] ? u : v[k]);
        }
        if (lane == 0) red[k][wid] = v[k];
    }
}

// Warps [w0, w1) of a stored key row combined in warp order.
__device__ __forceinline__ long long combine_keys(const long long *row, int w0, int w1, bool is_min) {
    long long r = row[w0];
    for (int w = w0 + 1; w < w1; ++w) r = is_min ? (row[w] < r ? row[w] : r) : (row[w] > r ? row[w] : r);
    return r;
}

// One CTA per tile, blockDim.x == T.
// Largest |coordinate| of the real particles into *out (the bit pattern of a
// non-negative double orders like the value, so an integer max is exact).
__global__ void absmax_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, const double *__restrict__ h, double pscale,
                              unsigned long long *__restrict__ out) {
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(h[i] < 0.0))
            v = fmax(v, fmax(fabs(x[i] * pscale), fmax(fabs(y[i] * pscale), fabs(z[i] * pscale))));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// Tile centre component rounded to the grid q (q = 0: no rounding).  With
// max|x| < 2^e and q = 2^(e-22), a rounded centre has at most 23 significant
// bits and the difference of two centres at most 24: both exact in FP32.
// qinv = 1/q (both powers of two: mid * qinv equals mid / q, without an FP64
// division).
__device__ __forceinline__ float grid_centre(double mid, double q, double qinv) {
    return q > 0.0 ? (float)(rint(mid * qinv) * q) : __double2float_rn(mid);
}

__global__ void stage_kernel(int64_t n, int T, const double *__restrict__ x,
                             const double *__restrict__ y, const double *__restrict__ z,
                             const double *__restrict__ m, const double *__restrict__ h,
                             float4 *__restrict__ jdup, float4 *__restrict__ rdup,
                             float4 *__restrict__ fdup, float4 *__restrict__ sdup,
                             const unsigned long long *__restrict__ qmax, double pscale, int qemin,
                             float4 *__restrict__ tbox_c, float4 *__restrict__ tbox_e,
                             float4 *__restrict__ tbox_hc, float4 *__restrict__ tbox_he) {
    // per-warp partials: the bounding box, largest softening and mass, then
    // the extents (the whole tile's in 0-2, the halves' in 3-5)
    __shared__ long long kbox[7][32];
    __shared__ double kmass[32];
    __shared__ long long kext[6][32];
    const int64_t tile = blockIdx.x;
    const int64_t p = tile * T + threadIdx.x;
    const bool valid = p < n && !(h[p] < 0.0);  // negative softening marks padding
    double px = 0, py = 0, pz = 0, pm = 0, ph = 0;
    if (valid) {
        px = x[p] * pscale;
        py = y[p] * pscale;
        pz = z[p] * pscale;
        pm = m[p];
        ph = h[p] * pscale;
    }
    const int wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    // the tile's warps, and the warps of this thread's half (first or last T/2)
    const int hw = nw / 2, w0 = wid < hw ? 0 : hw;
    {
        long long kv[7] = {ord_key(valid ? px : DBL_MAX),  ord_key(valid ? py : DBL_MAX),
                           ord_key(valid ? pz : DBL_MAX),  ord_key(valid ? px : -DBL_MAX),
                           ord_key(valid ? py : -DBL_MAX), ord_key(valid ? pz : -DBL_MAX),
                           ord_key(valid ? ph : 0.0)};
        warp_keys<7>(kv, 0x7u, kbox);
        double sm = valid ? pm : 0.0;
        for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if ((threadIdx.x & 31) == 0) kmass[wid] = sm;
    }
    __syncthreads();
    const double lox = key_value(combine_keys(kbox[0], 0, nw, true));
    const double loy = key_value(combine_keys(kbox[1], 0, nw, true));
    const double loz = key_value(combine_keys(kbox[2], 0, nw, true));
    const double hix = key_value(combine_keys(kbox[3], 0, nw, false));
    const double hiy = key_value(combine_keys(kbox[4], 0, nw, false));
    const double hiz = key_value(combine_keys(kbox[5], 0, nw, false));
    const double hmax = key_value(combine_keys(kbox[6], 0, nw, false));
    double mass = kmass[0];
    for (int w = 1; w < nw; ++w) mass += kmass[w];
    const bool any = lox <= hix;  // tile holds at least one real particle
    // FP32 centre (exactly representable), FP64 offsets rounded once to FP32
    double q = 0.0, qinv = 0.0;
    if (qmax) {
        const double amax = __longlong_as_double((long long)*qmax);
        int e = 0;
        bool grid = false;
        if (amax > 0.0) {
            frexp(amax, &e);  // amax < 2^e
            grid = true;
        }
        if (qemin > -1000 && (!grid || e < qemin)) {
            e = qemin;
            grid = true;
        }
        if (grid) {
            q = ldexp(1.0, e - 22);
            qinv = ldexp(1.0, 22 - e);
        }
    }
    const float cx = any ? grid_centre(0.5 * (lox + hix), q, qinv) : 0.f;
    const float cy = any ? grid_centre(0.5 * (loy + hiy), q, qinv) : 0.f;
    const float cz = any ? grid_centre(0.5 * (loz + hiz), q, qinv) : 0.f;
    const double dx = px - (double)cx, dy = py - (double)cy, dz = pz - (double)cz;
    // the halves' boxes (sub-block near tests): centres need not lie on the
    // grid, these boxes only classify
    float hcx = 0.f, hcy = 0.f, hcz = 0.f, hh = 0.f, hm = 0.f;
    if (tbox_hc) {
        const double hlox = key_value(combine_keys(kbox[0], w0, w0 + hw, true));
        const double hloy = key_value(combine_keys(kbox[1], w0, w0 + hw, true));
        const double hloz = key_value(combine_keys(kbox[2], w0, w0 + hw, true));
        const double hhix = key_value(combine_keys(kbox[3], w0, w0 + hw, false));
        const double hhiy = key_value(combine_keys(kbox[4], w0, w0 + hw, false));
        const double hhiz = key_value(combine_keys(kbox[5], w0, w0 + hw, false));
        hh = __double2float_ru(key_value(combine_keys(kbox[6], w0, w0 + hw, false)));
        double hms = kmass[w0];
        for (int w = w0 + 1; w < w0 + hw; ++w) hms += kmass[w];
        hm = __double2float_rn(hms);
        if (hlox <= hhix) {
            hcx = __double2float_rn(0.5 * (hlox + hhix));
            hcy = __double2float_rn(0.5 * (hloy + hhiy));
            hcz = __double2float_rn(0.5 * (hloz + hhiz));
        }
    }
    {
        long long kv[6] = {ord_key(valid ? fabs(dx) : 0.0), ord_key(valid ? fabs(dy) : 0.0),
                           ord_key(valid ? fabs(dz) : 0.0), ord_key(valid ? fabs(px - (double)hcx) : 0.0),
                           ord_key(valid ? fabs(py - (double)hcy) : 0.0),
                           ord_key(valid ? fabs(pz - (double)hcz) : 0.0)};
        warp_keys<6>(kv, 0u, kext);
    }
    __syncthreads();
    const double ex = key_value(combine_keys(kext[0], 0, nw, false));
    const double ey = key_value(combine_keys(kext[1], 0, nw, false));
    const double ez = key_value(combine_keys(kext[2], 0, nw, false));
    float ox, oy, oz, rx, ry, rz, fm, fh;
    if (valid) {
        ox = __double2float_rn(dx);
        oy = __double2float_rn(dy);
        oz = __double2float_rn(dz);
        // what the FP32 offset lost: x = c + o + r to ~2^-48 relative
        rx = __double2float_rn(dx - (double)ox);
        ry = __double2float_rn(dy - (double)oy);
        rz = __double2float_rn(dz - (double)oz);
        fm = __double2float_rn(pm);
        fh = __double2float_rn(ph);
    } else {
        ox = oy = oz = kPadOffset;
        rx = ry = rz = 0.f;
        fm = fh = 0.f;
    }
    jdup[2 * p] = make_float4(ox, ox, oy, oy);
    jdup[2 * p + 1] = make_float4(oz, oz, fm, fm);
    rdup[2 * p] = make_float4(rx, rx, ry, ry);
    rdup[2 * p + 1] = make_float4(rz, rz, fh, fh);
    if (sdup) {
        // chunks of 32 particles, component-major inside a chunk
        const int64_t base = (p >> 5) * 64 + (p & 31);
        sdup[base] = make_float4(ox, ox, oy, oy);
        sdup[base + 32] = make_float4(oz, oz, fm, fm);
    }
    if (fdup) {
        // Far-field expansion: with k = m^(-2/3) rounded once to FP32,
        //   k |o_j - s|^2 = k |s|^2 + k |o_j|^2 - 2 k o_j . s
        // so (k |o_j - s|^2)^(-3/2) = m_j / |o_j - s|^3 (to the rounding of k).
        // The coefficients are formed in FP64 from the FP32 values actually used.
        float fk, ax, ay, az, fb;
        if (valid) {
            const double cm = cbrt(pm);
            fk = __double2float_rn(1.0 / (cm * cm));
            const double k = (double)fk;
            ax = __double2float_rn(2.0 * k * (double)ox);
            ay = __double2float_rn(2.0 * k * (double)oy);
            az = __double2float_rn(2.0 * k * (double)oz);
            fb = __double2float_rn(
                k * ((double)ox * (double)ox + (double)oy * (double)oy + (double)oz * (double)oz));
        } else {
            // k |o - s|^2 evaluates to +inf for every target: the pair adds exactly 0
            fk = 1.0e10f;
            ax = ay = az = 0.f;
            fb = __int_as_float(0x7f800000);
        }
        fdup[4 * p] = make_float4(ox, ox, oy, oy);
        fdup[4 * p + 1] = make_float4(oz, oz, fk, fk);
        fdup[4 * p + 2] = make_float4(ax, ax, ay, ay);
        fdup[4 * p + 3] = make_float4(az, az, fb, fb);
    }
    if (threadIdx.x == 0) {
        // extents and softening rounded up so the box tests stay conservative
        tbox_c[tile] = make_float4(cx, cy, cz, __double2float_ru(hmax));
        tbox_e[tile] = make_float4(__double2float_ru(ex), __double2float_ru(ey), __double2float_ru(ez),
                                   __double2float_rn(mass));
    }
    if (tbox_hc && (threadIdx.x & (blockDim.x / 2 - 1)) == 0) {
        const int64_t hb = 2 * tile + (threadIdx.x >= blockDim.x / 2 ? 1 : 0);
        const double hex = key_value(combine_keys(kext[3], w0, w0 + hw, false));
        const double hey = key_value(combine_keys(kext[4], w0, w0 + hw, false));
        const double hez = key_value(combine_keys(kext[5], w0, w0 + hw, false));
        tbox_hc[hb] = make_float4(hcx, hcy, hcz, hh);
        tbox_he[hb] = make_float4(__double2float_ru(hex), __double2float_ru(hey), __double2float_ru(hez), hm);
    }
}

// ---------------- Morton sort ----------------

// Bounding box of the positions in two passes: per-CTA minima and maxima on
// order-preserving integer keys (exact, and on the integer pipe; NaN entries
// are skipped as fmin / fmax would), then one warp combines the CTAs in
// order.  part: [6][gridDim.x] keys.
constexpr int kBoxCtas = 256;

__global__ void bbox_partial_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                    const double *__restrict__ z, long long *__restrict__ part) {
    __shared__ long long red[6][32];
    long long k[6];
    for (int c = 0; c < 3; ++c) {
        k[c] = ord_key(DBL_MAX);
        k[3 + c] = ord_key(-DBL_MAX);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v[3] = {x[i], y[i], z[i]};
        for (int c = 0; c < 3; ++c) {
            if (!(v[c] == v[c])) continue;
            const long long q = ord_key(v[c]);
            k[c] = q < k[c] ? q : k[c];
            k[3 + c] = q > k[3 + c] ? q : k[3 + c];
        }
    }
    warp_keys<6>(k, 0x7u, red);
    __syncthreads();
    if (threadIdx.x < 6)
        part[threadIdx.x * gridDim.x + blockIdx.x] =
            combine_keys(red[threadIdx.x], 0, (blockDim.x + 31) >> 5, threadIdx.x < 3);
}

__global__ void bbox_final_kernel(int G, const long long *__restrict__ part, double *__restrict__ bbox) {
    const int c = threadIdx.x;
    if (c < 6) bbox[c] = key_value(combine_keys(part + (size_t)c * G, 0, G, c < 3));
}

__device__ __forceinline__ unsigned long long spread21(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void morton_kernel(int64_t n, int64_t npow2, const double *__restrict__ x,
                              const double *__restrict__ y, const double *__restrict__ z,
                              const double *__restrict__ bbox, unsigned long long *__restrict__ keys,
                              unsigned int *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    if (i >= n) {
        keys[i] = ~0ull;
        vals[i] = (unsigned int)i;
        return;
    }
    const double span = fmax(fmax(bbox[3] - bbox[0], bbox[4] - bbox[1]), fmax(bbox[5] - bbox[2], 1e-300));
    const double scale = 2097151.0 / span;
    const double v[3] = {x[i], y[i], z[i]};
    unsigned long long c[3];
    for (int k = 0; k < 3; ++k) {
        double q = (v[k] - bbox[k]) * scale;
        q = fmin(fmax(q, 0.0), 2097151.0);
        c[k] = (unsigned long long)q;
    }
    keys[i] = (spread21(c[0]) << 2) | (spread21(c[1]) << 1) | spread21(c[2]);
    vals[i] = (unsigned int)i;
}

// One compare-exchange stage of a bitonic network over (key, val); ties are
// broken by val so that the order is total and deterministic.
__global__ void bitonic_global(int64_t npow2, int64_t j, int64_t k, unsigned long long *keys,
                               unsigned int *vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const bool up = (i & k) == 0;
    const unsigned long long ki = keys[i], kl = keys[l];
    const unsigned int vi = vals[i], vl = vals[l];
    const bool gt = (ki > kl) || (ki == kl && vi > vl);
    if (gt == up) {
        keys[i] = kl;
        keys[l] = ki;
        vals[i] = vl;
        vals[l] = vi;
    }
}

// All stages with j < 1024 of one k, inside a 2048-element shared-memory block.
__global__ void bitonic_shared(int64_t npow2, int64_t k, int64_t jstart, unsigned long long *keys,
                               unsigned int *vals) {
    __shared__ unsigned long long sk[2048];
    __shared__ unsigned int sv[2048];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        sk[t] = keys[base + t];
        sv[t] = vals[base + t];
    }
    __syncthreads();
    for (int64_t j = jstart; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            const int l = t ^ (int)j;
            if (l > t) {
                const int64_t gi = base + t;
                const bool up = (gi & k) == 0;
                const unsigned long long ki = sk[t], kl = sk[l];
                const unsigned int vi = sv[t], vl = sv[l];
                const bool gt = (ki > kl) || (ki == kl && vi > vl);
                if (gt == up) {
                    sk[t] = kl;
                    sk[l] = ki;
                    sv[t] = vl;
                    sv[l] = vi;
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        keys[base + t] = sk[t];
        vals[base + t] = sv[t];
    }
}

__global__ void gather_f64_kernel(int64_t n, const unsigned int *__restrict__ idx,
                                  const double *__restrict__ in, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}

__global__ void gather_i64_kernel(int64_t n, const unsigned int *__restrict__ idx,
                                  const int64_t *__restrict__ in, int64_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}

inline unsigned blocks_for(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

}  // namespace

void launch_stage(const Staging &s, const double *x, const double *y, const double *z,
                  const double *m, const double *h, cudaStream_t st) {
    if (s.qmax) {
        cudaMemsetAsync(s.qmax, 0, sizeof(unsigned long long), st);
        absmax_kernel<<<152, 512, 0, st>>>(s.n, x, y, z, h, s.pscale, s.qmax);
    }
    stage_kernel<<<(unsigned)s.ntile, s.T, 0, st>>>(s.n, s.T, x, y, z, m, h, s.jdup, s.rdup, s.fdup, s.sdup,
                                                    s.qmax, s.pscale, s.qemin, s.tbox_c, s.tbox_e, s.tbox_hc,
                                                    s.tbox_he);
}

namespace {

// Ensemble keys: (system << 57) | 57-bit Morton code of the position inside
// the system's own bounding box; padding sorts to the end of its system.
__global__ void ens_bbox_kernel(const int64_t *__restrict__ off, const double *__restrict__ x,
                                const double *__restrict__ y, const double *__restrict__ z,
                                const double *__restrict__ h, double *__restrict__ bbox) {
    __shared__ double sbuf[32];
    const int s = blockIdx.x;
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) {
        if (h[i] < 0.0) continue;
        const double v[3] = {x[i], y[i], z[i]};
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], v[k]);
            hi[k] = fmax(hi[k], v[k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        const double a = block_reduce(lo[k], sbuf, MinOp());
        const double b = block_reduce(hi[k], sbuf, MaxOp());
        if (threadIdx.x == 0) {
            bbox[6 * s + k] = a;
            bbox[6 * s + 3 + k] = b;
        }
    }
}

__global__ void ens_morton_kernel(int64_t np_total, int64_t npow2, const int *__restrict__ sim,
                                  const double *__restrict__ x, const double *__restrict__ y,
                                  const double *__restrict__ z, const double *__restrict__ h,
                                  const double *__restrict__ bbox, unsigned long long *__restrict__ keys,
                                  unsigned int *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    vals[i] = (unsigned int)i;
    if (i >= np_total) {
        keys[i] = ~0ull;
        return;
    }
    const unsigned long long s = (unsigned long long)sim[i];
    const unsigned long long low = (1ull << 57) - 1;
    if (h[i] < 0.0) {
        keys[i] = (s << 57) | low;
        return;
    }
    const double *bb = bbox + 6 * s;
    const double span = fmax(fmax(bb[3] - bb[0], bb[4] - bb[1]), fmax(bb[5] - bb[2], 1e-300));
    const double scale = 524287.0 / span;
    const double v[3] = {x[i], y[i], z[i]};
    unsigned long long c[3];
    for (int k = 0; k < 3; ++k) {
        double q = (v[k] - bb[k]) * scale;
        q = fmin(fmax(q, 0.0), 524287.0);
        c[k] = (unsigned long long)q;
    }
    const unsigned long long code = (spread21(c[0]) << 2) | (spread21(c[1]) << 1) | spread21(c[2]);
    keys[i] = (s << 57) | (code & (low - 1));
}

int bitonic_network(SortScratch &s, cudaStream_t st) {
    const int64_t np2 = s.npow2;
    int count = 0;
    for (int64_t k = 2; k <= np2; k <<= 1) {
        int64_t j = k >> 1;
        for (; j > 0; j >>= 1) {
            if (j < 1024 && np2 >= 2048) {
                bitonic_shared<<<(unsigned)(np2 / 2048), 1024, 0, st>>>(np2, k, j, s.keys, s.vals);
                ++count;
                break;
            }
            bitonic_global<<<blocks_for(np2, 256), 256, 0, st>>>(np2, j, k, s.keys, s.vals);
            ++count;
        }
    }
    return count;
}

}  // namespace

cudaError_t ensemble_sort(int nsims, const int64_t *off, int64_t np_total, const int *sim,
                          const double *x, const double *y, const double *z, const double *h,
                          SortScratch &s, cudaStream_t st, int *launches) {
    ens_bbox_kernel<<<nsims, 512, 0, st>>>(off, x, y, z, h, s.bbox);
    ens_morton_kernel<<<blocks_for(s.npow2, 256), 256, 0, st>>>(np_total, s.npow2, sim, x, y, z, h,
                                                                 s.bbox, s.keys, s.vals);
    const int c = bitonic_network(s, st);
    if (launches) *launches = 2 + c;
    return cudaGetLastError();
}

cudaError_t morton_sort(int64_t n, const double *x, const double *y, const double *z,
                        SortScratch &s, cudaStream_t st, int *launches) {
    const int64_t np2 = s.npow2;
    int count = 3;
    // the per-CTA partials live after the box itself (bbox holds 8 + 6 kBoxCtas words)
    const int G = (int)std::min<int64_t>(kBoxCtas, std::max<int64_t>(1, (n + 255) / 256));
    long long *part = reinterpret_cast<long long *>(s.bbox + 8);
    bbox_partial_kernel<<<G, 256, 0, st>>>(n, x, y, z, part);
    bbox_final_kernel<<<1, 32, 0, st>>>(G, part, s.bbox);
    morton_kernel<<<blocks_for(np2, 256), 256, 0, st>>>(n, np2, x, y, z, s.bbox, s.keys, s.vals);
    for (int64_t k = 2; k <= np2; k <<= 1) {
        int64_t j = k >> 1;
        for (; j > 0; j >>= 1) {
            if (j < 1024 && np2 >= 2048) {
                bitonic_shared<<<(unsigned)(np2 / 2048), 1024, 0, st>>>(np2, k, j, s.keys, s.vals);
                ++count;
                break;
            }
            bitonic_global<<<blocks_for(np2, 256), 256, 0, st>>>(np2, j, k, s.keys, s.vals);
            ++count;
        }
    }
    if (launches) *launches = count;
    return cudaGetLastError();
}

cudaError_t gather_f64(int64_t n, const unsigned int *vals, const double *in, double *out,
                       cudaStream_t st) {
    gather_f64_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, vals, in, out);
    return cudaGetLastError();
}

cudaError_t gather_i64(int64_t n, const unsigned int *vals, const int64_t *in, int64_t *out,
                       cudaStream_t st) {
    gather_i64_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, vals, in, out);
    return cudaGetLastError();
}

}  // namespace steps

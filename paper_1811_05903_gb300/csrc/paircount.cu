// Exact pair counts DD(r) of many point sets in one launch: the targets of the
// correlation-function emulator (central-sphere xi(r) of batched runs).
// Positions are quantised to integer fixed point (q = llround(x / step),
// |q| <= 2^29), squared separations are exact int64, and a pair (i < j) falls
// in bin b when edge2[b] <= d^2 < edge2[b+1].  Counts are integers, so the
// result does not depend on the order of the additions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "steps_internal.h"

namespace {

constexpr int kTB = 256;       // targets per block
constexpr int kJT = 1024;      // sources staged per shared-memory tile
constexpr int kMaxBins = 64;

__global__ void quantise_kernel(int64_t n, const double *__restrict__ pos, const double *__restrict__ centre,
                                double inv_step, int *__restrict__ q, int *__restrict__ bad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const double v = (pos[k] - centre[k % 3]) * inv_step;
    if (!(fabs(v) < 536870912.0)) {  // |q| <= 2^29 keeps d^2 < 2^63; NaN rejected
        atomicOr(bad, 1);
        q[k] = 0;
        return;
    }
    q[k] = (int)llround(v);
}

__global__ void __launch_bounds__(kTB) paircount_kernel(const int *__restrict__ q, const int64_t *__restrict__ off,
                                                        int nbins, const long long *__restrict__ edge2,
                                                        unsigned long long *__restrict__ dd) {
    __shared__ int4 sj[kJT];
    __shared__ long long se[kMaxBins + 1];
    __shared__ unsigned int hist[kTB / 32][kMaxBins];
    const int set = blockIdx.y;
    const int64_t o = off[set], n = off[set + 1] - off[set];
    const int64_t i = (int64_t)blockIdx.x * kTB + threadIdx.x;
    const int warp = threadIdx.x >> 5;
    if ((int64_t)blockIdx.x * kTB >= n) return;  // whole block idle for this (shorter) set
    for (int b = threadIdx.x; b <= nbins; b += kTB) se[b] = edge2[b];
    for (int b = threadIdx.x; b < (kTB / 32) * kMaxBins; b += kTB) (&hist[0][0])[b] = 0u;
    int xi = 0, yi = 0, zi = 0;
    if (i < n) {
        xi = q[3 * (o + i)];
        yi = q[3 * (o + i) + 1];
        zi = q[3 * (o + i) + 2];
    }
    __syncthreads();
    const long long e_lo = se[0], e_hi = se[nbins];
    // sources j > i: start at this block's first target
    for (int64_t j0 = (int64_t)blockIdx.x * kTB; j0 < n; j0 += kJT) {
        __syncthreads();
        for (int t = threadIdx.x; t < kJT; t += kTB) {
            const int64_t j = j0 + t;
            if (j < n) sj[t] = make_int4(q[3 * (o + j)], q[3 * (o + j) + 1], q[3 * (o + j) + 2], 0);
        }
        __syncthreads();
        if (i >= n) continue;
        const int cnt = (n - j0 < kJT) ? (int)(n - j0) : kJT;
        const int first = (i + 1 - j0 > 0) ? (int)(i + 1 - j0) : 0;  // j > i
        for (int t = first; t < cnt; ++t) {
            const int4 p = sj[t];
            // |q| <= 2^29, so each difference fits in int32 and d^2 < 2^63
            const int dx = p.x - xi, dy = p.y - yi, dz = p.z - zi;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            if (d2 < e_lo || d2 >= e_hi) continue;
            int b = 0, e = nbins;  // se[b] <= d2 < se[e]
            while (e - b > 1) {
                const int mid = (b + e) >> 1;
                if (se[mid] <= d2) b = mid; else e = mid;
            }
            atomicAdd(&hist[warp][b], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kTB) {
        unsigned long long s = 0;
        for (int w = 0; w < kTB / 32; ++w) s += hist[w][b];
        if (s) atomicAdd(&dd[(int64_t)set * nbins + b], s);
    }
}

}  // namespace

using namespace steps;

extern "C" steps_status steps_paircount(int nsets, const int64_t *offsets, const double *pos,
                                        const double *centres, double step, int nbins,
                                        const int64_t *edge2, uint64_t *dd_out, void *cuda_stream) {
    if (nsets <= 0 || !offsets || !pos || !centres || !edge2 || !dd_out || nbins <= 0 || nbins > kMaxBins ||
        !(step > 0.0) || !std::isfinite(step)) {
        set_error("bad arguments to steps_paircount (nbins must be in [1, %d], step > 0)", kMaxBins);
        return STEPS_EINVAL;
    }
    std::vector<int64_t> off(offsets, offsets + nsets + 1);
    int64_t nmax = 0;
    for (int s = 0; s < nsets; ++s) {
        if (off[s + 1] < off[s]) {
            set_error("offsets must be non-decreasing");
            return STEPS_EINVAL;
        }
        nmax = std::max(nmax, off[s + 1] - off[s]);
    }
    for (int b = 0; b < nbins; ++b) {
        if (edge2[b + 1] < edge2[b] || edge2[b] < 0) {
            set_error("edge2 must be non-negative and non-decreasing");
            return STEPS_EINVAL;
        }
    }
    const int64_t N = off[nsets];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // scratch for this call: fixed-point coordinates, offsets, edges, centres, counts
    void *mem = nullptr;
    const size_t bytes = sizeof(int) * 3 * std::max<int64_t>(N, 1) + sizeof(int64_t) * (nsets + 1) +
                         sizeof(long long) * (nbins + 1) + sizeof(double) * 3 * nsets +
                         sizeof(unsigned long long) * nsets * nbins + 64;
    STEPS_TRY(counted_malloc(&mem, bytes + 256));
    char *p = static_cast<char *>(mem);
    auto carve = [&](size_t b) {
        char *r = p;
        p += (b + 15) / 16 * 16;
        return r;
    };
    int *q = reinterpret_cast<int *>(carve(sizeof(int) * 3 * std::max<int64_t>(N, 1)));
    int64_t *doff = reinterpret_cast<int64_t *>(carve(sizeof(int64_t) * (nsets + 1)));
    long long *de = reinterpret_cast<long long *>(carve(sizeof(long long) * (nbins + 1)));
    double *dc = reinterpret_cast<double *>(carve(sizeof(double) * 3 * nsets));
    unsigned long long *ddd = reinterpret_cast<unsigned long long *>(carve(sizeof(unsigned long long) * nsets * nbins));
    int *bad = reinterpret_cast<int *>(carve(sizeof(int)));
    steps_status status = STEPS_OK;
    do {
        cudaError_t e = cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (nsets + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(de, edge2, sizeof(long long) * (nbins + 1), cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dc, centres, sizeof(double) * 3 * nsets, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ddd, 0, sizeof(unsigned long long) * nsets * nbins, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            status = cuda_status(e, "steps_paircount setup");
            break;
        }
        // quantise every set about its own centre
        for (int s = 0; s < nsets && e == cudaSuccess; ++s) {
            const int64_t ns = off[s + 1] - off[s];
            if (ns == 0) continue;
            quantise_kernel<<<(unsigned)((3 * ns + 255) / 256), 256, 0, st>>>(
                ns, pos + 3 * off[s], dc + 3 * s, 1.0 / step, q + 3 * off[s], bad);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            status = cuda_status(e, "quantise_kernel");
            break;
        }
        int hbad = 0;
        e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            status = cuda_status(e, "steps_paircount");
            break;
        }
        if (hbad) {
            set_error("a coordinate is non-finite or 2^29 or more steps from its centre");
            status = STEPS_EINVAL;
            break;
        }
        if (nmax > 0) {
            dim3 grid((unsigned)((nmax + kTB - 1) / kTB), (unsigned)nsets);
            paircount_kernel<<<grid, kTB, 0, st>>>(q, doff, nbins, de, ddd);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dd_out, ddd, sizeof(unsigned long long) * nsets * nbins, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) status = cuda_status(e, "paircount_kernel");
    } while (0);
    cudaStreamSynchronize(st);
    counted_free(mem, bytes + 256);
    return status;
}

// Correlation-function emulator: a 5 -> 256 -> 256 -> 256 -> 1 SiLU network
// trained by Adam, every matrix product on the tensor cores with bfloat16
// operands and FP32 accumulation (mma.sync m16n8k16), everything else FP32.
//
// Device layout (all padded so that every product is a multiple of 16 wide):
//   layer l weight W_l [N_l][K_l], N = (256, 256, 256, 16), K = (16, 256, 256, 256);
//   the input layer's columns 5..15 and the output layer's rows 1..15 are zero
//   and stay zero (their gradients are exactly zero, so Adam never moves them).
//   master / Adam m / Adam v / gradient: one packed FP32 array each,
//   W1 b1 W2 b2 W3 b3 W4 b4 in that order; bf16 copies W_l and W_l^T.
//   activations A_l [B][K_l] bf16 and A_l^T [K_l][B]; pre-activations Z_l FP32.
//
// Every product is a "TN" product C[m][n] = sum_k X[m][k] Y[n][k] with both
// operands contiguous in k:
//   forward      Z_l    = A_{l-1} W_l^T            X = A_{l-1}, Y = W_l
//   input grad   dA_l   = dZ_{l+1} W_{l+1}         X = dZ_{l+1}, Y = W_{l+1}^T
//   weight grad  dW_l   = dZ_l^T A_{l-1}           X = dZ_l^T,  Y = A_{l-1}^T
// with the element-wise parts (bias, SiLU, SiLU', BF16 rounding, transposed
// copies, bias-gradient column sums) fused into the product's epilogue.
// All reductions run in a fixed order: results are deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/steps_emu.h"
#include "steps_internal.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kLayers = 4;
constexpr int kIn = STEPS_EMU_IN, kInP = 16, kH = STEPS_EMU_WIDTH, kOutP = 16;
constexpr int kKp[kLayers] = {kInP, kH, kH, kH};
constexpr int kNp[kLayers] = {kH, kH, kH, kOutP};
constexpr int kKu[kLayers] = {kIn, kH, kH, kH};  // unpadded fan-in
constexpr int kNu[kLayers] = {kH, kH, kH, 1};    // unpadded fan-out

struct Offsets {
    int64_t seg[2 * kLayers + 1];  // W1 b1 W2 b2 W3 b3 W4 b4, end
};

constexpr Offsets padded_offsets() {
    Offsets o{};
    int64_t k = 0;
    for (int l = 0; l < kLayers; ++l) {
        o.seg[2 * l] = k;
        k += (int64_t)kNp[l] * kKp[l];
        o.seg[2 * l + 1] = k;
        k += kNp[l];
    }
    o.seg[2 * kLayers] = k;
    return o;
}
constexpr Offsets kPad = padded_offsets();
constexpr int64_t kP = kPad.seg[2 * kLayers];

// ---------------------------------------------------------------------------
// bf16 tensor-core product with fused epilogues
// ---------------------------------------------------------------------------
enum { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_BWD = 2, EPI_DW = 3 };

struct Epi {
    const float *bias = nullptr;  // FWD: bias [N]
    float *z = nullptr;           // FWD: Z out [M][N]; BWD: dZ out (FP32) [M][N]
    bf16 *a = nullptr;            // FWD_HIDDEN: A out [M][N]; BWD: bf16(dZ) [M][N]
    bf16 *at = nullptr;           // transposed copy of a: [N][ldt]
    int ldt = 0;
    const float *zprev = nullptr; // BWD: pre-activation of the layer below [M][N]
    float *g = nullptr;           // DW: weight gradient [M][N]
    const float *dzsrc = nullptr; // DW: FP32 dZ [K][M] for the bias gradient
    float *gb = nullptr;          // DW: bias gradient [M]
};

constexpr int BM = 64, BN = 64, BK = 32, SK = BK + 8;  // +8: conflict-free fragment loads

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// C[M][N] = sum_k X[m][k] Y[n][k]; X [M][K], Y [N][K] bf16, K a multiple of 8.
// 64x64 tile per CTA, 4 warps of 32x32, k staged 32 at a time.
template <int MODE>
__global__ void __launch_bounds__(128) tn_gemm(int M, int N, int K, const bf16 *__restrict__ X,
                                               const bf16 *__restrict__ Y, Epi e) {
    __shared__ __align__(16) bf16 Xs[BM][SK];
    __shared__ __align__(16) bf16 Ys[BN][SK];
    __shared__ float part[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;

    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int v = tid + 128 * r, row = v >> 2, kv = (v & 3) * 8;
            uint4 xv = make_uint4(0u, 0u, 0u, 0u), yv = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + row < M && k0 + kv < K)
                xv = *reinterpret_cast<const uint4 *>(X + (size_t)(m0 + row) * K + k0 + kv);
            if (n0 + row < N && k0 + kv < K)
                yv = *reinterpret_cast<const uint4 *>(Y + (size_t)(n0 + row) * K + k0 + kv);
            *reinterpret_cast<uint4 *>(&Xs[row][kv]) = xv;
            *reinterpret_cast<uint4 *>(&Ys[row][kv]) = yv;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r0 = wm * 32 + mi * 16 + g;
                af[mi][0] = *reinterpret_cast<const uint32_t *>(&Xs[r0][ks + 2 * t4]);
                af[mi][1] = *reinterpret_cast<const uint32_t *>(&Xs[r0 + 8][ks + 2 * t4]);
                af[mi][2] = *reinterpret_cast<const uint32_t *>(&Xs[r0][ks + 2 * t4 + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t *>(&Xs[r0 + 8][ks + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int c = wn * 32 + ni * 8 + g;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Ys[c][ks + 2 * t4]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Ys[c][ks + 2 * t4 + 8]);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) mma_bf16_16816(acc[mi][ni], af[mi], b0, b1);
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm * 32 + mi * 16 + g + ((c & 2) ? 8 : 0);
                const int n = n0 + wn * 32 + ni * 8 + 2 * t4 + (c & 1);
                if (m >= M || n >= N) continue;
                const float v = acc[mi][ni][c];
                const size_t o = (size_t)m * N + n;
                if (MODE == EPI_FWD_HIDDEN) {
                    const float z = v + e.bias[n];
                    e.z[o] = z;
                    const bf16 h = __float2bfloat16_rn(z * sigmoidf_(z));
                    e.a[o] = h;
                    e.at[(size_t)n * e.ldt + m] = h;
                } else if (MODE == EPI_FWD_OUT) {
                    e.z[o] = v + e.bias[n];
                } else if (MODE == EPI_BWD) {
                    const float zp = e.zprev[o];
                    const float s = sigmoidf_(zp);
                    const float dz = v * (s * (1.0f + zp * (1.0f - s)));
                    e.z[o] = dz;
                    const bf16 h = __float2bfloat16_rn(dz);
                    e.a[o] = h;
                    e.at[(size_t)n * e.ldt + m] = h;
                } else {
                    e.g[o] = v;
                }
            }

    if (MODE == EPI_DW && blockIdx.x == 0) {
        // bias gradient of rows m0..m0+63: column sums of the FP32 dZ, even
        // and odd batch rows summed separately, then added (fixed order)
        const int mm = tid & 63, half = tid >> 6;
        float s = 0.f;
        if (m0 + mm < M)
            for (int b = half; b < K; b += 2) s += e.dzsrc[(size_t)b * M + m0 + mm];
        part[tid] = s;
        __syncthreads();
        if (half == 0 && m0 + mm < M) e.gb[m0 + mm] = part[tid] + part[tid + 64];
    }
}

// Inputs of M rows -> bf16 A_0 [M][16] (zero padded) and its transpose; the
// targets of the rows.  rows_all == nullptr: rows are 0..M-1 of x.
__global__ void gather_kernel(int M, int ldt, const float *__restrict__ x, const float *__restrict__ tall,
                              const int32_t *__restrict__ rows_all, const int *__restrict__ scal, int bstep,
                              bf16 *__restrict__ a0, bf16 *__restrict__ a0t, float *__restrict__ tgt) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * kInP) return;
    const int b = idx / kInP, k = idx % kInP;
    int64_t r = b;
    if (rows_all) r = rows_all[(int64_t)scal[0] * bstep + b];
    const bf16 h = __float2bfloat16_rn(k < kIn ? x[r * kIn + k] : 0.f);
    a0[(size_t)b * kInP + k] = h;
    a0t[(size_t)k * ldt + b] = h;
    if (k == 0 && tgt) tgt[b] = tall[r];
}

// Mean squared error of column 0 of Z_4 against the targets, dL/dz of the
// output layer (FP32, bf16, transposed bf16; padded columns zero).  In a
// training step it also records the loss, advances the step counters and
// sets this step's Adam hyper-parameters (lr, 1 - beta1^t, 1 - beta2^t).
__global__ void __launch_bounds__(1024) loss_kernel(int B, const float *__restrict__ z4, const float *__restrict__ tgt,
                                                    float *__restrict__ dz, bf16 *__restrict__ dzb,
                                                    bf16 *__restrict__ dzt, int ldt, int *scal,
                                                    const float *__restrict__ lr_all, float *hyper,
                                                    float *loss_all, float *loss_one) {
    __shared__ float red[32];
    float part = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float d = z4[(size_t)b * kOutP] - tgt[b];
        part += d * d;
        const float dzv = 2.0f * d / (float)B;
        for (int c = 0; c < kOutP; ++c) {
            const float val = (c == 0) ? dzv : 0.f;
            const bf16 h = __float2bfloat16_rn(val);
            dz[(size_t)b * kOutP + c] = val;
            dzb[(size_t)b * kOutP + c] = h;
            dzt[(size_t)c * ldt + b] = h;
        }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        const float loss = s / (float)B;
        if (scal) {
            const int step = scal[0];
            loss_all[step] = loss;
            hyper[0] = lr_all[step];
            const int t = scal[1] + 1;
            scal[1] = t;
            hyper[1] = (float)(1.0 - pow(0.9, (double)t));
            hyper[2] = (float)(1.0 - pow(0.999, (double)t));
            scal[0] = step + 1;
        } else {
            *loss_one = loss;
        }
    }
}

struct Copies {
    bf16 *wb[kLayers], *wt[kLayers];
    int64_t seg[2 * kLayers + 1];  // packed offsets (kPad), passed by value
    int K[kLayers], N[kLayers];
};

// Adam on the packed FP32 master (update != 0), then the bf16 copies W_l and
// W_l^T of every weight.
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, const float *__restrict__ hyper, int update, Copies cp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP) return;
    float wi = w[i];
    if (update) {
        const float lr = hyper[0], c1 = hyper[1], c2 = hyper[2];
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * (gi * gi);
        m[i] = mi;
        v[i] = vi;
        wi -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        w[i] = wi;
    }
    int seg = 0;
    while (seg < 2 * kLayers - 1 && i >= cp.seg[seg + 1]) ++seg;
    if ((seg & 1) == 0) {
        const int l = seg >> 1;
        const int64_t local = i - cp.seg[seg];
        const int K = cp.K[l], N = cp.N[l];
        const int n = (int)(local / K), k = (int)(local % K);
        const bf16 h = __float2bfloat16_rn(wi);
        cp.wb[l][local] = h;
        cp.wt[l][(size_t)k * N + n] = h;
    }
}

__global__ void take_col0(int M, const float *__restrict__ z4, float *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) y[i] = z4[(size_t)i * kOutP];
}

__global__ void finite_f32(int64_t n, const float *__restrict__ a, int *__restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(a[i])) atomicOr(bad, 1);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

using namespace steps;

struct steps_emu {
    int B = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    Copies cp{};
    bf16 *act[kLayers] = {}, *actT[kLayers] = {};
    float *z[kLayers] = {};
    float *dz[2] = {};
    bf16 *dzb[2] = {}, *dzt[2] = {};
    float *tgt = nullptr, *hyper = nullptr, *loss_one = nullptr, *xs = nullptr, *ts = nullptr, *ys = nullptr;
    int *scal = nullptr, *bad = nullptr;
    // training set and per-call step tables
    float *xd = nullptr, *td = nullptr;
    int64_t nd = 0;
    size_t data_bytes = 0;
    int32_t *rows = nullptr;
    float *lr = nullptr, *losses = nullptr;
    int cap_steps = 0;
    size_t steps_bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t adam_steps = 0;
};

namespace {

void drop_graph(steps_emu *e) {
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
}

template <int MODE>
cudaError_t gemm(steps_emu *e, int M, int N, int K, const bf16 *X, const bf16 *Y, const Epi &epi) {
    dim3 grid(blocks(N, BN), blocks(M, BM));
    tn_gemm<MODE><<<grid, 128, 0, e->st>>>(M, N, K, X, Y, epi);
    return cudaGetLastError();
}

// Forward pass of M rows already gathered into act[0].
cudaError_t forward(steps_emu *e, int M) {
    cudaError_t err = cudaSuccess;
    for (int l = 0; l < kLayers && err == cudaSuccess; ++l) {
        Epi epi;
        epi.bias = e->w + kPad.seg[2 * l + 1];
        epi.z = e->z[l];
        if (l < kLayers - 1) {
            epi.a = e->act[l + 1];
            epi.at = e->actT[l + 1];
            epi.ldt = e->B;
            err = gemm<EPI_FWD_HIDDEN>(e, M, kNp[l], kKp[l], e->act[l], e->cp.wb[l], epi);
        } else {
            err = gemm<EPI_FWD_OUT>(e, M, kNp[l], kKp[l], e->act[l], e->cp.wb[l], epi);
        }
    }
    return err;
}

// Backward pass of a full batch: dZ of the output layer is in slot 0.
cudaError_t backward(steps_emu *e) {
    const int B = e->B;
    int cur = 0;
    cudaError_t err = cudaSuccess;
    for (int l = kLayers - 1; l >= 0 && err == cudaSuccess; --l) {
        Epi dw;
        dw.g = e->g + kPad.seg[2 * l];
        dw.dzsrc = e->dz[cur];
        dw.gb = e->g + kPad.seg[2 * l + 1];
        err = gemm<EPI_DW>(e, kNp[l], kKp[l], B, e->dzt[cur], e->actT[l], dw);
        if (err != cudaSuccess || l == 0) break;
        const int nxt = cur ^ 1;
        Epi bw;
        bw.zprev = e->z[l - 1];
        bw.z = e->dz[nxt];
        bw.a = e->dzb[nxt];
        bw.at = e->dzt[nxt];
        bw.ldt = B;
        err = gemm<EPI_BWD>(e, B, kKp[l], kNp[l], e->dzb[cur], e->cp.wt[l], bw);
        cur = nxt;
    }
    return err;
}

cudaError_t refresh_copies(steps_emu *e) {
    adam_kernel<<<blocks(kP, 256), 256, 0, e->st>>>(e->w, e->m, e->v, e->g, e->hyper, 0, e->cp);
    return cudaGetLastError();
}

// One training step on the rows the step counter selects.
cudaError_t train_step(steps_emu *e) {
    const int B = e->B;
    gather_kernel<<<blocks((int64_t)B * kInP, 256), 256, 0, e->st>>>(B, B, e->xd, e->td, e->rows, e->scal, B,
                                                                     e->act[0], e->actT[0], e->tgt);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = forward(e, B);
    if (err == cudaSuccess) {
        loss_kernel<<<1, 1024, 0, e->st>>>(B, e->z[kLayers - 1], e->tgt, e->dz[0], e->dzb[0], e->dzt[0], B,
                                           e->scal, e->lr, e->hyper, e->losses, nullptr);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = backward(e);
    if (err == cudaSuccess) {
        adam_kernel<<<blocks(kP, 256), 256, 0, e->st>>>(e->w, e->m, e->v, e->g, e->hyper, 1, e->cp);
        err = cudaGetLastError();
    }
    return err;
}

// Packed caller layout (unpadded) <-> padded device layout.
void pad_params(const float *src, std::vector<float> &dst) {
    dst.assign(kP, 0.f);
    int64_t k = 0;
    for (int l = 0; l < kLayers; ++l) {
        for (int n = 0; n < kNu[l]; ++n)
            for (int c = 0; c < kKu[l]; ++c) dst[kPad.seg[2 * l] + (int64_t)n * kKp[l] + c] = src[k++];
        for (int n = 0; n < kNu[l]; ++n) dst[kPad.seg[2 * l + 1] + n] = src[k++];
    }
}

void unpad_params(const std::vector<float> &src, float *dst) {
    int64_t k = 0;
    for (int l = 0; l < kLayers; ++l) {
        for (int n = 0; n < kNu[l]; ++n)
            for (int c = 0; c < kKu[l]; ++c) dst[k++] = src[kPad.seg[2 * l] + (int64_t)n * kKp[l] + c];
        for (int n = 0; n < kNu[l]; ++n) dst[k++] = src[kPad.seg[2 * l + 1] + n];
    }
}

steps_status check_bad(steps_emu *e, const char *what) {
    int h = 0;
    STEPS_CUDA(cudaMemcpyAsync(&h, e->bad, sizeof(int), cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    if (h) {
        set_error("%s: non-finite value", what);
        return STEPS_EINVAL;
    }
    return STEPS_OK;
}

}  // namespace

static_assert(STEPS_EMU_NPARAMS == 5 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1, "packed parameter count");

extern "C" steps_status steps_emu_create(steps_emu **out, const float *params, int batch, void *cuda_stream) {
    if (!out || !params || batch < 64 || batch > 4096 || batch % 64 != 0) {
        set_error("steps_emu_create: batch must be a multiple of 64 in [64, 4096]");
        return STEPS_EINVAL;
    }
    *out = nullptr;
    for (int64_t i = 0; i < STEPS_EMU_NPARAMS; ++i)
        if (!std::isfinite(params[i])) {
            set_error("steps_emu_create: parameter %lld is not finite", (long long)i);
            return STEPS_EINVAL;
        }
    steps_emu *e = new steps_emu;
    e->B = batch;
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
    const int64_t B = batch;
    // arena: every buffer 256-byte aligned
    std::vector<std::pair<void **, size_t>> plan;
    auto add = [&](void **p, size_t bytes) { plan.push_back({p, (bytes + 255) / 256 * 256}); };
    add((void **)&e->w, 4 * kP);
    add((void **)&e->m, 4 * kP);
    add((void **)&e->v, 4 * kP);
    add((void **)&e->g, 4 * kP);
    for (int k = 0; k <= 2 * kLayers; ++k) e->cp.seg[k] = kPad.seg[k];
    for (int l = 0; l < kLayers; ++l) {
        e->cp.K[l] = kKp[l];
        e->cp.N[l] = kNp[l];
        add((void **)&e->cp.wb[l], 2 * (size_t)kNp[l] * kKp[l]);
        add((void **)&e->cp.wt[l], 2 * (size_t)kNp[l] * kKp[l]);
        add((void **)&e->act[l], 2 * (size_t)B * kKp[l]);
        add((void **)&e->actT[l], 2 * (size_t)B * kKp[l]);
        add((void **)&e->z[l], 4 * (size_t)B * kNp[l]);
    }
    for (int s = 0; s < 2; ++s) {
        add((void **)&e->dz[s], 4 * (size_t)B * kH);
        add((void **)&e->dzb[s], 2 * (size_t)B * kH);
        add((void **)&e->dzt[s], 2 * (size_t)B * kH);
    }
    add((void **)&e->tgt, 4 * B);
    add((void **)&e->xs, 4 * B * kIn);
    add((void **)&e->ts, 4 * B);
    add((void **)&e->ys, 4 * B);
    add((void **)&e->hyper, 16);
    add((void **)&e->loss_one, 16);
    add((void **)&e->scal, 16);
    add((void **)&e->bad, 16);
    size_t total = 0;
    for (auto &p : plan) total += p.second;
    steps_status s = counted_malloc(&e->arena, total);
    if (s != STEPS_OK) {
        steps_emu_free(e);
        return s;
    }
    e->arena_bytes = total;
    char *p = static_cast<char *>(e->arena);
    for (auto &q : plan) {
        *q.first = p;
        p += q.second;
    }
    std::vector<float> padded;
    pad_params(params, padded);
    cudaError_t ce = cudaMemsetAsync(e->arena, 0, total, e->st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(e->w, padded.data(), 4 * kP, cudaMemcpyHostToDevice, e->st);
    if (ce == cudaSuccess) ce = refresh_copies(e);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->st);
    if (ce != cudaSuccess) {
        steps_emu_free(e);
        return cuda_status(ce, "steps_emu_create");
    }
    *out = e;
    return STEPS_OK;
}

extern "C" steps_status steps_emu_set_data(steps_emu *e, int64_t n, const float *x, const float *t) {
    if (!e || n < 1 || !x || !t) {
        set_error("steps_emu_set_data: bad arguments");
        return STEPS_EINVAL;
    }
    drop_graph(e);
    if (e->xd) counted_free(e->xd, e->data_bytes);
    e->xd = e->td = nullptr;
    e->nd = 0;
    const size_t xb = ((size_t)n * kIn * 4 + 255) / 256 * 256;
    e->data_bytes = xb + (size_t)n * 4;
    void *mem = nullptr;
    STEPS_TRY(counted_malloc(&mem, e->data_bytes));
    e->xd = static_cast<float *>(mem);
    e->td = reinterpret_cast<float *>(static_cast<char *>(mem) + xb);
    e->nd = n;
    STEPS_CUDA(cudaMemcpyAsync(e->xd, x, (size_t)n * kIn * 4, cudaMemcpyDefault, e->st));
    STEPS_CUDA(cudaMemcpyAsync(e->td, t, (size_t)n * 4, cudaMemcpyDefault, e->st));
    STEPS_CUDA(cudaMemsetAsync(e->bad, 0, sizeof(int), e->st));
    finite_f32<<<blocks(n * kIn, 256), 256, 0, e->st>>>(n * kIn, e->xd, e->bad);
    finite_f32<<<blocks(n, 256), 256, 0, e->st>>>(n, e->td, e->bad);
    STEPS_CUDA(cudaGetLastError());
    steps_status s = check_bad(e, "steps_emu_set_data");
    if (s != STEPS_OK) {
        counted_free(e->xd, e->data_bytes);
        e->xd = e->td = nullptr;
        e->nd = 0;
    }
    return s;
}

extern "C" steps_status steps_emu_train(steps_emu *e, int nsteps, const int32_t *rows, const float *lr,
                                        float *loss_out) {
    if (!e || nsteps < 0 || (nsteps > 0 && (!rows || !lr))) {
        set_error("steps_emu_train: bad arguments");
        return STEPS_EINVAL;
    }
    if (nsteps == 0) return STEPS_OK;
    if (!e->xd) {
        set_error("steps_emu_train: no training set (steps_emu_set_data)");
        return STEPS_EINVAL;
    }
    const int64_t nr = (int64_t)nsteps * e->B;
    for (int64_t i = 0; i < nr; ++i)
        if (rows[i] < 0 || rows[i] >= e->nd) {
            set_error("steps_emu_train: row index %d out of range [0, %lld)", rows[i], (long long)e->nd);
            return STEPS_EINVAL;
        }
    for (int s = 0; s < nsteps; ++s)
        if (!std::isfinite(lr[s]) || lr[s] < 0.f) {
            set_error("steps_emu_train: learning rate %d is negative or not finite", s);
            return STEPS_EINVAL;
        }
    if (nsteps > e->cap_steps) {
        drop_graph(e);
        if (e->rows) counted_free(e->rows, e->steps_bytes);
        e->rows = nullptr;
        e->cap_steps = 0;
        const int cap = std::max(nsteps, 64);
        const size_t rb = ((size_t)cap * e->B * 4 + 255) / 256 * 256;
        e->steps_bytes = rb + 2 * (((size_t)cap * 4 + 255) / 256 * 256);
        void *mem = nullptr;
        STEPS_TRY(counted_malloc(&mem, e->steps_bytes));
        e->rows = static_cast<int32_t *>(mem);
        e->lr = reinterpret_cast<float *>(static_cast<char *>(mem) + rb);
        e->losses = reinterpret_cast<float *>(static_cast<char *>(mem) + rb + ((size_t)cap * 4 + 255) / 256 * 256);
        e->cap_steps = cap;
    }
    STEPS_CUDA(cudaMemcpyAsync(e->rows, rows, (size_t)nr * 4, cudaMemcpyHostToDevice, e->st));
    STEPS_CUDA(cudaMemcpyAsync(e->lr, lr, (size_t)nsteps * 4, cudaMemcpyHostToDevice, e->st));
    STEPS_CUDA(cudaMemsetAsync(e->scal, 0, sizeof(int), e->st));  // step within this call
    if (!e->graph) {
        cudaGraph_t gr = nullptr;
        STEPS_CUDA(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = train_step(e);
        cudaError_t ce2 = cudaStreamEndCapture(e->st, &gr);
        if (ce == cudaSuccess) ce = ce2;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->graph, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (ce != cudaSuccess) {
            e->graph = nullptr;
            return cuda_status(ce, "steps_emu_train capture");
        }
    }
    for (int s = 0; s < nsteps; ++s) STEPS_CUDA(cudaGraphLaunch(e->graph, e->st));
    if (loss_out)
        STEPS_CUDA(cudaMemcpyAsync(loss_out, e->losses, (size_t)nsteps * 4, cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    e->adam_steps += nsteps;
    return STEPS_OK;
}

extern "C" steps_status steps_emu_predict(steps_emu *e, int64_t n, const float *x, float *y) {
    if (!e || n < 0 || (n > 0 && (!x || !y))) {
        set_error("steps_emu_predict: bad arguments");
        return STEPS_EINVAL;
    }
    for (int64_t o = 0; o < n; o += e->B) {
        const int M = (int)std::min<int64_t>(e->B, n - o);
        STEPS_CUDA(cudaMemcpyAsync(e->xs, x + o * kIn, (size_t)M * kIn * 4, cudaMemcpyDefault, e->st));
        gather_kernel<<<blocks((int64_t)M * kInP, 256), 256, 0, e->st>>>(M, e->B, e->xs, nullptr, nullptr, nullptr,
                                                                         0, e->act[0], e->actT[0], nullptr);
        STEPS_CUDA(cudaGetLastError());
        STEPS_CUDA(forward(e, M));
        take_col0<<<blocks(M, 256), 256, 0, e->st>>>(M, e->z[kLayers - 1], e->ys);
        STEPS_CUDA(cudaGetLastError());
        STEPS_CUDA(cudaMemcpyAsync(y + o, e->ys, (size_t)M * 4, cudaMemcpyDefault, e->st));
    }
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    return STEPS_OK;
}

extern "C" steps_status steps_emu_gradients(steps_emu *e, const float *x, const float *t, float *grads,
                                            float *loss) {
    if (!e || !x || !t || !grads) {
        set_error("steps_emu_gradients: bad arguments");
        return STEPS_EINVAL;
    }
    const int B = e->B;
    STEPS_CUDA(cudaMemcpyAsync(e->xs, x, (size_t)B * kIn * 4, cudaMemcpyDefault, e->st));
    STEPS_CUDA(cudaMemcpyAsync(e->ts, t, (size_t)B * 4, cudaMemcpyDefault, e->st));
    gather_kernel<<<blocks((int64_t)B * kInP, 256), 256, 0, e->st>>>(B, B, e->xs, e->ts, nullptr, nullptr, 0,
                                                                     e->act[0], e->actT[0], e->tgt);
    STEPS_CUDA(cudaGetLastError());
    STEPS_CUDA(forward(e, B));
    loss_kernel<<<1, 1024, 0, e->st>>>(B, e->z[kLayers - 1], e->tgt, e->dz[0], e->dzb[0], e->dzt[0], B, nullptr,
                                       nullptr, nullptr, nullptr, e->loss_one);
    STEPS_CUDA(cudaGetLastError());
    STEPS_CUDA(backward(e));
    std::vector<float> padded(kP);
    float l = 0.f;
    STEPS_CUDA(cudaMemcpyAsync(padded.data(), e->g, 4 * kP, cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaMemcpyAsync(&l, e->loss_one, 4, cudaMemcpyDeviceToHost, e->st));
    STEPS_CUDA(cudaStreamSynchronize(e->st));
    unpad_params(padded, grads);
    if (loss) *loss = l;
    return STEPS_OK;
}

extern "C" steps_status steps_emu_get_params(steps_emu *e, float *params, float *adam_m, float *adam_v,
                                             int64_t *adam_steps) {
    if (!e) {
        set_error("steps_emu_get_params: null context");
        return STEPS_EINVAL;
    }
    float *dst[3] = {params, adam_m, adam_v};
    const float *src[3] = {e->w, e->m, e->v};
    std::vector<float> padded(kP);
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        STEPS_CUDA(cudaMemcpyAsync(padded.data(), src[k], 4 * kP, cudaMemcpyDeviceToHost, e->st));
        STEPS_CUDA(cudaStreamSynchronize(e->st));
        unpad_params(padded, dst[k]);
    }
    if (adam_steps) *adam_steps = e->adam_steps;
    return STEPS_OK;
}

extern "C" void steps_emu_free(steps_emu *e) {
    if (!e) return;
    if (e->st) cudaStreamSynchronize(e->st);
    drop_graph(e);
    if (e->rows) counted_free(e->rows, e->steps_bytes);
    if (e->xd) counted_free(e->xd, e->data_bytes);
    if (e->arena) counted_free(e->arena, e->arena_bytes);
    if (e->own_stream && e->st) cudaStreamDestroy(e->st);
    delete e;
}

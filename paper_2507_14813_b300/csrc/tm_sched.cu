// Learned scheduling: a small cost model predicts each root edge's search
// cost, and the plan orders roots by predicted cost (largest first) and cuts
// the predicted-heavy ones into slices that other warps take.
//
// The paper balances load reactively (intra-/inter-warp rebalancing,
// Section 4.5); it has no learned component.  This file adds one:
//   k_features   8 per-root features (log1p): out/in-degree of the root's
//                destination, out-degree of its source, the delta-window
//                lengths of those three lists after the root, tree depth and
//                the root node's fan-out;
//   k_mlp_fwd    8 -> 64 -> 64 -> 1 perceptron, ReLU, FP16 weights, FP32
//                accumulation, standardised inputs;
//   k_mlp_grad   the mean-squared-error gradient of a minibatch (chain rule,
//                one thread per sample, FP32 accumulation) into per-block
//                partial sums, which k_grad_sum adds in block order: no
//                floating-point atomics, so training is reproducible run to
//                run (and with it the plan);
//   k_adam       Adam on FP32 master weights, refreshing the FP16 copy;
//   k_plan_keys  sort keys (descending predicted cost) and split counts.
// Labels are log1p of the work each root's search measured (adjacency
// entries scanned + probes), from the mining kernel's work counters.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tm_internal.h"

struct tm_model {
    float *master = nullptr;   // TM_MODEL_PARAMS fp32
    __half *half = nullptr;    // fp16 copy used by the kernels
    float *m = nullptr, *v = nullptr, *grad = nullptr;
    float *part = nullptr;     // kGradSlots x (TM_MODEL_PARAMS + 1): per-block gradient and loss sums
    float *norm = nullptr;     // 16: feature mean[8], inverse std[8]
    float *acc = nullptr;      // loss accumulator
    int64_t step = 0;
};

namespace tmo {
namespace {

constexpr int kIn = TM_FEATURES;
constexpr int kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kParams = oB3 + 1;
static_assert(kParams == TM_MODEL_PARAMS, "parameter count");
constexpr int kGradThreads = 64;
constexpr int kGradSlots = 64;      // blocks of a gradient launch, each with its own partial sums
constexpr int kPart = kParams + 1;  // one slot: the gradient, then the loss
constexpr int kNormThreads = 256;

__device__ __forceinline__ float h2f(__half x) { return __half2float(x); }

__device__ int32_t win_end(const int64_t *__restrict__ t, int64_t E, int32_t r, int64_t limit) {
    int64_t lo = r, step = 1, hi = E;
    while (true) {
        int64_t q = lo + step;
        if (q >= E) break;
        if (__ldg(t + q) <= limit) { lo = q; step <<= 1; } else { hi = q; break; }
    }
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (__ldg(t + mid) <= limit) lo = mid; else hi = mid;
    }
    return (int32_t)lo;
}

__device__ int64_t ub(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&adj[mid].y) <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_features(DevGraph g, const int32_t *roots, int64_t n, int64_t delta, float depth, float fanout,
                           float *X) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t r = roots[i];
    float *x = X + i * kIn;
    if (r < 0 || r >= g.E) {                 // a root outside the graph has no features
        for (int f = 0; f < kIn; f++) x[f] = 0.f;
        return;
    }
    const int32_t a = __ldg(g.src + r), b = __ldg(g.dst + r);
    const int64_t t0 = __ldg(g.t + r);
    const int64_t lim = (delta > 0 && t0 > INT64_MAX - delta) ? INT64_MAX : t0 + delta;
    const int32_t hi = win_end(g.t, g.E, r, lim);
    const int64_t ob0 = __ldg(g.out_off + b), ob1 = __ldg(g.out_off + b + 1);
    const int64_t ib0 = __ldg(g.in_off + b), ib1 = __ldg(g.in_off + b + 1);
    const int64_t oa0 = __ldg(g.out_off + a), oa1 = __ldg(g.out_off + a + 1);
    const float wob = (float)(ub(g.out_adj, ob0, ob1, hi) - ub(g.out_adj, ob0, ob1, r));
    const float wib = (float)(ub(g.in_adj, ib0, ib1, hi) - ub(g.in_adj, ib0, ib1, r));
    const float woa = (float)(ub(g.out_adj, oa0, oa1, hi) - ub(g.out_adj, oa0, oa1, r));
    x[0] = log1pf((float)(ob1 - ob0));
    x[1] = log1pf((float)(ib1 - ib0));
    x[2] = log1pf((float)(oa1 - oa0));
    x[3] = log1pf(wob);
    x[4] = log1pf(wib);
    x[5] = log1pf(woa);
    x[6] = log1pf(depth);
    x[7] = log1pf(fanout);
}

// sums[f] and sums[8 + f] of feature f and its square
// Feature mean and inverse standard deviation over n samples, one block:
// each thread sums a fixed stride of samples, then a fixed-order tree adds
// the threads' sums (FP64), so the result does not depend on scheduling.
__global__ void __launch_bounds__(kNormThreads) k_feat_norm(const float *X, int64_t n, float *norm) {
    __shared__ double s[2 * kIn][kNormThreads];
    double a[2 * kIn];
#pragma unroll
    for (int f = 0; f < 2 * kIn; f++) a[f] = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads)
#pragma unroll
        for (int f = 0; f < kIn; f++) {
            const double x = X[i * kIn + f];
            a[f] += x;
            a[kIn + f] += x * x;
        }
#pragma unroll
    for (int f = 0; f < 2 * kIn; f++) s[f][threadIdx.x] = a[f];
    __syncthreads();
    for (int h = kNormThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int f = 0; f < 2 * kIn; f++) s[f][threadIdx.x] += s[f][threadIdx.x + h];
        __syncthreads();
    }
    const int f = threadIdx.x;
    if (f >= kIn) return;
    const double mean = s[f][0] / (double)n;
    const double var = fmax(s[kIn + f][0] / (double)n - mean * mean, 0.0);
    norm[f] = (float)mean;
    norm[kIn + f] = var > 1e-8 ? (float)(1.0 / sqrt(var)) : 1.f;
}

__device__ __forceinline__ void load_weights(const __half *W, __half *sW) {
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) sW[i] = W[i];
}

__global__ void k_mlp_fwd(const __half *W, const float *norm, const float *X, int64_t n, float *Y) {
    __shared__ __half sW[kParams];
    __shared__ float sN[2 * kIn];
    load_weights(W, sW);
    if (threadIdx.x < 2 * kIn) sN[threadIdx.x] = norm[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[kIn];
#pragma unroll
    for (int f = 0; f < kIn; f++) x[f] = (X[i * kIn + f] - sN[f]) * sN[kIn + f];
    float h1[kH];
#pragma unroll
    for (int j = 0; j < kH; j++) {
        float z = h2f(sW[oB1 + j]);
#pragma unroll
        for (int f = 0; f < kIn; f++) z = fmaf(h2f(sW[oW1 + j * kIn + f]), x[f], z);
        h1[j] = fmaxf(z, 0.f);
    }
    float y = h2f(sW[oB3]);
    for (int j = 0; j < kH; j++) {
        float z = h2f(sW[oB2 + j]);
#pragma unroll
        for (int q = 0; q < kH; q++) z = fmaf(h2f(sW[oW2 + j * kH + q]), h1[q], z);
        y = fmaf(h2f(sW[oW3 + j]), fmaxf(z, 0.f), y);
    }
    Y[i] = y;
}

// Gradient of sum over the minibatch of (y - t)^2 * inv_n, and that loss,
// into per-block partial sums: block b takes the 64-sample tiles b,
// b + gridDim.x, ... in that order and owns part[b * kPart .. + kPart)
// (every parameter's sum belongs to one thread of the block, the loss to
// thread 0), so nothing is added atomically.
__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const __half *W, const float *norm, const float *X,
                                                           const float *T, int64_t n, float inv_n, float *part) {
    __shared__ __half sW[kParams];
    __shared__ float sN[2 * kIn];
    __shared__ float sX[kGradThreads][kIn];
    __shared__ float sH1[kGradThreads][kH + 1];   // h1, later dz1
    __shared__ float sH2[kGradThreads][kH + 1];   // h2, later dz2
    __shared__ float sDy[kGradThreads];
    __shared__ float sE[kGradThreads];            // squared error * inv_n
    load_weights(W, sW);
    if (threadIdx.x < 2 * kIn) sN[threadIdx.x] = norm[threadIdx.x];
    __syncthreads();
    const int s = threadIdx.x;
    float *slot = part + (int64_t)blockIdx.x * kPart;
    const int64_t n_tiles = (n + kGradThreads - 1) / kGradThreads;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;
        auto put = [&](int idx, float g) { slot[idx] = first ? g : slot[idx] + g; };
        const int64_t i = tile * kGradThreads + s;
        const bool live = i < n;
        // forward
#pragma unroll
        for (int f = 0; f < kIn; f++) sX[s][f] = live ? (X[i * kIn + f] - sN[f]) * sN[kIn + f] : 0.f;
        for (int j = 0; j < kH; j++) {
            float z = h2f(sW[oB1 + j]);
#pragma unroll
            for (int f = 0; f < kIn; f++) z = fmaf(h2f(sW[oW1 + j * kIn + f]), sX[s][f], z);
            sH1[s][j] = live ? fmaxf(z, 0.f) : 0.f;
        }
        float y = h2f(sW[oB3]);
        for (int j = 0; j < kH; j++) {
            float z = h2f(sW[oB2 + j]);
            for (int q = 0; q < kH; q++) z = fmaf(h2f(sW[oW2 + j * kH + q]), sH1[s][q], z);
            const float h = live ? fmaxf(z, 0.f) : 0.f;
            sH2[s][j] = h;
            y = fmaf(h2f(sW[oW3 + j]), h, y);
        }
        const float err = live ? y - T[i] : 0.f;
        sDy[s] = 2.f * err * inv_n;
        sE[s] = err * err * inv_n;
        __syncthreads();
        // output layer: dW3[j] = sum_s dy_s h2_s[j]; the loss
        {
            const int j = s;
            float g = 0.f;
            for (int q = 0; q < kGradThreads; q++) g = fmaf(sDy[q], sH2[q][j], g);
            put(oW3 + j, g);
            if (s == 0) {
                float b = 0.f, l = 0.f;
                for (int q = 0; q < kGradThreads; q++) {
                    b += sDy[q];
                    l += sE[q];
                }
                put(oB3, b);
                put(kParams, l);
            }
        }
        __syncthreads();
        // dz2 = dy * W3 where h2 > 0 (overwrites h2 of this sample)
        for (int j = 0; j < kH; j++) sH2[s][j] = (sH2[s][j] > 0.f) ? sDy[s] * h2f(sW[oW3 + j]) : 0.f;
        __syncthreads();
        // dW2[j][q] = sum_s dz2_s[j] h1_s[q]; db2[j] = sum_s dz2_s[j]
        {
            const int j = s;
            float b = 0.f;
            for (int q = 0; q < kGradThreads; q++) b += sH2[q][j];
            put(oB2 + j, b);
            for (int q = 0; q < kH; q++) {
                float g = 0.f;
                for (int r = 0; r < kGradThreads; r++) g = fmaf(sH2[r][j], sH1[r][q], g);
                put(oW2 + j * kH + q, g);
            }
        }
        __syncthreads();
        // dz1[q] = sum_j W2[j][q] dz2[j] where h1 > 0 (overwrites h1 of this sample)
        {
            float d[kH];
            for (int q = 0; q < kH; q++) {
                float z = 0.f;
                for (int j = 0; j < kH; j++) z = fmaf(h2f(sW[oW2 + j * kH + q]), sH2[s][j], z);
                d[q] = z;
            }
            for (int q = 0; q < kH; q++) sH1[s][q] = (sH1[s][q] > 0.f) ? d[q] : 0.f;
        }
        __syncthreads();
        // dW1[q][f] = sum_s dz1_s[q] x_s[f]; db1[q] = sum_s dz1_s[q]
        {
            const int q = s;
            float b = 0.f;
            float g[kIn];
#pragma unroll
            for (int f = 0; f < kIn; f++) g[f] = 0.f;
            for (int r = 0; r < kGradThreads; r++) {
                const float d = sH1[r][q];
                b += d;
#pragma unroll
                for (int f = 0; f < kIn; f++) g[f] = fmaf(d, sX[r][f], g[f]);
            }
            put(oB1 + q, b);
#pragma unroll
            for (int f = 0; f < kIn; f++) put(oW1 + q * kIn + f, g[f]);
        }
        __syncthreads();                 // the next tile overwrites the shared arrays
    }
}

// grad[i] = the blocks' partial sums of parameter i, added in block order;
// the loss likewise, stored (add == 0) or added (add == 1) to *loss.
__global__ void k_grad_sum(const float *part, int n_blocks, float *grad, float *loss, int add) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPart) return;
    float v = 0.f;
    for (int b = 0; b < n_blocks; b++) v += part[(int64_t)b * kPart + i];
    if (i < kParams) grad[i] = v;
    else *loss = add ? *loss + v : v;
}

__global__ void k_adam(float *w, __half *wh, float *m, float *v, const float *g, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wh[i] = __float2half_rn(wi);
}

__global__ void k_to_half(const float *w, __half *wh, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wh[i] = __float2half_rn(w[i]);
}

// descending predicted cost -> ascending key; split count from predicted work
__global__ void k_plan_keys(const float *Y, int64_t n, float unit_log, int32_t max_split, float thread_log,
                            uint32_t *key, int32_t *idx, int32_t *split) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float y = Y[i];
    uint32_t b = __float_as_uint(y);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // order-preserving
    key[i] = ~b;
    idx[i] = (int32_t)i;
    // slices of about exp(unit_log) predicted work each
    const float d = y - unit_log;
    int32_t sp = d <= 0.f ? 1 : (int32_t)fminf((float)max_split, ceilf(expf(fminf(d, 30.f))));
    if (y < thread_log) sp = 0;                        // predicted light: the thread tier
    split[i] = sp;
}

__global__ void k_plan_apply(const int32_t *order, const int32_t *roots, const int32_t *split_in, int64_t n,
                             int32_t *roots_out, int32_t *split_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t j = order[i];
    roots_out[i] = roots[j];
    split_out[i] = split_in[j];
}

unsigned grid(int64_t n, int b = 256) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

}  // namespace

int sort_u32_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s);

}  // namespace tmo

using namespace tmo;

extern "C" {

int tm_features(const tm_graph *g, const tm_tree *tr, const int32_t *roots, int64_t n_roots, float *feats,
                void *stream) {
    if (!g || !tr || (!roots && n_roots > 0) || (!feats && n_roots > 0) || n_roots < 0) {
        set_error("tm_features: bad argument");
        return TM_EINVAL;
    }
    if (n_roots == 0) return TM_OK;
    int64_t dmax = 0;
    for (int64_t d : tr->h.motif_delta) dmax = std::max(dmax, d);
    const float depth = (float)tr->h.depth;
    const float fanout = (float)tr->h.nodes[0].children.size();
    k_features<<<grid(n_roots), 256, 0, (cudaStream_t)stream>>>(g->d, roots, n_roots, dmax, depth, fanout, feats);
    TM_CUDA_TRY(cudaGetLastError());
    return TM_OK;
}

int tm_model_create(uint64_t seed, tm_model **out) {
    if (!out) { set_error("tm_model_create: out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    tm_model *m = new tm_model();
    // He initialisation from a splitmix64 stream; biases zero
    std::vector<float> w(kParams, 0.f);
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() {
        double u1 = std::max(next(), 1e-300), u2 = next();
        return (float)(std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    };
    for (int i = 0; i < kH * kIn; i++) w[oW1 + i] = normal() * std::sqrt(2.f / kIn);
    for (int i = 0; i < kH * kH; i++) w[oW2 + i] = normal() * std::sqrt(2.f / kH);
    for (int i = 0; i < kH; i++) w[oW3 + i] = normal() * std::sqrt(1.f / kH);
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&m->master, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->half, sizeof(__half) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(float) * kGradSlots * kPart);
    if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * 2 * kIn);
    if (e == cudaSuccess) e = cudaMalloc(&m->acc, sizeof(float) * 32);
    std::vector<float> norm(2 * kIn, 0.f);
    for (int f = 0; f < kIn; f++) norm[kIn + f] = 1.f;
    if (e == cudaSuccess) e = cudaMemcpy(m->master, w.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->norm, norm.data(), sizeof(float) * 2 * kIn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * kParams);
    if (e == cudaSuccess) {
        k_to_half<<<grid(kParams), 256>>>(m->master, m->half, kParams);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        set_error(std::string("tm_model_create: ") + cudaGetErrorString(e));
        tm_model_free(m);
        return e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA;
    }
    *out = m;
    return TM_OK;
}

int tm_model_free(tm_model *m) {
    if (!m) return TM_OK;
    cudaFree(m->master);
    cudaFree(m->half);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->part);
    cudaFree(m->norm);
    cudaFree(m->acc);
    delete m;
    return TM_OK;
}

int tm_model_get_params(const tm_model *m, float *params, float *norm) {
    if (!m) { set_error("tm_model_get_params: NULL model"); return TM_EINVAL; }
    if (params) TM_CUDA_TRY(cudaMemcpy(params, m->master, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    if (norm) TM_CUDA_TRY(cudaMemcpy(norm, m->norm, sizeof(float) * 2 * kIn, cudaMemcpyDeviceToHost));
    return TM_OK;
}

int tm_model_set_params(tm_model *m, const float *params, const float *norm) {
    if (!m) { set_error("tm_model_set_params: NULL model"); return TM_EINVAL; }
    if (params) {
        TM_CUDA_TRY(cudaMemcpy(m->master, params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
        k_to_half<<<grid(kParams), 256>>>(m->master, m->half, kParams);
        TM_CUDA_TRY(cudaGetLastError());
    }
    if (norm) TM_CUDA_TRY(cudaMemcpy(m->norm, norm, sizeof(float) * 2 * kIn, cudaMemcpyHostToDevice));
    TM_CUDA_TRY(cudaDeviceSynchronize());
    return TM_OK;
}

int tm_model_fit_norm(tm_model *m, const float *feats, int64_t n, void *stream) {
    if (!m || !feats || n <= 0) { set_error("tm_model_fit_norm: bad argument"); return TM_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    k_feat_norm<<<1, kNormThreads, 0, s>>>(feats, n, m->norm);
    TM_CUDA_TRY(cudaGetLastError());
    return TM_OK;
}

int tm_model_predict(const tm_model *m, const float *feats, int64_t n, float *out, void *stream) {
    if (!m || n < 0 || (n > 0 && (!feats || !out))) { set_error("tm_model_predict: bad argument"); return TM_EINVAL; }
    if (n == 0) return TM_OK;
    k_mlp_fwd<<<grid(n, 128), 128, 0, (cudaStream_t)stream>>>(m->half, m->norm, feats, n, out);
    TM_CUDA_TRY(cudaGetLastError());
    return TM_OK;
}

namespace {
// m->grad = the gradient of the mean squared error over n samples; the loss
// stored (add == 0) or added (add == 1) to *loss.  Reproducible: per-block
// partial sums in fixed slots, added in block order.
int gradient(const tm_model *m, const float *feats, const float *labels, int64_t n, float *loss, int add,
             cudaStream_t s) {
    const int64_t n_tiles = (n + kGradThreads - 1) / kGradThreads;
    const int blocks = (int)std::min<int64_t>(n_tiles, kGradSlots);
    k_mlp_grad<<<blocks, kGradThreads, 0, s>>>(m->half, m->norm, feats, labels, n, 1.f / (float)n, m->part);
    k_grad_sum<<<grid(kPart), 256, 0, s>>>(m->part, blocks, m->grad, loss, add);
    TM_CUDA_TRY(cudaGetLastError());
    return TM_OK;
}
}  // namespace

int tm_model_loss_grad(const tm_model *m, const float *feats, const float *labels, int64_t n, float *loss,
                       float *grad, void *stream) {
    if (!m || n <= 0 || !feats || !labels) { set_error("tm_model_loss_grad: bad argument"); return TM_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    TM_TRY(gradient(m, feats, labels, n, m->acc, 0, s));
    if (loss) TM_CUDA_TRY(cudaMemcpyAsync(loss, m->acc, sizeof(float), cudaMemcpyDeviceToHost, s));
    if (grad) TM_CUDA_TRY(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
    TM_CUDA_TRY(cudaStreamSynchronize(s));
    return TM_OK;
}

int tm_model_train(tm_model *m, const float *feats, const float *labels, int64_t n, int32_t epochs, int32_t batch,
                   float lr, float *loss_history, void *stream) {
    if (!m || n <= 0 || !feats || !labels || epochs < 0 || batch <= 0 || !(lr > 0)) {
        set_error("tm_model_train: bad argument");
        return TM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ep++) {
        TM_CUDA_TRY(cudaMemsetAsync(m->acc + 1, 0, sizeof(float), s));
        for (int64_t lo = 0; lo < n; lo += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - lo);
            TM_TRY(gradient(m, feats + lo * kIn, labels + lo, nb, m->acc + 1, 1, s));
            m->step++;
            const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
            k_adam<<<grid(kParams), 256, 0, s>>>(m->master, m->half, m->m, m->v, m->grad, kParams, lr, b1, b2, eps,
                                                 c1, c2);
            TM_CUDA_TRY(cudaGetLastError());
        }
        if (loss_history) {
            float tot = 0.f;
            TM_CUDA_TRY(cudaMemcpyAsync(&tot, m->acc + 1, sizeof(float), cudaMemcpyDeviceToHost, s));
            TM_CUDA_TRY(cudaStreamSynchronize(s));
            const int64_t nbatches = (n + batch - 1) / batch;
            loss_history[ep] = tot / (float)nbatches;
        }
    }
    TM_CUDA_TRY(cudaStreamSynchronize(s));
    return TM_OK;
}

namespace {
int plan(const tm_model *m, const float *feats, const int32_t *roots, int64_t n, double unit_work, int32_t max_split,
         double thread_work, int32_t *roots_out, int32_t *split_out, void *stream, const char *who) {
    if (!m || n < 0 || (n > 0 && (!feats || !roots || !roots_out || !split_out)) || !(unit_work >= 1.0) ||
        max_split < 1 || !(thread_work >= 0.0)) {
        set_error(std::string(who) + ": bad argument");
        return TM_EINVAL;
    }
    if (n == 0) return TM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char *buf = nullptr;
    const size_t bytes = (size_t)n * (sizeof(float) + sizeof(uint32_t) + 2 * sizeof(int32_t));
    TM_CUDA_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    float *y = (float *)buf;
    uint32_t *key = (uint32_t *)(y + n);
    int32_t *idx = (int32_t *)(key + n);
    int32_t *split = idx + n;
    int rc = TM_OK;
    // predictions are log1p(work); no root is below a threshold of 0
    const float thread_log = thread_work > 0.0 ? (float)std::log1p(thread_work) : -INFINITY;
    k_mlp_fwd<<<grid(n, 128), 128, 0, s>>>(m->half, m->norm, feats, n, y);
    k_plan_keys<<<grid(n), 256, 0, s>>>(y, n, (float)std::log(unit_work), max_split, thread_log, key, idx, split);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = TM_ECUDA; }
    if (rc == TM_OK) rc = sort_u32_pairs(key, idx, n, 32, s);
    if (rc == TM_OK) {
        k_plan_apply<<<grid(n), 256, 0, s>>>(idx, roots, split, n, roots_out, split_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = TM_ECUDA; }
    }
    cudaFreeAsync(buf, s);
    return rc;
}
}  // namespace

int tm_plan(const tm_model *m, const float *feats, const int32_t *roots, int64_t n, double unit_work,
            int32_t max_split, int32_t *roots_out, int32_t *split_out, void *stream) {
    return plan(m, feats, roots, n, unit_work, max_split, 0.0, roots_out, split_out, stream, "tm_plan");
}

int tm_plan_tiers(const tm_model *m, const float *feats, const int32_t *roots, int64_t n, double unit_work,
                  int32_t max_split, double thread_work, int32_t *roots_out, int32_t *split_out, void *stream) {
    return plan(m, feats, roots, n, unit_work, max_split, thread_work, roots_out, split_out, stream, "tm_plan_tiers");
}

}  // extern "C"

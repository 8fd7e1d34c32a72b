// cdf.cu -- the learned splitter proposal: a 1-32-32-1 CDF network of the
// keys, trained on the device from (key, rank) pairs and inverted to propose
// the splitters of the next job before round 1 of the histogram rounds.
//
// The paper proposes no learned model; its rounds (Sec. 4.2.2) accept any
// candidate cuts, and this network is one source of them.  Everything is
// float32 on the CUDA cores: the network has 1153 parameters and a training
// batch holds a few thousand points, far too small a contraction for tensor
// cores to matter.  Under HSS_CDF_W_BF16 every evaluation uses the parameters
// rounded to bfloat16 (the float32 master copy takes the Adam updates).
//
//   feature   x = clip((raw(u) - lo) / (hi - lo), 0, 1), raw(u) = u or
//             log2(1 + u), u = order-preserving key bits (double precision)
//   network   y = w3 . relu(W2 relu(w1 x + b1) + b2) + b3
//   loss      L = (1/n) sum_b (y_b - rank_b / N)^2
//   update    Adam (Kingma and Ba, 2015), bias-corrected
#include "hss_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace hss {
namespace {

constexpr int kH = HSS_CDF_HIDDEN;
constexpr int kP = HSS_CDF_NPARAM;
constexpr int kOffB1 = kH, kOffW2 = 2 * kH, kOffB2 = 2 * kH + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
constexpr int kGradThreads = 256;
constexpr int kMaxGradBlocks = 32;  // training shares the GPU with the sorts it serves: a few SMs
constexpr int kPartStride = kP + 3;  // gradient, loss partial, padding
constexpr int kStage = kH + 1;       // padded row of a staged activation vector
constexpr uint32_t kInitTag = 0x43444621u;
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kAdamEps = 1e-8f;

__device__ __forceinline__ float feature_of(uint64_t bits, const hss_cdf_model* M, uint64_t flip) {
    const double u = (double)(bits ^ flip);
    const double raw = M->feature == HSS_CDF_LOG ? log2(1.0 + u) : u;
    double x = (raw - M->lo) / (M->hi - M->lo);
    x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
    return (float)x;
}

// Parameter k as the network uses it: float32, or rounded to bfloat16
// (nearest, ties to even) under HSS_CDF_W_BF16.
__device__ __forceinline__ float weight_of(const hss_cdf_model* M, int k) {
    const float w = M->theta[k];
    return M->weights == HSS_CDF_W_BF16 ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

// y(x) with the parameters in shared memory (every thread reads the same
// weight at the same time: broadcasts).
__device__ __forceinline__ float net(const float* th, float x) {
    float h1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) h1[i] = fmaxf(fmaf(th[i], x, th[kOffB1 + i]), 0.f);
    float y = th[kOffB3];
#pragma unroll 4
    for (int i = 0; i < kH; ++i) {
        float a = th[kOffB2 + i];
#pragma unroll
        for (int j = 0; j < kH; ++j) a = fmaf(th[kOffW2 + i * kH + j], h1[j], a);
        y = fmaf(th[kOffW3 + i], fmaxf(a, 0.f), y);
    }
    return y;
}

__global__ void k_cdf_init(hss_cdf_model* M, uint64_t seed, int feature, int key_type, double lo, double hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        M->step = 0; M->feature = feature; M->key_type = key_type; M->weights = HSS_CDF_W_FP32; M->lo = lo; M->hi = hi;
    }
    if (k >= kP) return;
    const Philox4 r = philox4x32_10((uint32_t)k, 0u, 0u, kInitTag, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u = (float)(r.v[0] >> 8) * (1.0f / 16777216.0f);
    const float scale = 0.4330127018922193f;  // sqrt(6 / 32)
    float w;
    if (k < kOffB1) {
        w = ((k & 1) ? -1.f : 1.f) * (1.f + u) * 4.f;
    } else if (k < kOffW2) {  // knot of hidden-1 unit i at (i + 0.5) / 32
        const int i = k - kOffB1;
        const Philox4 r1 = philox4x32_10((uint32_t)i, 0u, 0u, kInitTag, (uint32_t)seed, (uint32_t)(seed >> 32));
        const float u1 = (float)(r1.v[0] >> 8) * (1.0f / 16777216.0f);
        const float w1 = ((i & 1) ? -1.f : 1.f) * (1.f + u1) * 4.f;
        w = -w1 * ((float)i + 0.5f) / (float)kH;
    } else if (k < kOffB2) {
        w = (2.f * u - 1.f) * scale;
    } else if (k < kOffW3) {
        w = 0.1f;
    } else if (k < kOffB3) {
        w = (2.f * u - 1.f) * scale;
    } else {
        w = 0.5f;
    }
    M->theta[k] = w;
    M->m[k] = 0.f;
    M->v[k] = 0.f;
}

// Partial gradient of the mean squared error over a grid-stride share of the
// n points.  Each thread runs the forward and backward pass of one point;
// the activations and their gradients are staged in shared memory and every
// thread then sums its own gradient entries over the 256 staged points, so
// each CTA writes one deterministic partial.
__global__ __launch_bounds__(kGradThreads) void k_cdf_grad(const hss_cdf_model* __restrict__ M,
                                                           const uint64_t* __restrict__ keys,
                                                           const uint64_t* __restrict__ ranks, uint32_t n, double invN,
                                                           float inv_n, float* __restrict__ part) {
    extern __shared__ __align__(16) float sm[];
    float* th = sm;                                 // kP (+3)
    float* H1s = th + kP + 3;                       // 256 x 33
    float* H2s = H1s + kGradThreads * kStage;
    float* DZ2s = H2s + kGradThreads * kStage;
    float* DZ1s = DZ2s + kGradThreads * kStage;
    float* Xs = DZ1s + kGradThreads * kStage;       // 256
    float* Ds = Xs + kGradThreads;                  // 256
    float* Ls = Ds + kGradThreads;                  // 256
    const int tid = threadIdx.x;
    for (int k = tid; k < kP; k += kGradThreads) th[k] = weight_of(M, k);
    const uint64_t flip = M->key_type == HSS_KEY_I64 ? kSignBit : 0ull;
    __syncthreads();

    float accW2[4] = {0.f, 0.f, 0.f, 0.f};
    float accS = 0.f;  // small entry owned by threads 0..128, loss by thread 129
    for (uint64_t base = (uint64_t)blockIdx.x * kGradThreads; base < n; base += (uint64_t)gridDim.x * kGradThreads) {
        const uint64_t b = base + tid;
        float x = 0.f, d = 0.f, l = 0.f;
        float h1[kH], h2[kH], dz2[kH];
        if (b < n) {
            x = feature_of(keys[b], M, flip);
            const float t = (float)((double)ranks[b] * invN);
#pragma unroll
            for (int i = 0; i < kH; ++i) h1[i] = fmaxf(fmaf(th[i], x, th[kOffB1 + i]), 0.f);
            float y = th[kOffB3];
#pragma unroll
            for (int i = 0; i < kH; ++i) {
                float a = th[kOffB2 + i];
#pragma unroll
                for (int j = 0; j < kH; ++j) a = fmaf(th[kOffW2 + i * kH + j], h1[j], a);
                h2[i] = fmaxf(a, 0.f);
                y = fmaf(th[kOffW3 + i], h2[i], y);
            }
            const float e = y - t;
            d = 2.f * e * inv_n;
            l = e * e;
#pragma unroll
            for (int i = 0; i < kH; ++i) dz2[i] = h2[i] > 0.f ? d * th[kOffW3 + i] : 0.f;
        } else {
#pragma unroll
            for (int i = 0; i < kH; ++i) { h1[i] = 0.f; h2[i] = 0.f; dz2[i] = 0.f; }
        }
#pragma unroll
        for (int i = 0; i < kH; ++i) {
            H1s[tid * kStage + i] = h1[i];
            H2s[tid * kStage + i] = h2[i];
            DZ2s[tid * kStage + i] = dz2[i];
        }
#pragma unroll 4
        for (int j = 0; j < kH; ++j) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < kH; ++i) a = fmaf(th[kOffW2 + i * kH + j], dz2[i], a);
            DZ1s[tid * kStage + j] = h1[j] > 0.f ? a : 0.f;
        }
        Xs[tid] = x;
        Ds[tid] = d;
        Ls[tid] = l;
        __syncthreads();
        // dW2[i][j] = sum_b dz2[b][i] h1[b][j]: thread owns entries tid + 256 q.
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * kGradThreads, i = e >> 5, j = e & 31;
            float a = accW2[q];
            for (int r = 0; r < kGradThreads; ++r) a = fmaf(DZ2s[r * kStage + i], H1s[r * kStage + j], a);
            accW2[q] = a;
        }
        if (tid < 130) {
            float a = accS;
            if (tid < 32) {              // dw1[j] = sum_b dz1[b][j] x_b
                for (int r = 0; r < kGradThreads; ++r) a = fmaf(DZ1s[r * kStage + tid], Xs[r], a);
            } else if (tid < 64) {       // db1[j]
                for (int r = 0; r < kGradThreads; ++r) a += DZ1s[r * kStage + tid - 32];
            } else if (tid < 96) {       // db2[i]
                for (int r = 0; r < kGradThreads; ++r) a += DZ2s[r * kStage + tid - 64];
            } else if (tid < 128) {      // dw3[i] = sum_b d_b h2[b][i]
                for (int r = 0; r < kGradThreads; ++r) a = fmaf(Ds[r], H2s[r * kStage + tid - 96], a);
            } else if (tid == 128) {     // db3
                for (int r = 0; r < kGradThreads; ++r) a += Ds[r];
            } else {                     // sum of squared errors
                for (int r = 0; r < kGradThreads; ++r) a += Ls[r];
            }
            accS = a;
        }
        __syncthreads();
    }
    float* out = part + (uint64_t)blockIdx.x * kPartStride;
#pragma unroll
    for (int q = 0; q < 4; ++q) out[kOffW2 + tid + q * kGradThreads] = accW2[q];
    if (tid < 32) out[tid] = accS;
    else if (tid < 64) out[kOffB1 + tid - 32] = accS;
    else if (tid < 96) out[kOffB2 + tid - 64] = accS;
    else if (tid < 128) out[kOffW3 + tid - 96] = accS;
    else if (tid == 128) out[kOffB3] = accS;
    else if (tid == 129) out[kP] = accS;
}

// Sum of the partials (in block order: deterministic), optional gradient and
// loss outputs, optional Adam step.
__global__ __launch_bounds__(1024) void k_cdf_adam(hss_cdf_model* M, const float* __restrict__ part, int G, float lr,
                                                   float inv_n, int apply, float* __restrict__ grad_out,
                                                   float* __restrict__ loss_out) {
    const uint32_t t = M->step + 1;
    const float c1 = (float)(1.0 - pow((double)kBeta1, (double)t));
    const float c2 = (float)(1.0 - pow((double)kBeta2, (double)t));
    for (int k = threadIdx.x; k < kP; k += blockDim.x) {
        float g = 0.f;
        for (int c = 0; c < G; ++c) g += part[(uint64_t)c * kPartStride + k];
        if (grad_out) grad_out[k] = g;
        if (apply) {
            const float m = kBeta1 * M->m[k] + (1.f - kBeta1) * g;
            const float v = kBeta2 * M->v[k] + (1.f - kBeta2) * g * g;
            M->m[k] = m;
            M->v[k] = v;
            M->theta[k] -= lr * (m / c1) / (sqrtf(v / c2) + kAdamEps);
        }
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int c = 0; c < G; ++c) l += part[(uint64_t)c * kPartStride + kP];
        if (loss_out) *loss_out = l * inv_n;
    }
    __syncthreads();
    if (apply && threadIdx.x == 0) M->step = t;
}

__global__ void k_cdf_set_weights(hss_cdf_model* M, int weights) { M->weights = weights; }

__global__ void k_cdf_eval(const hss_cdf_model* __restrict__ M, const uint64_t* __restrict__ keys, uint32_t n,
                           float* __restrict__ y) {
    __shared__ float th[kP];
    for (int k = threadIdx.x; k < kP; k += blockDim.x) th[k] = weight_of(M, k);
    __syncthreads();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const uint64_t flip = M->key_type == HSS_KEY_I64 ? kSignBit : 0ull;
    y[b] = net(th, feature_of(keys[b], M, flip));
}

// Cut q = (i-1) per + k of splitter i (1..p-1): target tau = i/p + delta
// (2k/(per-1) - 1) clipped to [0, 1] (i/p when per = 1); bisection for the
// smallest x in [0, 1] with y(x) >= tau, then the inverse feature map,
// clamped to the key range.
__global__ void k_cdf_propose(const hss_cdf_model* __restrict__ M, uint32_t p, uint32_t per, double delta, int iters,
                              uint64_t* __restrict__ out) {
    __shared__ float th[kP];
    for (int k = threadIdx.x; k < kP; k += blockDim.x) th[k] = weight_of(M, k);
    __syncthreads();
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (uint64_t)(p - 1) * per) return;
    const uint32_t i = (uint32_t)(q / per) + 1, k = (uint32_t)(q % per);
    double tau_d = (double)i / (double)p;
    if (per > 1) tau_d += delta * (2.0 * (double)k / (double)(per - 1) - 1.0);
    tau_d = tau_d < 0.0 ? 0.0 : (tau_d > 1.0 ? 1.0 : tau_d);
    const float tau = (float)tau_d;
    float a = 0.f, b = 1.f;
    for (int it = 0; it < iters; ++it) {
        const float mid = 0.5f * (a + b);
        if (net(th, mid) < tau) a = mid; else b = mid;
    }
    const double r = M->lo + (double)b * (M->hi - M->lo);
    const double u = M->feature == HSS_CDF_LOG ? exp2(r) - 1.0 : r;
    uint64_t bits;
    if (!(u > 0.0)) bits = 0ull;
    else if (u >= 18446744073709551615.0) bits = ~0ull;
    else bits = (uint64_t)u;
    const uint64_t flip = M->key_type == HSS_KEY_I64 ? kSignBit : 0ull;
    out[q] = bits ^ flip;
}

int grad_blocks(uint32_t n) { return (int)std::max<uint32_t>(1, std::min<uint32_t>(kMaxGradBlocks, (n + 255) / 256)); }

size_t grad_smem() { return (size_t)(kP + 3 + 4 * kGradThreads * kStage + 3 * kGradThreads) * sizeof(float); }

int launch_grad(const hss_cdf_model* M, const uint64_t* keys, const uint64_t* ranks, uint32_t n, uint64_t N,
                float* part, cudaStream_t st) {
    if (ensure_func_attrs((const void*)k_cdf_grad, (int)grad_smem()) != cudaSuccess) return HSS_ERR_CUDA;
    HSS_LAUNCH(k_cdf_grad, grad_blocks(n), kGradThreads, grad_smem(), st, M, keys, ranks, n, 1.0 / (double)N,
               (float)(1.0 / (double)n), part);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

bool raw_bound(uint64_t key, int feature, int key_type, double* out) {
    const uint64_t u = key ^ (key_type == HSS_KEY_I64 ? kSignBit : 0ull);
    *out = feature == HSS_CDF_LOG ? std::log2(1.0 + (double)u) : (double)u;
    return std::isfinite(*out);
}

}  // namespace
}  // namespace hss

using namespace hss;

extern "C" {

size_t hss_cdf_model_bytes(void) { return sizeof(hss_cdf_model); }

int hss_cdf_set_weights(hss_cdf_model* d_model, int weights, void* stream) {
    if (!d_model || (weights != HSS_CDF_W_FP32 && weights != HSS_CDF_W_BF16)) return HSS_ERR_INVALID;
    HSS_LAUNCH(k_cdf_set_weights, 1, 1, 0, (cudaStream_t)stream, d_model, weights);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

size_t hss_cdf_work_bytes(uint32_t n) { return (size_t)grad_blocks(n) * kPartStride * sizeof(float); }

int hss_cdf_init(hss_cdf_model* d_model, uint64_t seed, int feature, int key_type, uint64_t lo_key, uint64_t hi_key,
                 void* stream) {
    if (!d_model || (feature != HSS_CDF_LINEAR && feature != HSS_CDF_LOG)) return HSS_ERR_INVALID;
    if (key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) return HSS_ERR_INVALID;
    double lo, hi;
    if (!raw_bound(lo_key, feature, key_type, &lo) || !raw_bound(hi_key, feature, key_type, &hi) || !(hi > lo))
        return HSS_ERR_INVALID;
    HSS_LAUNCH(k_cdf_init, (kP + 255) / 256, 256, 0, (cudaStream_t)stream, d_model, seed, feature, key_type, lo, hi);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

int hss_cdf_grad(const hss_cdf_model* d_model, const void* d_keys, const uint64_t* d_ranks, uint32_t n, uint64_t N,
                 float* d_grad, float* d_loss, void* d_work, size_t work_bytes, void* stream) {
    if (!d_model || n == 0 || N == 0 || !d_keys || !d_ranks || !d_work) return HSS_ERR_INVALID;
    if (work_bytes < hss_cdf_work_bytes(n)) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    float* part = (float*)d_work;
    const int rc = launch_grad(d_model, (const uint64_t*)d_keys, d_ranks, n, N, part, st);
    if (rc != HSS_OK) return rc;
    HSS_LAUNCH(k_cdf_adam, 1, 1024, 0, st, const_cast<hss_cdf_model*>(d_model), part, grad_blocks(n), 0.f,
               (float)(1.0 / (double)n), 0, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

int hss_cdf_train(hss_cdf_model* d_model, const void* d_keys, const uint64_t* d_ranks, uint32_t n, uint64_t N,
                  uint32_t steps, float lr, float* d_loss, void* d_work, size_t work_bytes, void* stream) {
    if (!d_model || n == 0 || N == 0 || !d_keys || !d_ranks || !d_work || !(lr > 0.f)) return HSS_ERR_INVALID;
    if (work_bytes < hss_cdf_work_bytes(n)) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    float* part = (float*)d_work;
    for (uint32_t s = 0; s < steps; ++s) {
        const int rc = launch_grad(d_model, (const uint64_t*)d_keys, d_ranks, n, N, part, st);
        if (rc != HSS_OK) return rc;
        HSS_LAUNCH(k_cdf_adam, 1, 1024, 0, st, d_model, part, grad_blocks(n), lr, (float)(1.0 / (double)n), 1, nullptr,
                   s + 1 == steps ? d_loss : nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

int hss_cdf_eval(const hss_cdf_model* d_model, const void* d_keys, uint32_t n, float* d_y, void* stream) {
    if (!d_model || (n > 0 && (!d_keys || !d_y))) return HSS_ERR_INVALID;
    if (n == 0) return HSS_OK;
    HSS_LAUNCH(k_cdf_eval, (n + 255) / 256, 256, 0, (cudaStream_t)stream, d_model, (const uint64_t*)d_keys, n, d_y);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

int hss_cdf_propose(const hss_cdf_model* d_model, uint32_t p, uint32_t per_splitter, double delta, void* d_out_keys,
                    void* stream) {
    if (!d_model || p == 0 || per_splitter == 0 || !(delta >= 0.0) || (p > 1 && !d_out_keys)) return HSS_ERR_INVALID;
    if (p == 1) return HSS_OK;
    const uint64_t n = (uint64_t)(p - 1) * per_splitter;
    if (n > 0xffffffffull) return HSS_ERR_INVALID;
    HSS_LAUNCH(k_cdf_propose, (unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream, d_model, p, per_splitter, delta,
               40, (uint64_t*)d_out_keys);
    return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

}  // extern "C"

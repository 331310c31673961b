// Learned ROM error estimator: a 5 -> 64 -> 64 -> 1 network with tanh hidden
// units, trained by mean-squared error with Adam (Kingma & Ba 2015) on samples
// the reduction computes itself (the paper replaces its expensive error measure
// by a cheaper estimate, Sec. 5; here a network maps cheap features to the
// reduced model's true output error).
//
// Parameters (FP32 master copy, flat): W1 (64x5, row-major), b1, W2 (64x64), b2,
// W3 (1x64), b3.  Forward and backward passes use the weight matrices rounded
// to FP16 and accumulate in FP32; Adam updates the FP32 master copy.
//
// Training is one persistent CTA that runs every step: the mini-batch's
// activations (batch x 64, twice) stay in shared memory, the three GEMM-shaped
// products of each layer are done by all threads with conflict-free layouts
// (weights kept both row-major and transposed), gradients are reduced in a fixed
// order (deterministic), and the update of all 4609 parameters closes the step.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include "fsi_internal.h"

namespace fsi {

namespace {

constexpr int kIn = 5, kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kNP = oB3 + 1;   // 4609
static_assert(kNP == FSI_MLP_PARAMS, "parameter count");
constexpr int kTrainThreads = 256;
constexpr int kMaxBatch = 256;
constexpr int kS = kH + 1;     // padded row stride of the activation tiles

struct TrainSmem {
    float H1[kMaxBatch * kS];    // tanh(z1), then dL/dz1
    float H2[kMaxBatch * kS];    // tanh(z2), then dL/dz2
    float X[kMaxBatch * kIn];
    float t[kMaxBatch];
    float dy[kMaxBatch];
    float g[kNP];                // gradient of the step
    __half W1t[kIn * kH];        // [c][i]
    __half W2t[kH * kH];         // [j][i] (forward)
    __half W2r[kH * kH];         // [i][j] (backward)
    __half W3[kH];
    float red[kTrainThreads / 32];
};

__device__ float block_sum(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(float* P, float* M, float* V, const float* X,
                                                                  const float* T, const int32_t* order, int steps,
                                                                  int B, float lr, int step0, float* losses,
                                                                  float* grad_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const float inv_b = 1.f / float(B);
    for (int s = 0; s < steps; ++s) {
        // batch rows and FP16 weights of this step
        for (int e = tid; e < B * kIn; e += nt) {
            const int b = e / kIn, c = e - b * kIn;
            S.X[e] = X[int64_t(order[int64_t(s) * B + b]) * kIn + c];
        }
        for (int b = tid; b < B; b += nt) S.t[b] = T[order[int64_t(s) * B + b]];
        for (int e = tid; e < kH * kIn; e += nt) {
            const int i = e / kIn, c = e - i * kIn;
            S.W1t[c * kH + i] = __float2half_rn(P[oW1 + e]);
        }
        for (int e = tid; e < kH * kH; e += nt) {
            const int i = e / kH, j = e - i * kH;
            const __half w = __float2half_rn(P[oW2 + e]);
            S.W2r[e] = w;
            S.W2t[j * kH + i] = w;
        }
        for (int i = tid; i < kH; i += nt) S.W3[i] = __float2half_rn(P[oW3 + i]);
        __syncthreads();
        // forward
        for (int e = tid; e < B * kH; e += nt) {
            const int b = e / kH, i = e - b * kH;
            float z = P[oB1 + i];
#pragma unroll
            for (int c = 0; c < kIn; ++c) z = fmaf(__half2float(S.W1t[c * kH + i]), S.X[b * kIn + c], z);
            S.H1[b * kS + i] = tanhf(z);
        }
        __syncthreads();
        for (int e = tid; e < B * kH; e += nt) {
            const int b = e / kH, i = e - b * kH;
            float z = P[oB2 + i];
            for (int j = 0; j < kH; ++j) z = fmaf(__half2float(S.W2t[j * kH + i]), S.H1[b * kS + j], z);
            S.H2[b * kS + i] = tanhf(z);
        }
        __syncthreads();
        float l = 0.f;
        for (int b = tid; b < B; b += nt) {
            float y = P[oB3];
            for (int i = 0; i < kH; ++i) y = fmaf(__half2float(S.W3[i]), S.H2[b * kS + i], y);
            const float r = y - S.t[b];
            S.dy[b] = 2.f * r * inv_b;
            l += r * r;
        }
        l = block_sum(l, S.red);
        if (tid == 0 && losses) losses[s] = l * inv_b;
        __syncthreads();
        // backward: output layer
        for (int i = tid; i < kH; i += nt) {
            float a = 0.f;
            for (int b = 0; b < B; ++b) a = fmaf(S.dy[b], S.H2[b * kS + i], a);
            S.g[oW3 + i] = a;
        }
        if (tid == 0) {
            float a = 0.f;
            for (int b = 0; b < B; ++b) a += S.dy[b];
            S.g[oB3] = a;
        }
        __syncthreads();
        for (int e = tid; e < B * kH; e += nt) {
            const int b = e / kH, i = e - b * kH;
            const float h = S.H2[b * kS + i];
            S.H2[b * kS + i] = S.dy[b] * __half2float(S.W3[i]) * (1.f - h * h);   // dL/dz2
        }
        __syncthreads();
        // second layer: dW2 = dz2^T h1, db2, then dz1 = (dz2 W2) o (1 - h1^2) in place of h1
        for (int e = tid; e < kH * kH; e += nt) {
            const int i = e / kH, j = e - i * kH;
            float a = 0.f;
            for (int b = 0; b < B; ++b) a = fmaf(S.H2[b * kS + i], S.H1[b * kS + j], a);
            S.g[oW2 + e] = a;
        }
        for (int i = tid; i < kH; i += nt) {
            float a = 0.f;
            for (int b = 0; b < B; ++b) a += S.H2[b * kS + i];
            S.g[oB2 + i] = a;
        }
        __syncthreads();
        for (int e = tid; e < B * kH; e += nt) {
            const int b = e / kH, j = e - b * kH;
            float a = 0.f;
            for (int i = 0; i < kH; ++i) a = fmaf(S.H2[b * kS + i], __half2float(S.W2r[i * kH + j]), a);
            const float h = S.H1[b * kS + j];
            S.H1[b * kS + j] = a * (1.f - h * h);
        }
        __syncthreads();
        // first layer
        for (int e = tid; e < kH * kIn; e += nt) {
            const int i = e / kIn, c = e - i * kIn;
            float a = 0.f;
            for (int b = 0; b < B; ++b) a = fmaf(S.H1[b * kS + i], S.X[b * kIn + c], a);
            S.g[oW1 + e] = a;
        }
        for (int i = tid; i < kH; i += nt) {
            float a = 0.f;
            for (int b = 0; b < B; ++b) a += S.H1[b * kS + i];
            S.g[oB1 + i] = a;
        }
        __syncthreads();
        // Adam on the master copy
        const int k = step0 + s + 1;
        const float c1 = 1.f - powf(0.9f, float(k)), c2 = 1.f - powf(0.999f, float(k));
        for (int p = tid; p < kNP; p += nt) {
            const float g = S.g[p];
            if (grad_out && s + 1 == steps) grad_out[p] = g;
            const float m = 0.9f * M[p] + 0.1f * g;
            const float v = 0.999f * V[p] + 0.001f * g * g;
            M[p] = m;
            V[p] = v;
            P[p] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
        }
        __syncthreads();
    }
}

constexpr int kPredThreads = 128;

__global__ void __launch_bounds__(kPredThreads) mlp_predict_kernel(const float* P, const float* X, int n, float* y) {
    __shared__ __half W1t[kIn * kH];
    __shared__ __half W2r[kH * kH];
    __shared__ float W3[kH], b1[kH], b2[kH];
    for (int e = threadIdx.x; e < kH * kIn; e += blockDim.x) {
        const int i = e / kIn, c = e - i * kIn;
        W1t[c * kH + i] = __float2half_rn(P[oW1 + e]);
    }
    for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) W2r[e] = __float2half_rn(P[oW2 + e]);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        W3[i] = __half2float(__float2half_rn(P[oW3 + i]));
        b1[i] = P[oB1 + i];
        b2[i] = P[oB2 + i];
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x[kIn], h1[kH];
#pragma unroll
    for (int c = 0; c < kIn; ++c) x[c] = X[int64_t(q) * kIn + c];
#pragma unroll
    for (int i = 0; i < kH; ++i) {
        float z = b1[i];
#pragma unroll
        for (int c = 0; c < kIn; ++c) z = fmaf(__half2float(W1t[c * kH + i]), x[c], z);
        h1[i] = tanhf(z);
    }
    float out = P[oB3];
    for (int i = 0; i < kH; ++i) {
        float z = b2[i];
#pragma unroll
        for (int j = 0; j < kH; ++j) z = fmaf(__half2float(W2r[i * kH + j]), h1[j], z);
        out = fmaf(W3[i], tanhf(z), out);
    }
    y[q] = out;
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status mlp_train(float* params, float* adam_m, float* adam_v, const float* X, const float* T, int n,
                     const int32_t* order, int steps, int batch, float lr, int step0, float* losses, float* grad_out,
                     void* stream) {
    if (!(params && adam_m && adam_v && X && T && order && n > 0 && steps > 0 && batch > 0 &&
          batch <= kMaxBatch && step0 >= 0 && lr >= 0.f)) {
        set_error("mlp_train: bad arguments (batch must be in 1..256)");
        return FSI_EINVAL;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(TrainSmem)));
        attr = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_train_kernel<<<1, kTrainThreads, sizeof(TrainSmem), st>>>(params, adam_m, adam_v, X, T, order, steps, batch,
                                                                  lr, step0, losses, grad_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mlp_train: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    return FSI_OK;
}

fsi_status mlp_predict(const float* params, const float* X, int n, float* y, void* stream) {
    if (!(params && X && y && n > 0)) {
        set_error("mlp_predict: bad arguments");
        return FSI_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_predict_kernel<<<(n + kPredThreads - 1) / kPredThreads, kPredThreads, 0, st>>>(params, X, n, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mlp_predict: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    return FSI_OK;
}

}  // extern "C"

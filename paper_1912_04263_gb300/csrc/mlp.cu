// Learned rho policy: batched inference, training forward/backward and Adam
// for the 4-64-64-2 MLP (not part of the paper).  Operands are rounded to
// BF16 (weights, inputs, hidden activations and back-propagated signals) and
// every product is accumulated in FP32; master weights and Adam moments are
// FP32.  Gradients are summed per CTA and then across CTAs in a fixed order,
// so training is bitwise reproducible.
//
// Parameter vector (GBOSQP_POLICY_PARAMS floats, layout in policy.cuh):
// feature mean (4), feature std (4), W1 (64x4), b1, W2 (64x64), b2, W3 (2x64),
// b3, extras (4).  Features are raw: log ||r_prim||, log ||r_dual|| (scaled
// problem), log rho, log(1 + PCG steps since the last decision); the network
// sees bf16((f - mean) / std).  Loss: sum_k w_k (o_k - t_k)^2 / (2 N).
#include <math.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "policy.cuh"

namespace gb {
namespace {

constexpr int kMlpSamples = 16;  // samples per CTA in the training kernel (static smem < 48 KB)
constexpr int kNW = kOffExtra - kOffW1;  // trainable parameters (weights and biases)

__device__ __forceinline__ float relu(float a) { return a > 0.f ? a : 0.f; }

// Inference: one CTA per sample, through the solver's own device function.
__global__ void k_policy_forward(const float *P, const float *feat, int B, float *out) {
    __shared__ float x[kPolIn], h1[kPolHid], h2[kPolHid], o[kPolOut];
    const int b = blockIdx.x;
    if (b >= B) return;
    if (threadIdx.x < kPolIn)
        x[threadIdx.x] = bf16r((feat[b * kPolIn + threadIdx.x] - P[kOffMean + threadIdx.x]) / P[kOffStd + threadIdx.x]);
    __syncthreads();
    policy_forward(P, x, h1, h2, o);
    if (threadIdx.x < kPolOut) out[b * kPolOut + threadIdx.x] = o[threadIdx.x];
}

// Forward and backward for the samples idx[base .. base+count) of one CTA;
// writes the CTA's gradient (kNW floats, order W1 b1 W2 b2 W3 b3) and loss.
__global__ void __launch_bounds__(256) k_mlp_grad(const float *P, const float *feat, const float *tgt,
                                                  const float *wgt, const int *idx, int count, float inv_n,
                                                  float *gpart, float *lpart) {
    __shared__ float w1[kPolHid * kPolIn], w2[kPolHid * kPolHid], w3[kPolOut * kPolHid];
    __shared__ float xs[kMlpSamples][kPolIn];
    __shared__ float a1[kMlpSamples][kPolHid], h1[kMlpSamples][kPolHid];
    __shared__ float a2[kMlpSamples][kPolHid], h2[kMlpSamples][kPolHid];
    __shared__ float d2[kMlpSamples][kPolHid], d1[kMlpSamples][kPolHid];
    __shared__ float dout[kMlpSamples][kPolOut];
    __shared__ float lsum[256];
    const int t = threadIdx.x;
    const int base = blockIdx.x * kMlpSamples;
    const int ns = min(kMlpSamples, count - base);
    for (int i = t; i < kPolHid * kPolIn; i += blockDim.x) w1[i] = bf16r(P[kOffW1 + i]);
    for (int i = t; i < kPolHid * kPolHid; i += blockDim.x) w2[i] = bf16r(P[kOffW2 + i]);
    for (int i = t; i < kPolOut * kPolHid; i += blockDim.x) w3[i] = bf16r(P[kOffW3 + i]);
    for (int i = t; i < kMlpSamples * kPolIn; i += blockDim.x) {
        const int s = i / kPolIn, k = i % kPolIn;
        xs[s][k] = s < ns ? bf16r((feat[idx[base + s] * kPolIn + k] - P[kOffMean + k]) / P[kOffStd + k]) : 0.f;
    }
    __syncthreads();
    // layer 1
    for (int i = t; i < kMlpSamples * kPolHid; i += blockDim.x) {
        const int s = i / kPolHid, j = i % kPolHid;
        float a = P[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kPolIn; ++k) a = fmaf(w1[j * kPolIn + k], xs[s][k], a);
        a1[s][j] = a;
        h1[s][j] = bf16r(relu(a));
    }
    __syncthreads();
    // layer 2
    for (int i = t; i < kMlpSamples * kPolHid; i += blockDim.x) {
        const int s = i / kPolHid, j = i % kPolHid;
        float a = P[kOffB2 + j];
        for (int k = 0; k < kPolHid; ++k) a = fmaf(w2[j * kPolHid + k], h1[s][k], a);
        a2[s][j] = a;
        h2[s][j] = bf16r(relu(a));
    }
    __syncthreads();
    // layer 3, loss and its gradient
    float lacc = 0.f;
    for (int i = t; i < kMlpSamples * kPolOut; i += blockDim.x) {
        const int s = i / kPolOut, o = i % kPolOut;
        float g = 0.f;
        if (s < ns) {
            float a = P[kOffB3 + o];
            for (int k = 0; k < kPolHid; ++k) a = fmaf(w3[o * kPolHid + k], h2[s][k], a);
            const int r = idx[base + s];
            const float diff = a - tgt[r * kPolOut + o];
            const float w = wgt[r * kPolOut + o];
            lacc += w * diff * diff;
            g = w * diff * inv_n;
        }
        dout[s][o] = bf16r(g);
    }
    lsum[t] = lacc;
    __syncthreads();
    // back through layer 3 and the second ReLU
    for (int i = t; i < kMlpSamples * kPolHid; i += blockDim.x) {
        const int s = i / kPolHid, j = i % kPolHid;
        float g = 0.f;
#pragma unroll
        for (int o = 0; o < kPolOut; ++o) g = fmaf(w3[o * kPolHid + j], dout[s][o], g);
        d2[s][j] = bf16r(a2[s][j] > 0.f ? g : 0.f);
    }
    __syncthreads();
    // back through layer 2 and the first ReLU
    for (int i = t; i < kMlpSamples * kPolHid; i += blockDim.x) {
        const int s = i / kPolHid, j = i % kPolHid;
        float g = 0.f;
        for (int k = 0; k < kPolHid; ++k) g = fmaf(w2[k * kPolHid + j], d2[s][k], g);
        d1[s][j] = bf16r(a1[s][j] > 0.f ? g : 0.f);
    }
    __syncthreads();
    // parameter gradients of this CTA: sums over its samples in sample order
    float *g = gpart + (size_t)blockIdx.x * kNW;
    for (int i = t; i < kNW; i += blockDim.x) {
        const int p = kOffW1 + i;
        float acc = 0.f;
        if (p < kOffB1) {
            const int j = (p - kOffW1) / kPolIn, k = (p - kOffW1) % kPolIn;
            for (int s = 0; s < ns; ++s) acc = fmaf(d1[s][j], xs[s][k], acc);
        } else if (p < kOffW2) {
            const int j = p - kOffB1;
            for (int s = 0; s < ns; ++s) acc += d1[s][j];
        } else if (p < kOffB2) {
            const int j = (p - kOffW2) / kPolHid, k = (p - kOffW2) % kPolHid;
            for (int s = 0; s < ns; ++s) acc = fmaf(d2[s][j], h1[s][k], acc);
        } else if (p < kOffW3) {
            const int j = p - kOffB2;
            for (int s = 0; s < ns; ++s) acc += d2[s][j];
        } else if (p < kOffB3) {
            const int o = (p - kOffW3) / kPolHid, k = (p - kOffW3) % kPolHid;
            for (int s = 0; s < ns; ++s) acc = fmaf(dout[s][o], h2[s][k], acc);
        } else {
            const int o = p - kOffB3;
            for (int s = 0; s < ns; ++s) acc += dout[s][o];
        }
        g[i] = acc;
    }
    if (t == 0) {
        float l = 0.f;
        for (int i = 0; i < blockDim.x; ++i) l += lsum[i];
        lpart[blockIdx.x] = l;
    }
}

// Sum the CTA partials in CTA order: grad[i] = sum_b gpart[b][i]; loss.
__global__ void k_mlp_sum(const float *gpart, const float *lpart, int nblk, float inv_n, float *grad, float *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNW) {
        float acc = 0.f;
        for (int b = 0; b < nblk; ++b) acc += gpart[(size_t)b * kNW + i];
        grad[i] = acc;
    }
    if (i == 0) {
        float l = 0.f;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = 0.5f * l * inv_n;
    }
}

// Adam (Kingma & Ba) on the FP32 master weights, step t >= 1.
__global__ void k_adam(float *P, const float *grad, float *mom1, float *mom2, int t, float lr, float b1, float b2,
                       float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNW) return;
    const float g = grad[i];
    const float m = b1 * mom1[i] + (1.f - b1) * g;
    const float v = b2 * mom2[i] + (1.f - b2) * g * g;
    mom1[i] = m;
    mom2[i] = v;
    const float mh = m / (1.f - powf(b1, (float)t));
    const float vh = v / (1.f - powf(b2, (float)t));
    P[kOffW1 + i] -= lr * mh / (sqrtf(vh) + eps);
}

struct Dev {
    DevBuf params, feat, tgt, wgt, idx, gpart, lpart, grad, loss, m1, m2, out;
};

void upload(DevBuf &b, const void *src, size_t bytes, cudaStream_t s) {
    b.alloc(bytes);
    GB_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" {

// See include/gbosqp.h.
int gbosqp_policy_forward(const float *params, const float *features, int32_t batch, float *out) {
    if (!params || !features || !out || batch < 0) return GBOSQP_ERR_INVALID_ARG;
    if (batch == 0) return GBOSQP_OK;
    try {
        Dev d;
        upload(d.params, params, sizeof(float) * kPolTotal, 0);
        upload(d.feat, features, sizeof(float) * kPolIn * batch, 0);
        d.out.alloc(sizeof(float) * kPolOut * batch);
        launch(k_policy_forward, batch, 64, (cudaStream_t)0, d.params.as<float>(), d.feat.as<float>(), (int)batch,
               d.out.as<float>());
        GB_CUDA(cudaMemcpy(out, d.out.p, sizeof(float) * kPolOut * batch, cudaMemcpyDeviceToHost));
        return GBOSQP_OK;
    } catch (const GbError &e) {
        return e.code;
    }
}

int gbosqp_mlp_grad(const float *params, const float *features, const float *targets, const float *weights,
                    int32_t n, float *grad, float *loss) {
    if (!params || !features || !targets || !weights || !grad || n <= 0) return GBOSQP_ERR_INVALID_ARG;
    try {
        Dev d;
        upload(d.params, params, sizeof(float) * kPolTotal, 0);
        upload(d.feat, features, sizeof(float) * kPolIn * n, 0);
        upload(d.tgt, targets, sizeof(float) * kPolOut * n, 0);
        upload(d.wgt, weights, sizeof(float) * kPolOut * n, 0);
        std::vector<int> idx(n);
        for (int i = 0; i < n; ++i) idx[i] = i;
        upload(d.idx, idx.data(), sizeof(int) * n, 0);
        const int nblk = ceil_div(n, kMlpSamples);
        d.gpart.alloc(sizeof(float) * (size_t)kNW * nblk);
        d.lpart.alloc(sizeof(float) * nblk);
        d.grad.alloc(sizeof(float) * kNW);
        d.loss.alloc(sizeof(float));
        const float inv_n = 1.0f / (float)n;
        launch(k_mlp_grad, nblk, 256, (cudaStream_t)0, d.params.as<float>(), d.feat.as<float>(), d.tgt.as<float>(),
               d.wgt.as<float>(), d.idx.as<int>(), (int)n, inv_n, d.gpart.as<float>(), d.lpart.as<float>());
        launch(k_mlp_sum, ceil_div(kNW, 256), 256, (cudaStream_t)0, d.gpart.as<float>(), d.lpart.as<float>(), nblk,
               inv_n, d.grad.as<float>(), d.loss.as<float>());
        std::vector<float> g(kNW);
        GB_CUDA(cudaMemcpy(g.data(), d.grad.p, sizeof(float) * kNW, cudaMemcpyDeviceToHost));
        for (int i = 0; i < kPolTotal; ++i) grad[i] = 0.f;
        for (int i = 0; i < kNW; ++i) grad[kOffW1 + i] = g[i];
        if (loss) GB_CUDA(cudaMemcpy(loss, d.loss.p, sizeof(float), cudaMemcpyDeviceToHost));
        return GBOSQP_OK;
    } catch (const GbError &e) {
        return e.code;
    }
}

int gbosqp_mlp_train(float *params, const float *features, const float *targets, const float *weights, int32_t n,
                     const int32_t *batches, int32_t steps, int32_t batch, float lr, float *loss_history) {
    if (!params || !features || !targets || !weights || !batches || n <= 0 || steps < 0 || batch <= 0)
        return GBOSQP_ERR_INVALID_ARG;
    for (long long i = 0; i < (long long)steps * batch; ++i)
        if (batches[i] < 0 || batches[i] >= n) return GBOSQP_ERR_INVALID_ARG;
    try {
        Dev d;
        upload(d.params, params, sizeof(float) * kPolTotal, 0);
        upload(d.feat, features, sizeof(float) * kPolIn * n, 0);
        upload(d.tgt, targets, sizeof(float) * kPolOut * n, 0);
        upload(d.wgt, weights, sizeof(float) * kPolOut * n, 0);
        upload(d.idx, batches, sizeof(int) * (size_t)steps * batch, 0);
        const int nblk = ceil_div(batch, kMlpSamples);
        d.gpart.alloc(sizeof(float) * (size_t)kNW * nblk);
        d.lpart.alloc(sizeof(float) * nblk);
        d.grad.alloc(sizeof(float) * kNW);
        d.loss.alloc(sizeof(float) * std::max(steps, 1));
        d.m1.alloc(sizeof(float) * kNW);
        d.m2.alloc(sizeof(float) * kNW);
        GB_CUDA(cudaMemset(d.m1.p, 0, sizeof(float) * kNW));
        GB_CUDA(cudaMemset(d.m2.p, 0, sizeof(float) * kNW));
        const float inv_n = 1.0f / (float)batch;
        for (int s = 0; s < steps; ++s) {
            launch(k_mlp_grad, nblk, 256, (cudaStream_t)0, d.params.as<float>(), d.feat.as<float>(), d.tgt.as<float>(),
                   d.wgt.as<float>(), d.idx.as<int>() + (size_t)s * batch, (int)batch, inv_n, d.gpart.as<float>(),
                   d.lpart.as<float>());
            launch(k_mlp_sum, ceil_div(kNW, 256), 256, (cudaStream_t)0, d.gpart.as<float>(), d.lpart.as<float>(), nblk,
                   inv_n, d.grad.as<float>(), d.loss.as<float>() + s);
            launch(k_adam, ceil_div(kNW, 256), 256, (cudaStream_t)0, d.params.as<float>(), d.grad.as<float>(),
                   d.m1.as<float>(), d.m2.as<float>(), s + 1, lr, 0.9f, 0.999f, 1e-8f);
        }
        GB_CUDA(cudaMemcpy(params, d.params.p, sizeof(float) * kPolTotal, cudaMemcpyDeviceToHost));
        if (loss_history && steps > 0)
            GB_CUDA(cudaMemcpy(loss_history, d.loss.p, sizeof(float) * steps, cudaMemcpyDeviceToHost));
        return GBOSQP_OK;
    } catch (const GbError &e) {
        return e.code;
    }
}

}  // extern "C"

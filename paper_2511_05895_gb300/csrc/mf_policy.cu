// Training and inference kernels of the policy network (mf_mlp.cuh) and
// their C ABI (mf_mlp_* in mf.h).  The network chooses, per update batch,
// between the dynamic repair and a static recompute, and the KERNELCYCLES
// value (the paper finds a crossover batch size past which static wins,
// Sec. 6.5, and a trade-off in KERNELCYCLES, Note 2 of Sec. 3).
//
// One training step on a mini-batch of B samples is three kernels:
//   k_mlp_fwd_bwd  one thread per sample: forward pass, loss, and the
//                  error signals of every layer, into the workspace;
//   k_mlp_grad     one thread per parameter: the gradient as a sum over the
//                  samples in a fixed order (deterministic, no atomics);
//   k_mlp_adam     one thread per parameter: the Adam update.
// Loss per sample: BCE(y0, t0) + wkc * (y1 - t1)^2 / 2 + wmode * CE(softmax
// of y2..y4, class t2), averaged over the mini-batch (t2 is the index of the
// fastest processing mode, stored as a float).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "mf.h"
#include "mf_mlp.cuh"

namespace mf {
namespace mlp {

// Workspace row of one sample: z, h1, h2, d1, d2 (error signals of the
// hidden layers, after the ReLU mask), dy (output error), loss.
constexpr int rZ = 0, rH1 = rZ + kIn, rH2 = rH1 + kH1, rD1 = rH2 + kH2, rD2 = rD1 + kH1, rDY = rD2 + kH2,
              rLoss = rDY + kOut, kRow = rLoss + 1;

__device__ __forceinline__ float softplus(float y) { return fmaxf(y, 0.f) + log1pf(expf(-fabsf(y))); }
__device__ __forceinline__ float sigmoid(float y) { return 1.f / (1.f + expf(-y)); }

__global__ void k_mlp_fwd_bwd(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ T0,
                              const float *__restrict__ T1, const float *__restrict__ T2, int n, int base, int B,
                              float wkc, float wmode, float *__restrict__ W) {
    __shared__ float sP[kTotal];
    for (int i = threadIdx.x; i < kTotal; i += blockDim.x) sP[i] = P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const int idx = (base + s) % n;
    float *row = W + (size_t)s * kRow;
    float x[kIn], z[kIn], h1[kH1], h2[kH2], y[kOut];
    for (int j = 0; j < kIn; ++j) x[j] = X[(size_t)idx * kIn + j];
    forward(sP, x, z, h1, h2, y);
    const float t0 = T0[idx], t1 = T1[idx];
    const int t2 = (int)T2[idx];
    const float inv = 1.f / (float)B;
    float dy[kOut];
    dy[0] = (sigmoid(y[0]) - t0) * inv;
    dy[1] = wkc * (y[1] - t1) * inv;
    // softmax cross-entropy of the mode logits (shifted by their maximum)
    float mx = y[2];
    for (int c = 1; c < kModes; ++c) mx = fmaxf(mx, y[2 + c]);
    float se = 0.f;
    for (int c = 0; c < kModes; ++c) se += expf(y[2 + c] - mx);
    for (int c = 0; c < kModes; ++c) dy[2 + c] = wmode * (expf(y[2 + c] - mx) / se - (c == t2 ? 1.f : 0.f)) * inv;
    const float ce = mx + logf(se) - y[2 + t2];
    float d2[kH2];
    for (int j = 0; j < kH2; ++j) {
        float a = 0.f;
        for (int o = 0; o < kOut; ++o) a += sP[oW3 + o * kH2 + j] * dy[o];
        d2[j] = h2[j] > 0.f ? a : 0.f;
    }
    for (int j = 0; j < kH1; ++j) {
        float a = 0.f;
        for (int i = 0; i < kH2; ++i) a += sP[oW2 + i * kH1 + j] * d2[i];
        row[rD1 + j] = h1[j] > 0.f ? a : 0.f;
    }
    for (int j = 0; j < kIn; ++j) row[rZ + j] = z[j];
    for (int j = 0; j < kH1; ++j) row[rH1 + j] = h1[j];
    for (int j = 0; j < kH2; ++j) {
        row[rH2 + j] = h2[j];
        row[rD2 + j] = d2[j];
    }
    for (int o = 0; o < kOut; ++o) row[rDY + o] = dy[o];
    const float d = y[1] - t1;
    row[rLoss] = (softplus(y[0]) - t0 * y[0] + 0.5f * wkc * d * d + wmode * ce) * inv;
}

// Gradient of the mini-batch loss: parameter p is one weight or bias.
__global__ void k_mlp_grad(const float *__restrict__ W, int B, float *__restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    int dcol, acol = -1;   // error-signal column and activation column (-1: bias)
    if (p < oB1) {
        dcol = rD1 + (p - oW1) / kIn;
        acol = rZ + (p - oW1) % kIn;
    } else if (p < oW2) {
        dcol = rD1 + (p - oB1);
    } else if (p < oB2) {
        dcol = rD2 + (p - oW2) / kH1;
        acol = rH1 + (p - oW2) % kH1;
    } else if (p < oW3) {
        dcol = rD2 + (p - oB2);
    } else if (p < oB3) {
        dcol = rDY + (p - oW3) / kH2;
        acol = rH2 + (p - oW3) % kH2;
    } else {
        dcol = rDY + (p - oB3);
    }
    float g = 0.f;
    for (int s = 0; s < B; ++s) {
        const float *row = W + (size_t)s * kRow;
        g += row[dcol] * (acol >= 0 ? row[acol] : 1.f);
    }
    G[p] = g;
}

__global__ void k_mlp_loss(const float *__restrict__ W, int B, float *__restrict__ out) {
    __shared__ float red[256];
    float a = 0.f;
    for (int s = threadIdx.x; s < B; s += blockDim.x) a += W[(size_t)s * kRow + rLoss];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                           float *__restrict__ V, float lr, float b1t, float b2t) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = G[p];
    const float m = b1 * M[p] + (1.f - b1) * g;
    const float v = b2 * V[p] + (1.f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    const float mh = m / (1.f - b1t), vh = v / (1.f - b2t);
    P[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_mlp_forward(const float *__restrict__ P, const float *__restrict__ X, int n, float *__restrict__ Y) {
    __shared__ float sP[kTotal];
    for (int i = threadIdx.x; i < kTotal; i += blockDim.x) sP[i] = P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kIn], z[kIn], h1[kH1], h2[kH2], y[kOut];
    for (int j = 0; j < kIn; ++j) x[j] = X[(size_t)s * kIn + j];
    forward(sP, x, z, h1, h2, y);
    for (int o = 0; o < kOut; ++o) Y[(size_t)s * kOut + o] = y[o];
}

size_t workspace_bytes(int B) { return (size_t)B * kRow * sizeof(float) + (size_t)kParams * sizeof(float) + 256; }

}  // namespace mlp
}  // namespace mf

using namespace mf::mlp;

namespace {
int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return MF_OK;
    cudaGetLastError();
    return MF_ECUDA;
}
}  // namespace

extern "C" {

int mf_mlp_sizes(int32_t *n_in, int32_t *n_out, int32_t *n_trained, int32_t *n_total) {
    if (n_in) *n_in = kIn;
    if (n_out) *n_out = kOut;
    if (n_trained) *n_trained = kParams;
    if (n_total) *n_total = kTotal;
    return MF_OK;
}

int64_t mf_mlp_workspace_bytes(int32_t batch) { return batch > 0 ? (int64_t)workspace_bytes(batch) : -1; }

int mf_mlp_forward(const float *P, const float *X, int32_t n, float *Y, void *stream) {
    if (!P || (n > 0 && (!X || !Y)) || n < 0) return MF_EINVAL;
    if (n == 0) return MF_OK;
    k_mlp_forward<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(P, X, n, Y);
    return cuda_rc(cudaGetLastError());
}

int mf_mlp_grad(const float *P, const float *X, const float *T0, const float *T1, const float *T2, int32_t n,
                float wkc, float wmode, float *grad, float *loss, void *workspace, void *stream) {
    if (!P || !X || !T0 || !T1 || !T2 || !grad || !loss || !workspace || n <= 0) return MF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *W = static_cast<float *>(workspace);
    k_mlp_fwd_bwd<<<(n + 127) / 128, 128, 0, st>>>(P, X, T0, T1, T2, n, 0, n, wkc, wmode, W);
    k_mlp_grad<<<(kParams + 255) / 256, 256, 0, st>>>(W, n, grad);
    k_mlp_loss<<<1, 256, 0, st>>>(W, n, loss);
    return cuda_rc(cudaGetLastError());
}

int mf_mlp_train(float *P, float *M, float *V, const float *X, const float *T0, const float *T1, const float *T2,
                 int32_t n, int32_t steps, int32_t batch, float lr, float wkc, float wmode, int32_t step0,
                 float *loss_hist, void *workspace, void *stream) {
    if (!P || !M || !V || !X || !T0 || !T1 || !T2 || !workspace || n <= 0 || steps < 0 || batch <= 0 || step0 < 0)
        return MF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *W = static_cast<float *>(workspace);
    float *G = W + (size_t)batch * kRow;
    const int B = batch < n ? batch : n;
    for (int s = 0; s < steps; ++s) {
        const int base = (int)(((long long)(step0 + s) * B) % n);
        k_mlp_fwd_bwd<<<(B + 127) / 128, 128, 0, st>>>(P, X, T0, T1, T2, n, base, B, wkc, wmode, W);
        k_mlp_grad<<<(kParams + 255) / 256, 256, 0, st>>>(W, B, G);
        if (loss_hist) k_mlp_loss<<<1, 256, 0, st>>>(W, B, loss_hist + s);
        const double t = (double)(step0 + s + 1);
        k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(P, G, M, V, lr, (float)pow(0.9, t), (float)pow(0.999, t));
    }
    return cuda_rc(cudaGetLastError());
}

}  // extern "C"

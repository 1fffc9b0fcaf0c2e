// The policy network: a 12 -> 64 -> 64 -> 5 fully connected ReLU MLP in
// FP32 (used by mf_gpu.cu for decisions and by mf_policy.cu for training).
//
// Parameter array layout (floats, row-major weights out x in):
//   W1 [64 x 12], b1 [64], W2 [64 x 64], b2 [64], W3 [5 x 64], b3 [5]
//   then the input normalisation mu [12], sd [12] (not trained).
// The network sees z = (x - mu) / sd.  Output 0 is the logit that the
// dynamic repair beats a static recompute; output 1 is log2 of the
// KERNELCYCLES value to use; outputs 2, 3, 4 are the logits (softmax) of the
// processing mode of the repair: data-driven (Sec. 5.3), topology-driven
// (Sec. 5.2), Dynamic Push-Pull (Alg. 8).
#pragma once

namespace mf {
namespace mlp {

constexpr int kIn = 12, kH1 = 64, kH2 = 64, kOut = 5;
constexpr int kModes = 3;   // outputs 2 .. 4
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kH1 * kIn;
constexpr int oW2 = oB1 + kH1;
constexpr int oB2 = oW2 + kH2 * kH1;
constexpr int oW3 = oB2 + kH2;
constexpr int oB3 = oW3 + kOut * kH2;
constexpr int kParams = oB3 + kOut;      // 5317 trained parameters
constexpr int oMu = kParams;
constexpr int oSd = oMu + kIn;
constexpr int kTotal = oSd + kIn;        // 5341 floats in all

// Forward pass of one sample; x is the raw feature vector.  Writes the
// normalised input z, both hidden layers (after ReLU) and the outputs.
__host__ __device__ inline void forward(const float *P, const float *x, float *z, float *h1, float *h2, float *y) {
    for (int j = 0; j < kIn; ++j) z[j] = (x[j] - P[oMu + j]) / P[oSd + j];
    for (int i = 0; i < kH1; ++i) {
        float a = P[oB1 + i];
        for (int j = 0; j < kIn; ++j) a += P[oW1 + i * kIn + j] * z[j];
        h1[i] = a > 0.f ? a : 0.f;
    }
    for (int i = 0; i < kH2; ++i) {
        float a = P[oB2 + i];
        for (int j = 0; j < kH1; ++j) a += P[oW2 + i * kH1 + j] * h1[j];
        h2[i] = a > 0.f ? a : 0.f;
    }
    for (int o = 0; o < kOut; ++o) {
        float a = P[oB3 + o];
        for (int j = 0; j < kH2; ++j) a += P[oW3 + o * kH2 + j] * h2[j];
        y[o] = a;
    }
}

}  // namespace mlp
}  // namespace mf

// Layout of the learned skip's classifier (F -> 64 -> 64 -> 1, ReLU, FP16 weights, FP32
// accumulation) and the inference used by the factorization kernel and the forward entry
// point.  The model array (FP32) holds mean[F] std[F] W1[64][F] b1[64] W2[64][64] b2[64]
// w3[64] b3; on the device the normalisation stays FP32 and the weights are FP16.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "bilu.h"

constexpr int MF = BILU_MLP_FEATURES;
constexpr int MH = BILU_MLP_HIDDEN;
constexpr int MO_MEAN = 0, MO_STD = MF, MO_W1 = 2 * MF, MO_B1 = MO_W1 + MH * MF, MO_W2 = MO_B1 + MH,
              MO_B2 = MO_W2 + MH * MH, MO_W3 = MO_B2 + MH, MO_B3 = MO_W3 + MH, MO_N = MO_B3 + 1;
static_assert(MO_N == BILU_MLP_PARAMS, "model layout");
constexpr int MW = MO_N - 2 * MF;  // weights and biases (FP16 on the device), offset 2F

// counter-based 64-bit hash (splitmix64 finaliser): weight initialisation, sample draws and
// the recording's sampling decisions
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// weight / bias at model index i (>= 2F) from the FP16 device copy
__device__ __forceinline__ float mlp_w(const __half *w, int i) { return __half2float(w[i - 2 * MF]); }

// standardised feature: (x - mean) / std
__device__ __forceinline__ float mlp_std(const float *norm, int k, float x) {
    return (x - norm[MO_MEAN + k]) / norm[MO_STD + k];
}

// Logit of one standardised feature vector, every sum in increasing index order:
//   h1[u] = relu(b1[u] + sum_k W1[u][k] x[k]),  h2[u] = relu(b2[u] + sum_k W2[u][k] h1[k]),
//   z = b3 + sum_u w3[u] h2[u].
__device__ __forceinline__ float mlp_logit_seq(const float *xs, const __half *w) {
    float h1[MH];
#pragma unroll 4
    for (int u = 0; u < MH; ++u) {
        float acc = mlp_w(w, MO_B1 + u);
        for (int k = 0; k < MF; ++k) acc = fmaf(mlp_w(w, MO_W1 + u * MF + k), xs[k], acc);
        h1[u] = fmaxf(acc, 0.f);
    }
    float z = mlp_w(w, MO_B3);
    for (int u = 0; u < MH; ++u) {
        float acc = mlp_w(w, MO_B2 + u);
#pragma unroll
        for (int k = 0; k < MH; ++k) acc = fmaf(mlp_w(w, MO_W2 + u * MH + k), h1[k], acc);
        z = fmaf(mlp_w(w, MO_W3 + u), fmaxf(acc, 0.f), z);
    }
    return z;
}

// lp_mlp.cuh -- constants and the device-side evaluation of the learned state
// estimator (8 -> 32 ReLU -> 1 sigmoid, BF16 weights, FP32 accumulation), and
// the eight stencil features it reads.
#pragma once

#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {

constexpr int MLP_IN = 8;
constexpr int MLP_H = 32;
constexpr int OFF_B1 = MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H;
constexpr int MLP_NPARAM = OFF_B2 + 1;

// logit of the network for features x
__device__ inline float mlp_logit(const float (&x)[MLP_IN], const __nv_bfloat16* __restrict__ w)
{
    float z = __bfloat162float(w[OFF_B2]);
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float a = __bfloat162float(w[OFF_B1 + j]);
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) a = fmaf(__bfloat162float(w[j * MLP_IN + k]), x[k], a);
        z = fmaf(__bfloat162float(w[OFF_W2 + j]), a > 0.0f ? a : 0.0f, z);
    }
    return z;
}

__device__ inline float mlp_prob(const float (&x)[MLP_IN], const __nv_bfloat16* __restrict__ w)
{
    return 1.0f / (1.0f + __expf(-mlp_logit(x, w)));
}

// feature transform: log(1 + 10 |f|), with the sign kept for the divergence term
__device__ inline float feat_t(float f) { return log1pf(10.0f * fabsf(f)); }
__device__ inline float feat_ts(float f) { return copysignf(log1pf(10.0f * fabsf(f)), f); }

}  // namespace lp

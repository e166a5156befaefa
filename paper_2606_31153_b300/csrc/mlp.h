// Internal view of the learned stopping predictor (see mlp.cu).
#pragma once
#include <cuda_bf16.h>

#include "internal.h"

namespace gkb {

constexpr int kIn = 64, kHid = 256, kOut = 2;
constexpr int kParams = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;
// offsets of the flat parameter vector: W1 (256x64), b1, W2 (256x256), b2, W3 (2x256), b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
// normalisation block: feature means (64), feature deviations (64), target means (2), target deviations (2)
constexpr int kNorm = 2 * kIn + 2 * kOut;

}  // namespace gkb

struct gkb_mlp {
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // FP32 master copy and Adam state
  __nv_bfloat16 *theta_bf16 = nullptr;                                   // inference copy
  float *norm = nullptr;                                                 // device normalisation block
  float *work = nullptr;                                                 // activations of a training batch
  int work_batch = 0;
  int step = 0;
};

namespace gkb {

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// One sample through the network with BF16 weights and BF16-rounded
// activations, FP32 accumulation.  Call from all 256 threads of a block;
// feat (64 raw features) and the scratch arrays are in shared memory; the
// de-standardised outputs land in out[0..1] (valid after the call).
__device__ __forceinline__ void mlp_infer_block(const __nv_bfloat16 *__restrict__ theta, const float *__restrict__ norm,
                                                const float *feat, float *h1, float *h2, float *out) {
  const int t = threadIdx.x;
  if (t < kIn) h2[t] = __bfloat162float(__float2bfloat16_rn((feat[t] - norm[t]) / norm[kIn + t]));
  __syncthreads();
  {
    float acc = __bfloat162float(theta[kOffB1 + t]);
    const __nv_bfloat16 *w = theta + kOffW1 + t * kIn;
    for (int i = 0; i < kIn; ++i) acc = fmaf(__bfloat162float(w[i]), h2[i], acc);
    h1[t] = __bfloat162float(__float2bfloat16_rn(gelu_f(acc)));
  }
  __syncthreads();
  {
    float acc = __bfloat162float(theta[kOffB2 + t]);
    const __nv_bfloat16 *w = theta + kOffW2 + t * kHid;
    for (int i = 0; i < kHid; ++i) acc = fmaf(__bfloat162float(w[i]), h1[i], acc);
    h2[t] = __bfloat162float(__float2bfloat16_rn(gelu_f(acc)));
  }
  __syncthreads();
  if (t < 32) {
    for (int o = 0; o < kOut; ++o) {
      float acc = 0.f;
      for (int i = t; i < kHid; i += 32) acc = fmaf(__bfloat162float(theta[kOffW3 + o * kHid + i]), h2[i], acc);
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sh);
      if (t == 0) {
        const float y = acc + __bfloat162float(theta[kOffB3 + o]);
        out[o] = y * norm[2 * kIn + kOut + o] + norm[2 * kIn + o];
      }
    }
  }
  __syncthreads();
}

}  // namespace gkb

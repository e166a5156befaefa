// The learned stopping predictor: a 64 -> 256 -> 256 -> 2 perceptron with
// exact GELU, trained in FP32 on the device (forward, backward, Adam) and
// evaluated with BF16 weights.  All reductions run in a fixed order, so a
// training step is deterministic.
#include <cmath>
#include <new>

#include "mlp.h"

namespace gkb {
namespace {

constexpr int TS = 16;  // GEMM tile

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[n]); act 1 stores gelu(.) in C and
// the pre-activation in Z.  op(A)(m,k) = ta ? A[k*lda+m] : A[m*lda+k], op(B)(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n].
__global__ void __launch_bounds__(TS *TS) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda, int ta,
                                                 const float *__restrict__ B, int ldb, int tb, const float *__restrict__ bias,
                                                 float *__restrict__ C, int ldc, int act, float *__restrict__ Z) {
  __shared__ float As[TS][TS + 1], Bs[TS][TS + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m = blockIdx.y * TS + ty, n = blockIdx.x * TS + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += TS) {
    const int ka = k0 + tx, kb = k0 + ty;
    const int am = blockIdx.y * TS + ty, bn = blockIdx.x * TS + tx;
    As[ty][tx] = (am < M && ka < K) ? (ta ? A[(long long)ka * lda + am] : A[(long long)am * lda + ka]) : 0.f;
    Bs[ty][tx] = (kb < K && bn < N) ? (tb ? B[(long long)bn * ldb + kb] : B[(long long)kb * ldb + bn]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TS; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (m < M && n < N) {
    if (bias) acc += bias[n];
    if (act) {
      Z[(long long)m * ldc + n] = acc;
      acc = gelu_f(acc);
    }
    C[(long long)m * ldc + n] = acc;
  }
}

// out[n] = sum over rows of A[m*N + n] (fixed row order)
__global__ void k_colsum(int M, int N, const float *__restrict__ A, float *__restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int m = 0; m < M; ++m) acc += A[(long long)m * N + n];
  out[n] = acc;
}

// dY = (Y - T) / B and the loss 0.5 * sum (Y - T)^2 / B (one block, fixed order)
__global__ void k_output_grad(int Bn, const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY,
                              float *loss) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < Bn * kOut; i += blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d / (float)Bn;
    acc += 0.5 * (double)d * d;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0 && loss) *loss = (float)(acc / Bn);
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(long long n, const float *__restrict__ dH, const float *__restrict__ Z, float *__restrict__ dZ) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dH[i] * gelu_grad_f(Z[i]);
}

__global__ void k_adam(int n, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void k_to_bf16(int n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// Batched inference with BF16 weights on raw features (standardised inside).
__global__ void __launch_bounds__(kHid) k_infer_bf16(const __nv_bfloat16 *__restrict__ theta, const float *__restrict__ norm,
                                                     const float *__restrict__ X, float *__restrict__ Y) {
  __shared__ float feat[kIn], h1[kHid], h2[kHid], out[kOut];
  if (threadIdx.x < kIn) feat[threadIdx.x] = X[(long long)blockIdx.x * kIn + threadIdx.x];
  __syncthreads();
  mlp_infer_block(theta, norm, feat, h1, h2, out);
  if (threadIdx.x < kOut) Y[(long long)blockIdx.x * kOut + threadIdx.x] = out[threadIdx.x];
}

dim3 gemm_grid(int M, int N) { return dim3((N + TS - 1) / TS, (M + TS - 1) / TS); }

// work layout for batch B: Z1, H1, Z2, H2 (B x 256 each), Y, dY (B x 2), dH (B x 256), dZ (B x 256)
struct Work {
  float *Z1, *H1, *Z2, *H2, *Y, *dY, *dH, *dZ;
};
Work work_of(gkb_mlp *N, int B) {
  float *w = N->work;
  Work W;
  W.Z1 = w; W.H1 = w + (size_t)B * kHid; W.Z2 = w + 2 * (size_t)B * kHid; W.H2 = w + 3 * (size_t)B * kHid;
  W.dH = w + 4 * (size_t)B * kHid; W.dZ = w + 5 * (size_t)B * kHid;
  W.Y = w + 6 * (size_t)B * kHid; W.dY = W.Y + (size_t)B * kOut;
  return W;
}

gkb_status ensure_work(gkb_mlp *N, int B) {
  if (B <= N->work_batch) return GKB_OK;
  if (N->work) cudaFree(N->work);
  N->work = nullptr;
  N->work_batch = 0;
  GKB_CUDA_TRY(cudaMalloc(&N->work, sizeof(float) * ((size_t)6 * B * kHid + 2 * (size_t)B * kOut)));
  N->work_batch = B;
  return GKB_OK;
}

void forward_fp32(gkb_mlp *N, const float *X, int B, const Work &W, cudaStream_t s) {
  const float *th = N->theta;
  const dim3 tb(TS, TS);
  k_gemm<<<gemm_grid(B, kHid), tb, 0, s>>>(B, kHid, kIn, X, kIn, 0, th + kOffW1, kIn, 1, th + kOffB1, W.H1, kHid, 1, W.Z1);
  k_gemm<<<gemm_grid(B, kHid), tb, 0, s>>>(B, kHid, kHid, W.H1, kHid, 0, th + kOffW2, kHid, 1, th + kOffB2, W.H2, kHid, 1, W.Z2);
  k_gemm<<<gemm_grid(B, kOut), tb, 0, s>>>(B, kOut, kHid, W.H2, kHid, 0, th + kOffW3, kHid, 1, th + kOffB3, W.Y, kOut, 0, nullptr);
}

void backward_fp32(gkb_mlp *N, const float *X, const float *T, int B, const Work &W, float *g, float *loss, cudaStream_t s) {
  const float *th = N->theta;
  const dim3 tb(TS, TS);
  k_output_grad<<<1, 256, 0, s>>>(B, W.Y, T, W.dY, loss);
  // layer 3
  k_gemm<<<gemm_grid(kOut, kHid), tb, 0, s>>>(kOut, kHid, B, W.dY, kOut, 1, W.H2, kHid, 0, nullptr, g + kOffW3, kHid, 0, nullptr);
  k_colsum<<<1, 32, 0, s>>>(B, kOut, W.dY, g + kOffB3);
  k_gemm<<<gemm_grid(B, kHid), tb, 0, s>>>(B, kHid, kOut, W.dY, kOut, 0, th + kOffW3, kHid, 0, nullptr, W.dH, kHid, 0, nullptr);
  k_gelu_back<<<(B * kHid + 255) / 256, 256, 0, s>>>((long long)B * kHid, W.dH, W.Z2, W.dZ);
  // layer 2
  k_gemm<<<gemm_grid(kHid, kHid), tb, 0, s>>>(kHid, kHid, B, W.dZ, kHid, 1, W.H1, kHid, 0, nullptr, g + kOffW2, kHid, 0, nullptr);
  k_colsum<<<1, kHid, 0, s>>>(B, kHid, W.dZ, g + kOffB2);
  k_gemm<<<gemm_grid(B, kHid), tb, 0, s>>>(B, kHid, kHid, W.dZ, kHid, 0, th + kOffW2, kHid, 0, nullptr, W.dH, kHid, 0, nullptr);
  k_gelu_back<<<(B * kHid + 255) / 256, 256, 0, s>>>((long long)B * kHid, W.dH, W.Z1, W.dZ);
  // layer 1
  k_gemm<<<gemm_grid(kHid, kIn), tb, 0, s>>>(kHid, kIn, B, W.dZ, kHid, 1, X, kIn, 0, nullptr, g + kOffW1, kIn, 0, nullptr);
  k_colsum<<<1, kHid, 0, s>>>(B, kHid, W.dZ, g + kOffB1);
}

}  // namespace
}  // namespace gkb

using namespace gkb;

extern "C" gkb_status gkb_mlp_destroy(gkb_mlp *N) {
  if (!N) return GKB_ERR_INVALID_ARG;
  cudaFree(N->theta); cudaFree(N->m); cudaFree(N->v); cudaFree(N->grad);
  cudaFree(N->theta_bf16); cudaFree(N->norm);
  if (N->work) cudaFree(N->work);
  delete N;
  return GKB_OK;
}

extern "C" gkb_status gkb_mlp_create(gkb_mlp **out) {
  if (!out) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  gkb_mlp *N = new (std::nothrow) gkb_mlp();
  if (!N) return GKB_ERR_OOM;
  cudaError_t e = cudaSuccess;
  for (float **p : {&N->theta, &N->m, &N->v, &N->grad})
    if (e == cudaSuccess) e = cudaMalloc(p, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&N->theta_bf16, sizeof(__nv_bfloat16) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&N->norm, sizeof(float) * kNorm);
  if (e == cudaSuccess) e = cudaMemset(N->theta, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(N->m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(N->v, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(N->theta_bf16, 0, sizeof(__nv_bfloat16) * kParams);
  if (e == cudaSuccess) {
    float norm[kNorm];
    for (int i = 0; i < kNorm; ++i) norm[i] = (i < kIn || (i >= 2 * kIn && i < 2 * kIn + kOut)) ? 0.f : 1.f;
    e = cudaMemcpy(N->norm, norm, sizeof(norm), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    gkb_mlp_destroy(N);
    return e == cudaErrorMemoryAllocation ? GKB_ERR_OOM : GKB_ERR_CUDA;
  }
  *out = N;
  return GKB_OK;
}

extern "C" int gkb_mlp_num_params(void) { return kParams; }

extern "C" gkb_status gkb_mlp_set_params(gkb_mlp *N, const float *theta, const float *norm) {
  if (!N) return GKB_ERR_INVALID_ARG;
  if (theta) {
    GKB_CUDA_TRY(cudaMemcpy(N->theta, theta, sizeof(float) * kParams, cudaMemcpyDefault));
    GKB_CUDA_TRY(cudaMemset(N->m, 0, sizeof(float) * kParams));
    GKB_CUDA_TRY(cudaMemset(N->v, 0, sizeof(float) * kParams));
    N->step = 0;
    k_to_bf16<<<(kParams + 255) / 256, 256>>>(kParams, N->theta, N->theta_bf16);
    GKB_CUDA_TRY(cudaGetLastError());
  }
  if (norm) GKB_CUDA_TRY(cudaMemcpy(N->norm, norm, sizeof(float) * kNorm, cudaMemcpyDefault));
  GKB_CUDA_TRY(cudaDeviceSynchronize());
  return GKB_OK;
}

extern "C" gkb_status gkb_mlp_get_params(const gkb_mlp *N, float *theta, float *norm) {
  if (!N) return GKB_ERR_INVALID_ARG;
  if (theta) GKB_CUDA_TRY(cudaMemcpy(theta, N->theta, sizeof(float) * kParams, cudaMemcpyDefault));
  if (norm) GKB_CUDA_TRY(cudaMemcpy(norm, N->norm, sizeof(float) * kNorm, cudaMemcpyDefault));
  return GKB_OK;
}

extern "C" gkb_status gkb_mlp_forward(gkb_mlp *N, const float *X, int B, float *Y, int bf16, void *stream) {
  if (!N || !X || !Y || B < 1) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (bf16) {
    k_infer_bf16<<<B, kHid, 0, s>>>(N->theta_bf16, N->norm, X, Y);
  } else {
    gkb_status st = ensure_work(N, B);
    if (st != GKB_OK) return st;
    Work W = work_of(N, B);
    forward_fp32(N, X, B, W, s);
    GKB_CUDA_TRY(cudaMemcpyAsync(Y, W.Y, sizeof(float) * B * kOut, cudaMemcpyDeviceToDevice, s));
  }
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

extern "C" gkb_status gkb_mlp_gradient(gkb_mlp *N, const float *X, const float *T, int B, float *grad, float *loss,
                                       void *stream) {
  if (!N || !X || !T || B < 1) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gkb_status st = ensure_work(N, B);
  if (st != GKB_OK) return st;
  Work W = work_of(N, B);
  forward_fp32(N, X, B, W, s);
  backward_fp32(N, X, T, B, W, grad ? grad : N->grad, loss, s);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

extern "C" gkb_status gkb_mlp_train_step(gkb_mlp *N, const float *X, const float *T, int B, float lr, float *loss,
                                         void *stream) {
  gkb_status st = gkb_mlp_gradient(N, X, T, B, nullptr, loss, stream);
  if (st != GKB_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  N->step += 1;
  const float c1 = 1.0f - powf(0.9f, (float)N->step), c2 = 1.0f - powf(0.999f, (float)N->step);
  k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(kParams, N->theta, N->m, N->v, N->grad, lr, c1, c2);
  k_to_bf16<<<(kParams + 255) / 256, 256, 0, s>>>(kParams, N->theta, N->theta_bf16);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

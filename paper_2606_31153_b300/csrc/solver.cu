// AB-GKB (Algorithm 4), BA-GKB (Algorithm 5) and matched GKB (Algorithm 3) on
// the device.
//
// One iteration j (reading of the printed loop: iteration j produces s_{j+1},
// t_{j+1}, q_{j+1}, alpha_{j+1}; C_j has alpha_1..alpha_j on its diagonal and
// t_2..t_{j+1} below it):
//   s~ = M q_j - alpha_j s_j                    (two projector launches, the
//                                                second with a fused axpy and
//                                                a fused sum of squares)
//   t_{j+1} = ||s~||, s_{j+1} = s~/t_{j+1}
//   q~ = M^T s_{j+1} - t_{j+1} q_j               (two launches, fused axpy)
//   q~ -= sum_{i<=j} (q_i^T q~) q_i              (the one-sided
//                                                reorthogonalisation: classical
//                                                Gram-Schmidt pass(es))
//   alpha_{j+1} = ||q~||, q_{j+1} = q~/alpha_{j+1}
//   projected problem: the least-squares solution u_j of min ||C_j u - t_1 e_1||
//            (Eq. proj GKB) and x_j = Q_j u_j (BA, matched) or B Q_j u_j (AB).
//            C_j grows by one column per iteration, so the minimiser is
//            carried by the Givens QR of C_j (the recurrences of Paige and
//            Saunders' LSQR): rho_j, c_j, s_j, phi_j, phibar_{j+1} in FP64 and
//            x_j = x_{j-1} + (phi_j/rho_j) w_j with w_{j+1} = q_{j+1} - (theta_{j+1}/rho_j) w_j.
//            This is the same u_j the SVD of C_j gives (C_j has full column
//            rank until breakdown), in O(1) scalar work per step.
//   stopping: the data residual of Eq. (DP): A x_j - b is carried as an
//            m-vector r_j = r_{j-1} + (phi_j/rho_j) z_j where z_j = A w_j (BA,
//            matched) or M w_j (AB) follows the w recurrence applied to the
//            vector A q_j (resp. M q_j) the first projector pair already computes.  The stop
//            decision (DP, RNS, breakdown, k_max) is taken on the device and
//            every later kernel returns at once.
//
// The loop is a CUDA-graph WHILE node whose body is one iteration; a
// one-thread kernel at its end advances the iteration counter and clears the
// loop condition once the solve has stopped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "mlp.h"
#include "fast.h"

namespace gkb {
namespace {

constexpr int kVT = 256;          // vector-kernel block
constexpr int kLearnK0 = 16;      // iterations observed before the predictor runs
constexpr int kLearnDelta = 8;    // extra iterations beyond the predicted discrepancy index
constexpr int kRowsPerBlock = 1024;  // reorth dots: 256 threads x 4 rows
constexpr int kDotCols = 16;         // reorth dots: columns per block (second grid dimension)
constexpr int kUT = 128;             // reorth update block (4 rows per thread)

struct Ctl {
  double alpha_cur, t_cur, cz_cur;   // alpha_j, t_{j+1}, theta_j/rho_{j-1}
  double tsq_cur, asq_cur, rsq_cur;  // sums of squares produced by grid reductions
  double tau_e, rns_eps, scale0;
  double bsq, bscale, inv_bscale;    // FP16 storage solves b/||b||: x, t_1 and residuals are scaled back
  int done, k_stop, reason, status, iter, stop, kmax, bd;
  // learned stopping (BA, FP32): phase 1 runs kLearnK0 complete iterations,
  // the predictor sets kmax and lambda, phase 3 resumes; the first iteration
  // meeting the discrepancy principle is remembered (k_dp, x_dp)
  int learned, phase, k_dp, dp_now, stop_after, complete_last, kmax_user, fallback, hybrid, k_hat;
  double lambda, hyb_r2;
};

struct SK {
  Ctl *c;
  double *alpha, *t, *rho, *rhobar, *phibar, *cg, *sg, *resid;  // indexed by iteration
  double *partials;
  unsigned *counters;
  double *dotp, *coef;
  double *R, *hcol;   // GMRES: triangular factor of H_k (ldk x ldk, column-major), the current column of H_k
  double *lam;        // hybrid regularisation: lambda_k by iteration
  double *hyb;        // hybrid regularisation: tridiagonal scratch of 32 candidate lambdas (64 x ldk)
  int ldk;  // kmax + 2
};

template <typename T, typename C> struct V4 { C v[4]; };

template <typename T, typename C>
__device__ __forceinline__ void load4(const T *p, C (&o)[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) o[u] = to_c(p[u]);
}
template <>
__device__ __forceinline__ void load4<float, float>(const float *p, float (&o)[4]) {
  float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double, double>(const double *p, double (&o)[4]) {
  double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

__device__ __forceinline__ bool first_thread() {
  return blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0;
}

// ---------------------------------------------------------------------------
// initialisation (t_1, s_1, alpha_1, q_1)

__global__ void k_reset(SK S, int kmax, int stop, double tau_e, double rns_eps) {
  Ctl *c = S.c;
  c->done = 0; c->k_stop = 0; c->reason = GKB_REASON_K_MAX; c->status = GKB_OK;
  c->iter = 1; c->stop = stop; c->kmax = kmax; c->bd = 0;
  c->tau_e = tau_e; c->rns_eps = rns_eps; c->scale0 = 0.0;
  c->alpha_cur = 0.0; c->t_cur = 0.0; c->cz_cur = 0.0;
  c->bscale = 1.0; c->inv_bscale = 1.0;
  c->kmax_user = kmax;
  c->learned = stop == GKB_STOP_LEARNED ? 1 : 0;
  c->phase = 1; c->k_dp = 0; c->dp_now = 0; c->stop_after = 0; c->fallback = 0; c->hybrid = 0; c->k_hat = 0;
  c->complete_last = c->learned;
  c->lambda = 0.0; c->hyb_r2 = 0.0;
  if (c->learned) c->kmax = kLearnK0;
}

// ||b||^2 of the data (FP16 storage only)
template <typename C>
__global__ void __launch_bounds__(kVT) k_bnorm(SK S, const C *__restrict__ b_in, long long m) {
  __shared__ double sh[32];
  double sq = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const double v = (double)b_in[i];
    sq += v * v;
  }
  grid_sum_finalize(sq, S.partials, S.counters + 3, &S.c->bsq, sh);
}

__global__ void k_bscale(SK S) {
  if (threadIdx.x != 0) return;
  const double nb = sqrt(S.c->bsq);
  if (nb > 0.0 && isfinite(nb)) {
    S.c->bscale = nb;
    S.c->inv_bscale = 1.0 / nb;
  }
}

// x = bscale * src (the final iterate in the caller's units)
template <typename C>
__global__ void k_copy_scaled(SK S, const C *src, C *dst, long long n) {
  const C f = (C)S.c->bscale;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = f * src[i];
}

// r = -b, z = 0, x = 0, w = 0; b in storage type; for AB/matched also s~ = b with ||b||^2.
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_init_vectors(SK S, const C *__restrict__ b_in, T *__restrict__ b_st,
                                                      C *__restrict__ r, C *__restrict__ z, long long m,
                                                      C *__restrict__ xacc, C *__restrict__ w, long long dq,
                                                      T *__restrict__ s_tmp) {
  __shared__ double sh[32];
  double sq = 0.0;
  const C inv = (C)S.c->inv_bscale;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const C bv = b_in[i] * inv;
    const T bt = from_c<T>(bv);
    b_st[i] = bt;
    r[i] = -bv;
    z[i] = C(0);
    if (s_tmp) {
      s_tmp[i] = bt;
      const double v = (double)to_c(bt);
      sq += v * v;
    }
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dq; i += stride) {
    xacc[i] = C(0);
    w[i] = C(0);
  }
  if (s_tmp) grid_sum_finalize(sq, S.partials, S.counters + 0, &S.c->tsq_cur, sh);
}

// t_1 = ||r_0||, s_1 = r_0 / t_1
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_scale_s1(SK S, const T *__restrict__ s_tmp, T *__restrict__ s_cur, long long ds) {
  if (S.c->done) return;
  const double t = sqrt(S.c->tsq_cur);
  const bool ok = t > 0.0 && isfinite(t);
  const C inv = ok ? (C)(1.0 / t) : C(0);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ds; i += stride)
    s_cur[i] = from_c<T>(to_c(s_tmp[i]) * inv);
  if (first_thread()) {
    S.t[1] = t * S.c->bscale;
    S.phibar[1] = t;
    S.c->scale0 = t;
    if (!ok) {
      S.c->done = 1; S.c->k_stop = 0;
      S.c->reason = isfinite(t) ? GKB_REASON_BREAKDOWN : GKB_REASON_ERROR;
      if (!isfinite(t)) S.c->status = GKB_ERR_NONFINITE;
    }
  }
}

// alpha_1 = ||q~||, q_1 = q~/alpha_1; w_1 = q_1; rhobar_1 = alpha_1
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_init_q1(SK S, const T *__restrict__ qt, T *__restrict__ Q0, T *__restrict__ q_cur,
                                                 C *__restrict__ w, long long dq) {
  if (S.c->done) return;
  const double a = sqrt(S.c->asq_cur);
  const bool ok = a > 0.0 && isfinite(a);
  const C inv = ok ? (C)(1.0 / a) : C(0);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dq; i += stride) {
    const T q = from_c<T>(to_c(qt[i]) * inv);
    Q0[i] = q;
    q_cur[i] = q;
    w[i] = to_c(q);
  }
  if (first_thread()) {
    S.alpha[1] = a;
    S.rhobar[1] = a;
    S.c->alpha_cur = a;
    S.c->cz_cur = 0.0;
    S.c->scale0 = fmax(S.c->scale0, a);
    if (!ok) {
      S.c->done = 1; S.c->k_stop = 0;
      S.c->reason = isfinite(a) ? GKB_REASON_BREAKDOWN : GKB_REASON_ERROR;
      if (!isfinite(a)) S.c->status = GKB_ERR_NONFINITE;
    }
  }
}

// ---------------------------------------------------------------------------
// one iteration

// t_{j+1}, s_{j+1} and the Givens update of the projected problem:
// t_{j+1}, s_{j+1}, x_j, r_j = A x_j - b and ||r_j||^2.
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_half1(SK S, const T *__restrict__ s_tmp, T *__restrict__ s_cur, long long ds,
                                               C *__restrict__ xacc, const C *__restrict__ w, long long dq,
                                               C *__restrict__ r, const C *__restrict__ z, long long m) {
  if (S.c->done) return;
  __shared__ double sh[32];
  // the scalars of this step, once per block (FP64 arithmetic is scarce: a
  // few dozen FP64 operations in every thread cost more than the vectors)
  __shared__ double s_v[8];
  __shared__ int s_f[2];
  const int j = S.c->iter;
  if (threadIdx.x == 0) {
    const double t = sqrt(S.c->tsq_cur);
    const bool finite = isfinite(t);
    const bool bd = !(t > 1e-13 * S.c->scale0);
    const double tg = (bd || !finite) ? 0.0 : t;
    const double rb = S.rhobar[j], pb = S.phibar[j];
    double rho = hypot(rb, tg), cg = 1.0, sg = 0.0;
    if (rho > 0.0) { cg = rb / rho; sg = tg / rho; }
    const double phi = cg * pb;
    s_v[0] = t; s_v[1] = tg; s_v[2] = rho; s_v[3] = cg; s_v[4] = sg; s_v[5] = sg * pb;
    s_v[6] = rho > 0.0 ? phi / rho : 0.0;
    s_v[7] = (bd || !finite) ? 0.0 : 1.0 / t;
    s_f[0] = finite; s_f[1] = bd;
  }
  __syncthreads();
  const double t = s_v[0], tg = s_v[1], rho = s_v[2], cg = s_v[3], sg = s_v[4], pb1 = s_v[5];
  const bool finite = s_f[0], bd = s_f[1];
  const C inv = (C)s_v[7];
  const C cx = (C)s_v[6];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < ds; i += stride) s_cur[i] = from_c<T>(to_c(s_tmp[i]) * inv);
  for (long long i = i0; i < dq; i += stride) xacc[i] += cx * w[i];
  double sq = 0.0;
  for (long long i = i0; i < m; i += stride) {
    const C rv = r[i] + cx * z[i];
    r[i] = rv;
    sq += (double)rv * (double)rv;
  }
  grid_sum_finalize(sq, S.partials, S.counters + 1, &S.c->rsq_cur, sh);
  if (first_thread()) {
    S.t[j + 1] = t;
    S.c->t_cur = tg;
    S.rho[j] = rho; S.cg[j] = cg; S.sg[j] = sg;
    S.phibar[j + 1] = pb1;
    S.c->bd = bd ? 1 : 0;
    if (!finite) S.c->status = GKB_ERR_NONFINITE;
  }
}

// the stopping rule on ||A x_j - b||
__global__ void k_stopcheck(SK S) {
  Ctl *c = S.c;
  if (c->done || threadIdx.x != 0) return;
  const int j = c->iter;
  const double res = sqrt(c->rsq_cur) * c->bscale;
  S.resid[j] = res;
  int stop = 0, reason = GKB_REASON_K_MAX;
  if (!isfinite(res) || c->status == GKB_ERR_NONFINITE) {
    stop = 1; reason = GKB_REASON_ERROR; c->status = GKB_ERR_NONFINITE;
  } else if (c->stop == GKB_STOP_DP && res <= c->tau_e) {
    stop = 1; reason = GKB_REASON_DP;
  } else if (c->stop == GKB_STOP_RNS && j >= 2 && fabs(S.resid[j - 1] - res) < c->rns_eps * S.resid[j - 1]) {
    stop = 1; reason = GKB_REASON_RNS;
  } else if (c->stop == GKB_STOP_HYBRID && j >= 2 && S.lam[j - 1] > 0.0 &&
             fabs(S.lam[j] - S.lam[j - 1]) <= c->rns_eps * S.lam[j - 1]) {
    stop = 1; reason = GKB_REASON_HYBRID;
  } else if (c->bd) {
    stop = 1; reason = GKB_REASON_BREAKDOWN;
  } else if (c->learned) {
    // remember the first discrepancy-principle iterate; stop at the
    // predicted index (phase 3: only once the principle has been met) or k_max
    if (res <= c->tau_e && c->k_dp == 0) { c->k_dp = j; c->dp_now = 1; }
    if (j >= c->kmax_user || (j >= c->kmax && (c->phase == 1 || c->k_dp > 0))) {
      stop = 1; reason = (c->phase == 3 && c->k_dp > 0) ? GKB_REASON_LEARNED : GKB_REASON_K_MAX;
    }
  } else if (j >= c->kmax) {
    stop = 1; reason = GKB_REASON_K_MAX;
  }
  if (stop) {
    c->k_stop = j; c->reason = reason;
    if (c->complete_last && reason == GKB_REASON_K_MAX) c->stop_after = 1;  // finish q_{j+1} and alpha_{j+1} first (resumable)
    else c->done = 1;
  }
}

// iterate history: row j-1 of hist receives x_j
template <typename C>
__global__ void k_record(SK S, const C *__restrict__ xacc, C *__restrict__ hist, long long n) {
  if (S.c->done) return;
  const long long base = (long long)(S.c->iter - 1) * n;
  const C f = (C)S.c->bscale;  // FP16 storage iterates are in units of b/||b||
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) hist[base + i] = f * xacc[i];
}

// learned mode: keep a copy of the discrepancy-principle iterate
template <typename C>
__global__ void k_save_dp(SK S, const C *__restrict__ xacc, C *__restrict__ x_dp, long long n) {
  if (!S.c->dp_now) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x_dp[i] = xacc[i];
}

// reorthogonalisation, first half: partial dot products q_i^T q~ (i < j) per 1024-row chunk
// Sums 16 values over a warp at once (a reduce-scatter: 8 + 4 + 2 + 1 + 1
// shuffles instead of 5 per value): lanes 2i and 2i + 1 end with the warp
// sum of x[i].  The order of the additions is fixed.
template <typename C>
__device__ __forceinline__ C warp_reduce_scatter16(C (&x)[16], int lane) {
  const unsigned full = 0xffffffffu;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const C send = b4 ? x[i] : x[i + 8], keep = b4 ? x[i + 8] : x[i];
    x[i] = keep + __shfl_xor_sync(full, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const C send = b3 ? x[i] : x[i + 4], keep = b3 ? x[i + 4] : x[i];
    x[i] = keep + __shfl_xor_sync(full, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const C send = b2 ? x[i] : x[i + 2], keep = b2 ? x[i + 2] : x[i];
    x[i] = keep + __shfl_xor_sync(full, send, 4);
  }
  C v = (b1 ? x[1] : x[0]) + __shfl_xor_sync(full, b1 ? x[0] : x[1], 2);
  return v + __shfl_xor_sync(full, v, 1);
}

// reorthogonalisation, first half: partial dot products of q~ with stored columns.  Block
// (chunk, group) covers 1024 rows (four per thread) and 16 columns: the 16
// loads of a thread are in flight together, a warp's 128 rows are summed in
// the compute type (FP64 arithmetic is scarce on this part) by one
// reduce-scatter, and the eight warps add in FP64 in order.
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_dots(SK S, const T *__restrict__ Q, long long ldq, const T *__restrict__ qt) {
  if (S.c->done) return;
  const int j = S.c->iter;
  const int c0 = blockIdx.y * kDotCols;
  if (c0 >= j) return;
  __shared__ C red[8][kDotCols];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const long long base = (long long)blockIdx.x * kRowsPerBlock + 4LL * tid;
  const bool in = base < ldq;
  const int nb = min(kDotCols, j - c0);
  C v[4] = {C(0), C(0), C(0), C(0)};
  if (in) load4<T, C>(qt + base, v);
  C x[kDotCols];
#pragma unroll
  for (int u = 0; u < kDotCols; ++u) {
    x[u] = C(0);
    if (in && u < nb) {
      C q[4];
      load4<T, C>(Q + (long long)(c0 + u) * ldq + base, q);
      x[u] = q[0] * v[0] + q[1] * v[1] + q[2] * v[2] + q[3] * v[3];
    }
  }
  const C ws = warp_reduce_scatter16(x, lane);
  if ((lane & 1) == 0) red[wp][lane >> 1] = ws;
  __syncthreads();
  if (tid < nb) {
    double sum = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < 8; ++w2) sum += (double)red[w2][tid];
    S.dotp[(long long)blockIdx.x * S.ldk + c0 + tid] = sum;
  }
}

// reorthogonalisation: coefficient i = sum over chunks, fixed order
// (GMRES: the coefficients of every pass add up to the column of H_k; the
// first pass sets it)
__global__ void __launch_bounds__(128) k_dots_reduce(SK S, int nchunks, int hess_pass) {
  if (S.c->done) return;
  __shared__ double sh[32];
  const int j = S.c->iter;
  const int i = blockIdx.x;
  if (i >= j) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nchunks; b += blockDim.x) acc += S.dotp[(long long)b * S.ldk + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    S.coef[i] = acc;
    if (hess_pass == 1) S.hcol[i] = acc;
    else if (hess_pass > 1) S.hcol[i] += acc;
  }
}

// reorthogonalisation, second half: q~ -= sum_i coef_i q_i, optionally with ||q~||^2
template <typename T, typename C>
__global__ void __launch_bounds__(kUT) k_update(SK S, const T *__restrict__ Q, long long ldq, T *__restrict__ qt, int with_norm) {
  if (S.c->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *cf = reinterpret_cast<C *>(smem_raw);
  __shared__ double sh[32];
  const int j = S.c->iter;
  for (int i = threadIdx.x; i < j; i += blockDim.x) cf[i] = (C)S.coef[i];
  __syncthreads();
  const long long base = 4LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  double sq = 0.0;
  if (base < ldq) {
    C acc[4] = {C(0), C(0), C(0), C(0)};
    int i = 0;
    // eight columns' loads in flight, added in the same pairs as below
    for (; i + 7 < j; i += 8) {
      C q[8][4];
#pragma unroll
      for (int c = 0; c < 8; ++c) load4<T, C>(Q + (long long)(i + c) * ldq + base, q[c]);
#pragma unroll
      for (int c = 0; c < 8; c += 2) {
        const C a0 = cf[i + c], a1 = cf[i + c + 1];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += a0 * q[c][u] + a1 * q[c + 1][u];
      }
    }
    for (; i + 3 < j; i += 4) {
      C q0[4], q1[4], q2[4], q3[4];
      load4<T, C>(Q + (long long)i * ldq + base, q0);
      load4<T, C>(Q + (long long)(i + 1) * ldq + base, q1);
      load4<T, C>(Q + (long long)(i + 2) * ldq + base, q2);
      load4<T, C>(Q + (long long)(i + 3) * ldq + base, q3);
      const C a0 = cf[i], a1 = cf[i + 1], a2 = cf[i + 2], a3 = cf[i + 3];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += a0 * q0[u] + a1 * q1[u];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += a2 * q2[u] + a3 * q3[u];
    }
    for (; i + 1 < j; i += 2) {
      C q0[4], q1[4];
      load4<T, C>(Q + (long long)i * ldq + base, q0);
      load4<T, C>(Q + (long long)(i + 1) * ldq + base, q1);
      const C a0 = cf[i], a1 = cf[i + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += a0 * q0[u] + a1 * q1[u];
    }
    if (i < j) {
      C q0[4];
      load4<T, C>(Q + (long long)i * ldq + base, q0);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += cf[i] * q0[u];
    }
    C v[4];
    load4<T, C>(qt + base, v);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T st = from_c<T>(v[u] - acc[u]);
      qt[base + u] = st;
      const double d = (double)to_c(st);
      sq += d * d;
    }
  }
  if (with_norm) grid_sum_finalize(sq, S.partials, S.counters + 2, &S.c->asq_cur, sh);
}

// alpha_{j+1}, q_{j+1} and the second Givens half (q_{j+1} stored as column j
// of Q and as the current q), theta_{j+1}, rhobar_{j+1}, w_{j+1}.
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_half2(SK S, const T *__restrict__ qt, T *__restrict__ Q, long long ldq,
                                               T *__restrict__ q_cur, C *__restrict__ w, long long dq) {
  if (S.c->done) return;
  const int j = S.c->iter;
  __shared__ double s_v[5];
  __shared__ int s_f[2];
  if (threadIdx.x == 0) {   // once per block, as in k_half1
    const double a = sqrt(S.c->asq_cur);
    const bool finite = isfinite(a);
    const bool bd = !(a > 1e-13 * S.c->scale0);
    const double al = (bd || !finite) ? 0.0 : a;
    const double theta = S.sg[j] * al;
    s_v[0] = a; s_v[1] = al; s_v[2] = -S.cg[j] * al;
    s_v[3] = S.rho[j] > 0.0 ? theta / S.rho[j] : 0.0;
    s_v[4] = (bd || !finite) ? 0.0 : 1.0 / a;
    s_f[0] = finite; s_f[1] = bd;
  }
  __syncthreads();
  const double a = s_v[0], al = s_v[1], rb1 = s_v[2], cz = s_v[3];
  const bool finite = s_f[0], bd = s_f[1];
  const C inv = (C)s_v[4];
  const C czc = (C)cz;
  T *Qj = Q + (long long)j * ldq;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dq; i += stride) {
    const T q = from_c<T>(to_c(qt[i]) * inv);
    Qj[i] = q;
    q_cur[i] = q;
    w[i] = to_c(q) - czc * w[i];
  }
  if (first_thread()) {
    S.alpha[j + 1] = a;
    S.rhobar[j + 1] = rb1;
    S.c->alpha_cur = al;
    S.c->cz_cur = cz;
    if (!finite) {
      S.c->status = GKB_ERR_NONFINITE;
      S.c->done = 1; S.c->k_stop = j; S.c->reason = GKB_REASON_ERROR;
    } else if (bd) {
      S.c->done = 1; S.c->k_stop = j; S.c->reason = GKB_REASON_BREAKDOWN;
    }
  }
}

__global__ void k_advance(SK S, cudaGraphConditionalHandle h, int use_cond) {
  if (threadIdx.x != 0) return;
  Ctl *c = S.c;
  if (c->stop_after) {
    c->stop_after = 0;
    c->done = 1;
  } else if (!c->done) {
    c->iter += 1;
  }
  c->dp_now = 0;
  if (!c->done && c->iter > c->kmax_user) c->done = 1;  // never more than k_max bodies
  if (use_cond) cudaGraphSetConditional(h, c->done ? 0u : 1u);
}

template <typename C>
__global__ void k_copy(const C *__restrict__ src, C *__restrict__ dst, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// mixed precision: the 16-bit projector operand copy of an FP32 Krylov vector
template <typename O>
__global__ void k_to_operand(SK S, const float *__restrict__ src, O *__restrict__ dst, long long n) {
  if (S.c->done) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = from_c<O>(src[i]);
}

// ---------------------------------------------------------------------------
// AB-GMRES (Algorithm 1) and BA-GMRES (Algorithm 2)
//
// Arnoldi on M = AB or BA from q_1 = r_0 / ||r_0||: iteration j forms
// w = M q_j, orthogonalises it against q_1..q_j -- classical
// Gram-Schmidt passes whose coefficients add up to the column h_{1..j,j}
// (the printed modified Gram-Schmidt and two classical passes
// agree in exact arithmetic) -- and sets h_{j+1,j} = ||w||,
// q_{j+1} = w / h_{j+1,j}, so M Q_j = Q_{j+1} H_j.  The
// projected problem min ||H_j u - ||r_0|| e_1|| is carried by the
// Givens QR of H_j (one rotation per column, FP64): g = Q^T ||r_0|| e_1 and
// R_j u_j = g_{1..j}, |g_{j+1}| its residual.  For AB-GMRES that residual is
// ||b - A x_j|| (Q orthonormal).  For BA-GMRES the data residual of Eq. DP is
// carried as r_j = A x_j - b = r_{j-1} + g_j z_j with z_j the new column of
// Z = (A Q_j) R_j^{-1}, z_j = (A q_j - sum_{i<j} R_{ij} z_i) / R_jj: the rows of
// R and of g above j never change once formed.  The iterate is formed once,
// at the stop: x = Q_k R_k^{-1} g (BA) or B Q_k R_k^{-1} g (AB).

// beta = ||r_0||, q_1 = r_0 / beta, g_1 = beta
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_gmres_q1(SK S, const T *__restrict__ r0, T *__restrict__ Q0,
                                                  T *__restrict__ q_cur, long long dq) {
  if (S.c->done) return;
  const double beta = sqrt(S.c->tsq_cur);
  const bool ok = beta > 0.0 && isfinite(beta);
  const C inv = ok ? (C)(1.0 / beta) : C(0);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dq; i += stride) {
    const T q = from_c<T>(to_c(r0[i]) * inv);
    Q0[i] = q;
    q_cur[i] = q;
  }
  if (first_thread()) {
    S.t[1] = beta * S.c->bscale;
    S.phibar[1] = beta;
    S.c->scale0 = beta;
    if (!ok) {
      S.c->done = 1; S.c->k_stop = 0;
      S.c->reason = isfinite(beta) ? GKB_REASON_BREAKDOWN : GKB_REASON_ERROR;
      if (!isfinite(beta)) S.c->status = GKB_ERR_NONFINITE;
    }
  }
}

// h_{j+1,j}, the Givens QR of the new column of H_j, g, and
// for AB-GMRES the residual |g_{j+1}|.  One thread: O(j) FP64 work.
__global__ void k_gmres_givens(SK S, int ab) {
  Ctl *c = S.c;
  if (c->done || threadIdx.x != 0) return;
  const int j = c->iter;
  const double hn = sqrt(c->asq_cur);
  const bool finite = isfinite(hn);
  const bool bd = !(hn > 1e-13 * c->scale0);
  double *h = S.hcol;
  S.alpha[j] = h[j - 1];                 // the diagonal of H_j, before rotation
  S.t[j + 1] = hn;                       // its subdiagonal (scale-free: the q_i are unit vectors)
  S.rho[j] = hn;
  for (int i = 1; i < j; ++i) {          // earlier rotations, in order
    const double cs = S.cg[i], sn = S.sg[i], a = h[i - 1], b = h[i];
    h[i - 1] = cs * a + sn * b;
    h[i] = -sn * a + cs * b;
  }
  const double a = h[j - 1], rho = hypot(a, hn);
  const double cs = rho > 0.0 ? a / rho : 1.0, sn = rho > 0.0 ? hn / rho : 0.0;
  S.cg[j] = cs;
  S.sg[j] = sn;
  double *Rj = S.R + (long long)(j - 1) * S.ldk;
  for (int i = 0; i < j - 1; ++i) Rj[i] = h[i];
  Rj[j - 1] = rho;
  const double gj = S.phibar[j];
  S.phibar[j] = cs * gj;
  S.phibar[j + 1] = -sn * gj;
  if (ab) c->rsq_cur = S.phibar[j + 1] * S.phibar[j + 1];
  c->bd = bd ? 1 : 0;
  if (!finite || !(rho > 0.0)) c->status = GKB_ERR_NONFINITE;
}

// q_{j+1} = w / h_{j+1,j}, stored as column j of Q and as the current q
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_gmres_qnext(SK S, const T *__restrict__ w, T *__restrict__ Q, long long ldq,
                                                     T *__restrict__ q_cur, long long dq) {
  if (S.c->done || S.c->bd) return;
  const int j = S.c->iter;
  const C inv = (C)(1.0 / S.rho[j]);
  T *Qj = Q + (long long)j * ldq;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < dq; i += stride) {
    const T q = from_c<T>(to_c(w[i]) * inv);
    Qj[i] = q;
    q_cur[i] = q;
  }
}

// BA-GMRES: z_j = (A q_j - sum_{i<j} R_ij z_i) / R_jj into column j-1 of Z,
// r += g_j z_j (r = A x_j - b) and ||r||^2
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_gmres_resid(SK S, const T *__restrict__ Aq, C *__restrict__ Z, long long ldz,
                                                     C *__restrict__ r, long long m) {
  if (S.c->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *cf = reinterpret_cast<C *>(smem_raw);
  __shared__ double sh[32];
  const int j = S.c->iter;
  const double *Rj = S.R + (long long)(j - 1) * S.ldk;
  for (int i = threadIdx.x; i < j - 1; i += blockDim.x) cf[i] = (C)Rj[i];
  const C inv = (C)(1.0 / Rj[j - 1]), gj = (C)S.phibar[j];
  __syncthreads();
  double sq = 0.0;
  C *Zj = Z + (long long)(j - 1) * ldz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
    C acc = to_c(Aq[k]);
    for (int i = 0; i < j - 1; ++i) acc -= cf[i] * Z[(long long)i * ldz + k];
    const C z = acc * inv;
    Zj[k] = z;
    const C rv = r[k] + gj * z;
    r[k] = rv;
    sq += (double)rv * (double)rv;
  }
  grid_sum_finalize(sq, S.partials, S.counters + 1, &S.c->rsq_cur, sh);
}

// at the stop: u = R_k^{-1} g_{1..k} (back substitution, FP64, one block) into coef
__global__ void __launch_bounds__(256) k_gmres_backsub(SK S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *gv = reinterpret_cast<double *>(smem_raw);
  const int k = S.c->k_stop;
  for (int i = threadIdx.x; i < k; i += blockDim.x) gv[i] = S.phibar[i + 1];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double *Ri = S.R + (long long)i * S.ldk;   // column i
    const double ui = gv[i] / Ri[i];
    for (int l = threadIdx.x; l < i; l += blockDim.x) gv[l] -= Ri[l] * ui;
    if (threadIdx.x == 0) S.coef[i] = ui;
    __syncthreads();
  }
}

// x = sum_{i < k} u_i q_{i+1}
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_qu(SK S, const T *__restrict__ Q, long long ldq, C *__restrict__ x,
                                            long long n) {
  const int k = S.c->k_stop;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    C acc = C(0);
    for (int i = 0; i < k; ++i) acc += (C)S.coef[i] * to_c(Q[(long long)i * ldq + r]);
    x[r] = acc;
  }
}

// ---------------------------------------------------------------------------
// learned stopping (BA, FP32)

// Projected Tikhonov problem on C_k: (C^T C + lam^2 I) u = t_1 alpha_1 e_1
// (C^T C is tridiagonal: diagonal alpha_{i+1}^2 + t_{i+2}^2, off-diagonal
// alpha_{i+2} t_{i+2}), solved by the Thomas algorithm in FP64.  Returns
// ||C_k u - t_1 e_1||.  u and cp need k entries.
__device__ double tikhonov_solve(const double *al, const double *tt, int k, double lam, double *u, double *cp) {
  const double l2 = lam * lam;
  double dprev = 0.0;
  for (int i = 0; i < k; ++i) {
    const double diag = al[i + 1] * al[i + 1] + tt[i + 2] * tt[i + 2] + l2;
    const double lower = (i > 0) ? al[i + 1] * tt[i + 1] : 0.0;   // couples i-1 and i
    const double rhs = (i == 0) ? tt[1] * al[1] : 0.0;
    const double mden = diag - (i > 0 ? lower * cp[i - 1] : 0.0);
    const double upper = (i + 1 < k) ? al[i + 2] * tt[i + 2] : 0.0;
    cp[i] = upper / mden;
    const double dcur = (rhs - (i > 0 ? lower * dprev : 0.0)) / mden;
    u[i] = dcur;
    dprev = dcur;
  }
  for (int i = k - 2; i >= 0; --i) u[i] -= cp[i] * u[i + 1];
  double r2 = 0.0, r = al[1] * u[0] - tt[1];
  r2 += r * r;
  for (int i = 1; i < k; ++i) {
    r = tt[i + 1] * u[i - 1] + al[i + 1] * u[i];
    r2 += r * r;
  }
  r = tt[k + 1] * u[k - 1];
  r2 += r * r;
  return sqrt(r2);
}

// The 64 features of the first kLearnK0 iterations: log alpha_1..16,
// log t_2..17, log(r_k / (tau ||e||)) and log(phibar_{k+1} / t_1) for k = 1..16.
__device__ __forceinline__ float learned_feature(const SK &S, int i) {
  const int g = i / kLearnK0, j = i % kLearnK0 + 1;
  double v;
  if (g == 0) v = S.alpha[j];
  else if (g == 1) v = S.t[j + 1];
  else if (g == 2) v = S.resid[j] / S.c->tau_e;
  else v = S.phibar[j + 1] / S.t[1];
  return (float)log(fmax(fabs(v), 1e-30));
}

__global__ void __launch_bounds__(kHid) k_learned_predict(const SK *__restrict__ sks, const __nv_bfloat16 *__restrict__ theta,
                                                         const float *__restrict__ norm, int delta) {
  const SK S = sks[blockIdx.x];
  Ctl *c = S.c;
  if (!c->learned || !(c->done && c->reason == GKB_REASON_K_MAX && c->phase == 1)) return;
  __shared__ float feat[kIn], h1[kHid], h2[kHid], out[kOut];
  if (threadIdx.x < kIn) feat[threadIdx.x] = learned_feature(S, threadIdx.x);
  __syncthreads();
  mlp_infer_block(theta, norm, feat, h1, h2, out);
  if (threadIdx.x == 0) {
    const float kf = expf(fminf(out[0], 20.f));
    int kh = (int)lrintf(kf);
    kh = max(kh, 1);
    c->k_hat = kh;
    c->lambda = (double)expf(fminf(fmaxf(out[1], -60.f), 60.f));
    c->kmax = min(max(kh + delta, kLearnK0 + 1), c->kmax_user);
  }
}

__global__ void k_resume(SK S) {
  Ctl *c = S.c;
  if (threadIdx.x != 0 || !c->learned || c->phase != 1) return;
  if (c->done && c->reason == GKB_REASON_K_MAX && c->k_stop < c->kmax_user) {
    c->done = 0;
    c->iter = c->k_stop + 1;
    c->phase = 3;
    c->complete_last = 0;
  }
}

// the hybrid step: u_lambda on C_k (FP64, one thread)
__global__ void k_learned_tikhonov(SK S) {
  Ctl *c = S.c;
  if (threadIdx.x != 0 || !c->learned) return;
  c->hybrid = 0;
  if (c->k_dp == 0 || c->status != GKB_OK || c->k_stop < 1) return;
  tikhonov_solve(S.alpha, S.t, c->k_stop, c->lambda, S.coef, S.dotp);
  c->hybrid = 1;
}

// Hybrid regularisation, after iteration j: lambda_j from the discrepancy
// principle on the projected problem.  lambda_j = 0 while the least-squares
// residual |phibar_{j+1}| is above tau ||e||; otherwise the root of
// ||C_j u_lambda - t_1 e_1|| = tau ||e|| (increasing in lambda) in log(lambda)
// over [1e-9, 10] alpha_1: each of six rounds evaluates 32 points of the
// bracket, one per lane (tikhonov_solve in FP64, a lane's tridiagonal
// scratch in global memory), and keeps the interval where the residual
// crosses the target, 33 times narrower; the result is lambda to ~2e-8
// relative.  One warp.
__global__ void __launch_bounds__(32) k_hybrid_lambda(SK S) {
  const Ctl *c = S.c;
  if (c->done) return;
  const int j = c->iter, lane = threadIdx.x;
  const double target = c->tau_e;
  if (!(fabs(S.phibar[j + 1]) < target)) {
    if (lane == 0) S.lam[j] = 0.0;
    return;
  }
  double *u = S.hyb + (long long)lane * 2 * S.ldk, *cp = u + S.ldk;
  double lo = log(S.alpha[1] * 1e-9), hi = log(S.alpha[1] * 10.0);
  for (int round = 0; round < 6; ++round) {
    const double mu = lo + (hi - lo) * (lane + 1) / 33.0;
    const bool above = tikhonov_solve(S.alpha, S.t, j, exp(mu), u, cp) > target;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    const int f = m ? __ffs(m) - 1 : 32;   // the crossing lies between points f and f + 1
    const double nlo = lo + (hi - lo) * f / 33.0, nhi = lo + (hi - lo) * (f + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) S.lam[j] = exp(0.5 * (lo + hi));
}

// at the stop: u_lambda of C_k into coef (lambda = 0: the least-squares u)
__global__ void k_hybrid_coef(SK S) {
  if (threadIdx.x != 0) return;
  const int k = S.c->k_stop;
  if (k >= 1) tikhonov_solve(S.alpha, S.t, k, S.lam[k], S.coef, S.dotp);
}

// x = sum_{i < k} u_i q_{i+1}
template <typename T, typename C>
__global__ void __launch_bounds__(kVT) k_combine(SK S, const T *__restrict__ Q, long long ldq, C *__restrict__ x, long long n) {
  if (!S.c->hybrid) return;
  const int k = S.c->k_stop;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    C acc = C(0);
    for (int i = 0; i < k; ++i) acc += (C)S.coef[i] * to_c(Q[(long long)i * ldq + r]);
    x[r] = acc;
  }
}

// ||A x_hyb - b||^2
template <typename C>
__global__ void __launch_bounds__(kVT) k_hyb_resid(SK S, const C *__restrict__ Ax, const C *__restrict__ b, long long m) {
  if (!S.c->hybrid) return;
  __shared__ double sh[32];
  double sq = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const double d = (double)Ax[i] - (double)b[i];
    sq += d * d;
  }
  grid_sum_finalize(sq, S.partials, S.counters + 4, &S.c->hyb_r2, sh);
}

// Accept the hybrid iterate if its data residual is within 5 % of tau ||e||,
// else fall back to the discrepancy-principle iterate (or to the last one).
template <typename C>
__global__ void __launch_bounds__(kVT) k_learned_select(SK S, C *__restrict__ x_out, const C *__restrict__ x_dp,
                                                        const C *__restrict__ xacc, long long n) {
  Ctl *c = S.c;
  if (!c->learned) return;
  const bool ok = c->hybrid && fabs(sqrt(c->hyb_r2) - c->tau_e) <= 0.05 * c->tau_e;
  if (!ok) {
    const C *src = c->k_dp > 0 ? x_dp : xacc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x_out[i] = src[i];
  }
  if (first_thread()) c->fallback = ok ? 0 : (c->k_dp > 0 ? 1 : 2);
}

// Training data of one slice solved without a stopping rule: the features,
// and the labels log k_DP and log lambda*, lambda* being the projected
// Tikhonov parameter at k_DP + delta whose projected residual equals that of
// the plain iterate at k_DP (bisection in log lambda, FP64).
__global__ void __launch_bounds__(kHid) k_learned_labels(const SK *__restrict__ sks, int delta, float *__restrict__ X,
                                                        float *__restrict__ Tg, int *__restrict__ valid) {
  const SK S = sks[blockIdx.x];
  const Ctl *c = S.c;
  if (threadIdx.x < kIn) X[(long long)blockIdx.x * kIn + threadIdx.x] = learned_feature(S, threadIdx.x);
  if (threadIdx.x != 0) return;
  const int kend = c->k_stop;
  int kdp = 0;
  for (int k = 1; k <= kend; ++k)
    if (S.resid[k] <= c->tau_e) { kdp = k; break; }
  const int klab = kdp + delta;
  int ok = kdp > kLearnK0 / 2 && klab <= kend && c->status == GKB_OK;
  double lam = 0.0;
  if (ok) {
    const double target = S.phibar[kdp + 1];
    double lo = log(S.alpha[1] * 1e-9), hi = log(S.alpha[1] * 10.0);
    for (int it = 0; it < 100; ++it) {
      const double mid = 0.5 * (lo + hi);
      const double r = tikhonov_solve(S.alpha, S.t, klab, exp(mid), S.coef, S.dotp);
      if (r > target) hi = mid; else lo = mid;
    }
    lam = exp(0.5 * (lo + hi));
    ok = isfinite(lam) && lam > 0.0;
  }
  valid[blockIdx.x] = ok;
  Tg[(long long)blockIdx.x * kOut + 0] = ok ? (float)log((double)kdp) : 0.f;
  Tg[(long long)blockIdx.x * kOut + 1] = ok ? (float)log(lam) : 0.f;
}

int vec_grid(long long len) {
  long long b = (len + kVT * 4 - 1) / (kVT * 4);
  if (b < 1) b = 1;
  if (b > 148 * 8) b = 148 * 8;
  return (int)b;
}

}  // namespace
}  // namespace gkb

// ---------------------------------------------------------------------------
// host side

using namespace gkb;

struct gkb_plan {
  const gkb_geometry *g = nullptr;
  gkb_solve_params p{};
  bool f64 = false;
  long long n = 0, m = 0, ds = 0, dq = 0, ldq = 0;
  int kmax = 0, nchunks = 0;
  size_t tsz = 0, csz = 0;   // storage and compute element sizes
  gkb_dtype io_dt = GKB_F32; // dtype of the compute-type vectors as a projector operand
  gkb_dtype op_dt = GKB_F32; // type the projectors read and write inside the iteration
  bool mixed = false;        // op_dt is 16-bit while the Krylov vectors are FP32
  void *q_op = nullptr, *s_op = nullptr, *b_op = nullptr;   // mixed: 16-bit copies of q_j, s_j and b
  // device memory
  void *arena = nullptr;
  void *Q = nullptr, *s_cur = nullptr, *s_tmp = nullptr, *qt = nullptr, *q_cur = nullptr;
  void *vM = nullptr, *tmp = nullptr, *b_st = nullptr;
  void *xacc = nullptr, *w = nullptr, *z = nullptr, *r = nullptr, *b_in = nullptr, *x_out = nullptr;
  void *xt = nullptr;  // transposed image for the banded projector kernels
  void *acc = nullptr;  // integer accumulators of the B^T scatter (m x 8 bytes + 256), zero between calls
  void *fadj = nullptr;  // the A^T scatter's two FP32 partial images (2 n floats)
  void *x_dp = nullptr;  // learned mode: the discrepancy-principle iterate
  void *hist = nullptr;  // optional: k_max iterates of n values (caller-owned)
  bool gmres = false;     // AB- or BA-GMRES (Algorithms 1-2)
  void *Z = nullptr;      // BA-GMRES: (A Q) R^{-1}, k_max columns of m (compute type)
  long long ldz = 0;
  double *scal = nullptr, *partials = nullptr, *dotp = nullptr, *coef = nullptr;
  unsigned *counters = nullptr;
  Ctl *ctl = nullptr;
  SK sk{};
  // graph
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr, cap_body = nullptr;
  int graph_ok = 0;
  cudaGraph_t body_graph = nullptr;                    // valid during capture only
  long long kernels_outer = -1, kernels_body = -1;    // kernel nodes of the captured graph
  struct Prof *prof = nullptr;                         // gkb_plan_profile: events between kernel groups
};

// grids of the reorthogonalisation kernels: dots over (row chunk, column
// group of kDotCols, enough groups for every stored column), update over
// kUT-thread blocks of four rows per thread
dim3 dots_grid(const gkb_plan *P) {
  return dim3((unsigned)P->nchunks, (unsigned)((P->kmax + 1 + kDotCols - 1) / kDotCols));
}
int update_blocks(const gkb_plan *P) { return (int)((P->ldq / 4 + kUT - 1) / kUT); }


namespace {

// An empty epilogue carrying the plan's transposed-image scratch buffer.
Epi plan_epi(const gkb_plan *P) {
  Epi e;
  e.scratch_t = P->xt;
  e.scratch_acc = P->acc;
  e.scratch_fadj = P->fadj;
  return e;
}

// Kernel classes of gkb_plan_profile: the four projectors, the two halves of
// the reorthogonalisation, everything else (scalars, vector updates, stop).
enum { PC_A = 0, PC_B, PC_AT, PC_BT, PC_DOTS, PC_UPDATE, PC_OTHER, PC_COUNT };

}  // namespace

// An event before every kernel group of a profiled run; the time to the next
// event belongs to the group's class.
struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  size_t used = 0;
  bool failed = false;
};

namespace {

void mark(gkb_plan *P, cudaStream_t s, int cls) {
  Prof *pr = P->prof;
  if (!pr || pr->failed) return;
  if (pr->used == pr->ev.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      pr->failed = true;
      return;
    }
    pr->ev.push_back(e);
    pr->cls.push_back(0);
  }
  cudaEventRecord(pr->ev[pr->used], s);
  pr->cls[pr->used] = cls;
  ++pr->used;
}

gkb_status opA(gkb_plan *P, gkb_dtype dt, const void *in, void *out, const Epi &e, cudaStream_t s) {
  mark(P, s, PC_A);
  return launch_forward(P->g, dt, in, out, e, s);
}
gkb_status opB(gkb_plan *P, gkb_dtype dt, const void *in, void *out, const Epi &e, cudaStream_t s) {
  mark(P, s, PC_B);
  return launch_back(P->g, dt, in, out, e, s);
}
gkb_status opAT(gkb_plan *P, gkb_dtype dt, const void *in, void *out, const Epi &e, cudaStream_t s) {
  mark(P, s, PC_AT);
  return launch_forward_adj(P->g, dt, in, out, e, s);
}
gkb_status opBT(gkb_plan *P, gkb_dtype dt, const void *in, void *out, const Epi &e, cudaStream_t s) {
  mark(P, s, PC_BT);
  return launch_back_adj(P->g, dt, in, out, e, s);
}

// Operands of the projectors: the Krylov vectors themselves, or (mixed
// precision) their 16-bit copies.
const void *q_in(const gkb_plan *P) { return P->mixed ? P->q_op : P->q_cur; }
const void *s_in(const gkb_plan *P) { return P->mixed ? P->s_op : P->s_cur; }
const void *b_in_op(const gkb_plan *P) { return P->mixed ? P->b_op : P->b_st; }
// The second projector of a step writes a Krylov vector: in mixed precision
// its epilogue stores the FP32 result and reads the FP32 previous vector.
Epi krylov_out(Epi e, const gkb_plan *P, void *dst) {
  if (P->mixed) {
    e.out32 = dst;
    e.prev32 = true;
  }
  return e;
}
void to_operand(const gkb_plan *P, const void *src, void *dst, long long n, cudaStream_t s) {
  if (!P->mixed) return;
  if (P->op_dt == GKB_BF16)
    k_to_operand<__nv_bfloat16><<<vec_grid(n), kVT, 0, s>>>(P->sk, (const float *)src, (__nv_bfloat16 *)dst, n);
  else
    k_to_operand<__half><<<vec_grid(n), kVT, 0, s>>>(P->sk, (const float *)src, (__half *)dst, n);
}

template <typename T, typename C>
gkb_status enqueue_init(gkb_plan *P, cudaStream_t s) {
  mark(P, s, PC_OTHER);
  const SK &S = P->sk;
  const gkb_dtype dt = P->op_dt;
  const double tau = P->p.tau > 0.0 ? P->p.tau : 1.0;
  k_reset<<<1, 1, 0, s>>>(S, P->kmax, (int)P->p.stop, tau * P->p.noise_norm, P->p.rns_eps);
  if (P->op_dt == GKB_F16) {  // FP16's range: run on b/||b||
    k_bnorm<C><<<vec_grid(P->m), kVT, 0, s>>>(S, (const C *)P->b_in, P->m);
    k_bscale<<<1, 32, 0, s>>>(S);
  }
  const bool ba = P->p.variant == GKB_BA || P->p.variant == GKB_BA_GMRES;
  k_init_vectors<T, C><<<vec_grid(std::max(P->m, P->dq)), kVT, 0, s>>>(
      S, (const C *)P->b_in, (T *)P->b_st, (C *)P->r, (C *)P->z, P->m, (C *)P->xacc, (C *)P->w, P->dq,
      ba ? (T *)nullptr : (T *)P->s_tmp);
  to_operand(P, P->b_st, P->b_op, P->m, s);
  GKB_CUDA_TRY(cudaGetLastError());
  Epi e = plan_epi(P);
  e.partials = P->partials; e.counter = P->counters + 0; e.result = &P->ctl->tsq_cur;
  gkb_status st;
  if (ba) {  // t_1 = ||B b||
    if ((st = opB(P, dt, b_in_op(P), P->s_tmp, krylov_out(e, P, P->s_tmp), s)) != GKB_OK) return st;
  }
  mark(P, s, PC_OTHER);
  if (P->gmres) {  // Algorithms 1-2: q_1 = r_0 / ||r_0||
    k_gmres_q1<T, C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const T *)P->s_tmp, (T *)P->Q, (T *)P->q_cur, P->dq);
    GKB_CUDA_TRY(cudaGetLastError());
    return GKB_OK;
  }
  k_scale_s1<T, C><<<vec_grid(P->ds), kVT, 0, s>>>(S, (const T *)P->s_tmp, (T *)P->s_cur, P->ds);
  to_operand(P, P->s_cur, P->s_op, P->ds, s);
  GKB_CUDA_TRY(cudaGetLastError());
  // q = M^T s_1
  Epi eq = plan_epi(P);
  eq.partials = P->partials; eq.counter = P->counters + 2; eq.result = &P->ctl->asq_cur; eq.done = &P->ctl->done;
  Epi en = plan_epi(P);
  en.done = &P->ctl->done;
  eq = krylov_out(eq, P, P->qt);
  if (P->p.variant == GKB_BA) {
    if ((st = opBT(P, dt, s_in(P), P->tmp, en, s)) != GKB_OK) return st;
    if ((st = opAT(P, dt, P->tmp, P->qt, eq, s)) != GKB_OK) return st;
  } else if (P->p.variant == GKB_AB) {
    if ((st = opAT(P, dt, s_in(P), P->tmp, en, s)) != GKB_OK) return st;
    if ((st = opBT(P, dt, P->tmp, P->qt, eq, s)) != GKB_OK) return st;
  } else {
    if ((st = opAT(P, dt, s_in(P), P->qt, eq, s)) != GKB_OK) return st;
  }
  mark(P, s, PC_OTHER);
  k_init_q1<T, C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const T *)P->qt, (T *)P->Q, (T *)P->q_cur, (C *)P->w, P->dq);
  to_operand(P, P->q_cur, P->q_op, P->dq, s);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

// One AB-/BA-GMRES iteration (Algorithms 1-2).
template <typename T, typename C>
gkb_status enqueue_body_gmres(gkb_plan *P, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  const SK &S = P->sk;
  const gkb_dtype dt = P->p.storage;
  const bool ba = P->p.variant == GKB_BA_GMRES;
  gkb_status st;
  Epi e1 = plan_epi(P);
  e1.done = &P->ctl->done;
  // w = M q_j (BA keeps A q_j in vM for the residual recurrence)
  if (ba) {
    if ((st = opA(P, dt, P->q_cur, P->vM, e1, s)) != GKB_OK) return st;
    if ((st = opB(P, dt, P->vM, P->qt, e1, s)) != GKB_OK) return st;
  } else {
    if ((st = opB(P, dt, P->q_cur, P->tmp, e1, s)) != GKB_OK) return st;
    if ((st = opA(P, dt, P->tmp, P->qt, e1, s)) != GKB_OK) return st;
  }
  // Gram-Schmidt passes; their coefficients add up to h_{1..j,j}
  const int passes = std::max(P->p.reorth, 1);
  for (int pass = 0; pass < passes; ++pass) {
    const int last = pass == passes - 1;
    mark(P, s, PC_DOTS);
    k_dots<T, C><<<dots_grid(P), kVT, 0, s>>>(S, (const T *)P->Q, P->ldq, (const T *)P->qt);
    k_dots_reduce<<<P->kmax + 1, 128, 0, s>>>(S, P->nchunks, pass + 1);
    mark(P, s, PC_UPDATE);
    k_update<T, C><<<update_blocks(P), kUT, (P->kmax + 1) * sizeof(C), s>>>(S, (const T *)P->Q, P->ldq, (T *)P->qt, last);
    GKB_CUDA_TRY(cudaGetLastError());
  }
  // h_{j+1,j}, q_{j+1}, the Givens QR of H_j, then the residual and the stop
  mark(P, s, PC_OTHER);
  k_gmres_givens<<<1, 32, 0, s>>>(S, ba ? 0 : 1);
  k_gmres_qnext<T, C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const T *)P->qt, (T *)P->Q, P->ldq, (T *)P->q_cur, P->dq);
  if (ba)
    k_gmres_resid<T, C><<<vec_grid(P->m), kVT, (P->kmax + 1) * sizeof(C), s>>>(S, (const T *)P->vM, (C *)P->Z, P->ldz,
                                                                              (C *)P->r, P->m);
  k_stopcheck<<<1, 32, 0, s>>>(S);
  k_advance<<<1, 32, 0, s>>>(S, h, use_cond);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

template <typename T, typename C>
gkb_status enqueue_body(gkb_plan *P, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  if (P->gmres) return enqueue_body_gmres<T, C>(P, s, h, use_cond);
  const SK &S = P->sk;
  const gkb_dtype dt = P->op_dt;
  gkb_status st;
  const int *done = &P->ctl->done;
  // s~ = M q_j - alpha_j s_j, with z <- (A q_j or M q_j) - cz z and ||s~||^2
  Epi e1 = plan_epi(P);  // plain
  e1.done = done;
  Epi es = plan_epi(P);  // final launch of s~ = M q_j - alpha_j s_j
  es.done = done;
  es.prev = P->s_cur; es.gamma = &P->ctl->alpha_cur;
  es.partials = P->partials; es.counter = P->counters + 0; es.result = &P->ctl->tsq_cur;
  es = krylov_out(es, P, P->s_tmp);
  if (P->p.variant == GKB_BA) {
    Epi ez = e1;
    ez.z = P->z; ez.cz = &P->ctl->cz_cur;
    if ((st = opA(P, dt, q_in(P), P->vM, ez, s)) != GKB_OK) return st;
    if ((st = opB(P, dt, P->vM, P->s_tmp, es, s)) != GKB_OK) return st;
  } else if (P->p.variant == GKB_AB) {
    if ((st = opB(P, dt, q_in(P), P->tmp, e1, s)) != GKB_OK) return st;
    es.z = P->z; es.cz = &P->ctl->cz_cur;
    if ((st = opA(P, dt, P->tmp, P->s_tmp, es, s)) != GKB_OK) return st;
  } else {
    es.z = P->z; es.cz = &P->ctl->cz_cur;
    if ((st = opA(P, dt, q_in(P), P->s_tmp, es, s)) != GKB_OK) return st;
  }
  // t_{j+1}, s_{j+1} + Givens + x, r updates
  mark(P, s, PC_OTHER);
  k_half1<T, C><<<vec_grid(std::max(std::max(P->ds, P->dq), P->m)), kVT, 0, s>>>(
      S, (const T *)P->s_tmp, (T *)P->s_cur, P->ds, (C *)P->xacc, (const C *)P->w, P->dq, (C *)P->r,
      (const C *)P->z, P->m);
  to_operand(P, P->s_cur, P->s_op, P->ds, s);
  if (P->hist)  // x_j is complete once s_{j+1} and the Givens update are done
    k_record<C><<<vec_grid(P->n), kVT, 0, s>>>(S, (const C *)P->xacc, (C *)P->hist, P->n);
  if (P->p.stop == GKB_STOP_HYBRID) k_hybrid_lambda<<<1, 32, 0, s>>>(S);
  k_stopcheck<<<1, 32, 0, s>>>(S);
  if (P->p.stop == GKB_STOP_LEARNED)
    k_save_dp<C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const C *)P->xacc, (C *)P->x_dp, P->dq);
  GKB_CUDA_TRY(cudaGetLastError());
  // q~ = M^T s_{j+1} - t_{j+1} q_j
  Epi eq = plan_epi(P);
  eq.done = done;
  eq.prev = P->q_cur; eq.gamma = &P->ctl->t_cur;
  if (P->p.reorth == 0) {
    eq.partials = P->partials; eq.counter = P->counters + 2; eq.result = &P->ctl->asq_cur;
  }
  eq = krylov_out(eq, P, P->qt);
  if (P->p.variant == GKB_BA) {
    if ((st = opBT(P, dt, s_in(P), P->tmp, e1, s)) != GKB_OK) return st;
    if ((st = opAT(P, dt, P->tmp, P->qt, eq, s)) != GKB_OK) return st;
  } else if (P->p.variant == GKB_AB) {
    if ((st = opAT(P, dt, s_in(P), P->tmp, e1, s)) != GKB_OK) return st;
    if ((st = opBT(P, dt, P->tmp, P->qt, eq, s)) != GKB_OK) return st;
  } else {
    if ((st = opAT(P, dt, s_in(P), P->qt, eq, s)) != GKB_OK) return st;
  }
  // reorthogonalisation
  for (int pass = 0; pass < P->p.reorth; ++pass) {
    const int last = pass == P->p.reorth - 1;
    mark(P, s, PC_DOTS);
    k_dots<T, C><<<dots_grid(P), kVT, 0, s>>>(S, (const T *)P->Q, P->ldq, (const T *)P->qt);
    k_dots_reduce<<<P->kmax + 1, 128, 0, s>>>(S, P->nchunks, 0);
    mark(P, s, PC_UPDATE);
    k_update<T, C><<<update_blocks(P), kUT, (P->kmax + 1) * sizeof(C), s>>>(S, (const T *)P->Q, P->ldq, (T *)P->qt, last);
    GKB_CUDA_TRY(cudaGetLastError());
  }
  // alpha_{j+1}, q_{j+1}
  mark(P, s, PC_OTHER);
  k_half2<T, C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const T *)P->qt, (T *)P->Q, P->ldq, (T *)P->q_cur, (C *)P->w, P->dq);
  to_operand(P, P->q_cur, P->q_op, P->dq, s);
  k_advance<<<1, 32, 0, s>>>(S, h, use_cond);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

template <typename T, typename C>
gkb_status enqueue_final(gkb_plan *P, cudaStream_t s) {
  mark(P, s, PC_OTHER);
  const bool hybrid = P->p.stop == GKB_STOP_HYBRID;
  if (P->gmres || hybrid) {  // u = R^{-1} g (GMRES) or u_lambda (hybrid); x = Q u (BA, matched) or B Q u (AB)
    const SK &S = P->sk;
    if (hybrid) k_hybrid_coef<<<1, 32, 0, s>>>(S);
    else k_gmres_backsub<<<1, 256, sizeof(double) * (P->kmax + 2), s>>>(S);
    k_qu<T, C><<<vec_grid(P->dq), kVT, 0, s>>>(S, (const T *)P->Q, P->ldq, (C *)P->xacc, P->dq);
    GKB_CUDA_TRY(cudaGetLastError());
    const bool scaled = P->op_dt == GKB_F16;
    if (P->p.variant == GKB_AB_GMRES || P->p.variant == GKB_AB) {
      gkb_status st = opB(P, P->io_dt, P->xacc, P->x_out, plan_epi(P), s);
      if (st != GKB_OK || !scaled) return st;
      k_copy_scaled<C><<<vec_grid(P->n), kVT, 0, s>>>(S, (const C *)P->x_out, (C *)P->x_out, P->n);
    } else if (scaled) {
      k_copy_scaled<C><<<vec_grid(P->n), kVT, 0, s>>>(S, (const C *)P->xacc, (C *)P->x_out, P->n);
    } else {
      k_copy<C><<<vec_grid(P->n), kVT, 0, s>>>((const C *)P->xacc, (C *)P->x_out, P->n);
    }
    GKB_CUDA_TRY(cudaGetLastError());
    return GKB_OK;
  }
  if (P->p.stop == GKB_STOP_LEARNED) {  // hybrid step with the predicted lambda, checked by the discrepancy principle
    const SK &S = P->sk;
    k_learned_tikhonov<<<1, 32, 0, s>>>(S);
    k_combine<T, C><<<vec_grid(P->n), kVT, 0, s>>>(S, (const T *)P->Q, P->ldq, (C *)P->x_out, P->n);
    gkb_status st = opA(P, P->io_dt, P->x_out, P->vM, plan_epi(P), s);
    if (st != GKB_OK) return st;
    k_hyb_resid<C><<<vec_grid(P->m), kVT, 0, s>>>(S, (const C *)P->vM, (const C *)P->b_in, P->m);
    k_learned_select<C><<<vec_grid(P->n), kVT, 0, s>>>(S, (C *)P->x_out, (const C *)P->x_dp, (const C *)P->xacc, P->n);
    GKB_CUDA_TRY(cudaGetLastError());
    return GKB_OK;
  }
  const bool scaled = P->op_dt == GKB_F16;
  if (P->p.variant == GKB_AB) {
    gkb_status st = opB(P, P->io_dt, P->xacc, P->x_out, plan_epi(P), s);
    if (st != GKB_OK || !scaled) return st;
    k_copy_scaled<C><<<vec_grid(P->n), kVT, 0, s>>>(P->sk, (const C *)P->x_out, (C *)P->x_out, P->n);
  } else if (scaled) {
    k_copy_scaled<C><<<vec_grid(P->n), kVT, 0, s>>>(P->sk, (const C *)P->xacc, (C *)P->x_out, P->n);
  } else {
    k_copy<C><<<vec_grid(P->n), kVT, 0, s>>>((const C *)P->xacc, (C *)P->x_out, P->n);
  }
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

// Enqueue a whole solve into the capture in progress on stream s: the
// initialisation, a WHILE node whose body (one iteration, captured through
// body_stream) runs until the device-side stop, and the final combination.
// part 0: the whole solve; 1: initialisation and loop (learned phase 1);
// 3: resume, loop and final combination (learned phase 3).
template <typename T, typename C>
gkb_status enqueue_solve_captured(gkb_plan *P, cudaStream_t s, cudaStream_t body_stream, int part = 0) {
  gkb_status st = GKB_OK;
  if (part == 3) {
    k_resume<<<1, 32, 0, s>>>(P->sk);
    GKB_CUDA_TRY(cudaGetLastError());
  } else {
    st = enqueue_init<T, C>(P, s);
  }
  if (st != GKB_OK) return st;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t cg = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNode_t node = nullptr;
  GKB_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
  GKB_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
  // zero-initialised parameter block (the type has no default constructor)
  alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
  std::memset(cpbuf, 0, sizeof(cpbuf));
  cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cpbuf);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  GKB_CUDA_TRY(cudaGraphAddNode(&node, cg, dv.data(), nullptr, dv.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  P->body_graph = body;
  GKB_CUDA_TRY(cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  st = enqueue_body<T, C>(P, body_stream, h, 1);
  cudaGraph_t bg = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(body_stream, &bg);
  if (st != GKB_OK) return st;
  GKB_CUDA_TRY(e2);
  GKB_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  if (part == 1) return GKB_OK;
  return enqueue_final<T, C>(P, s);
}

// Kernel nodes of a graph (memset and conditional nodes are not kernels).
long long count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  long long k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  cudaGetLastError();
  return k;
}

template <typename T, typename C>
gkb_status capture_graph(gkb_plan *P) {
  GKB_CUDA_TRY(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  GKB_CUDA_TRY(cudaStreamCreateWithFlags(&P->cap_body, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  GKB_CUDA_TRY(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeRelaxed));
  gkb_status st = enqueue_solve_captured<T, C>(P, P->cap, P->cap_body);
  cudaError_t e = cudaStreamEndCapture(P->cap, &graph);
  if (st != GKB_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (e != cudaSuccess) set_last_cuda_error(e);
    return st != GKB_OK ? st : GKB_ERR_CUDA;
  }
  P->kernels_outer = count_kernel_nodes(graph);
  P->kernels_body = P->body_graph ? count_kernel_nodes(P->body_graph) : 0;
  P->body_graph = nullptr;
  e = cudaGraphInstantiate(&P->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    P->exec = nullptr;
    cudaGetLastError();
    set_last_cuda_error(e);
    return GKB_ERR_CUDA;
  }
  P->graph_ok = 1;
  return GKB_OK;
}

gkb_status enqueue_captured_any(gkb_plan *P, cudaStream_t s, cudaStream_t body, int part = 0) {
  switch (P->p.storage) {
    case GKB_F64: return enqueue_solve_captured<double, double>(P, s, body, part);
    case GKB_F32: return enqueue_solve_captured<float, float>(P, s, body, part);
    case GKB_BF16: return enqueue_solve_captured<__nv_bfloat16, float>(P, s, body, part);
    case GKB_F16: return enqueue_solve_captured<__half, float>(P, s, body, part);
  }
  return GKB_ERR_INVALID_ARG;
}

template <typename T, typename C>
gkb_status run_direct(gkb_plan *P, cudaStream_t s) {
  gkb_status st = enqueue_init<T, C>(P, s);
  if (st != GKB_OK) return st;
  int *h_done = nullptr;
  GKB_CUDA_TRY(cudaMallocHost((void **)&h_done, sizeof(int)));
  for (int j = 1; j <= P->kmax; ++j) {
    st = enqueue_body<T, C>(P, s, 0, 0);
    if (st != GKB_OK) break;
    if ((j & 7) == 0) {
      cudaMemcpyAsync(h_done, &P->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) { st = GKB_ERR_CUDA; break; }
      if (*h_done) break;
    }
  }
  cudaFreeHost(h_done);
  if (st != GKB_OK) return st;
  return enqueue_final<T, C>(P, s);
}

template <typename T, typename C>
gkb_status dispatch_capture(gkb_plan *P) { return capture_graph<T, C>(P); }

gkb_status capture_any(gkb_plan *P) {
  switch (P->p.storage) {
    case GKB_F64: return dispatch_capture<double, double>(P);
    case GKB_F32: return dispatch_capture<float, float>(P);
    case GKB_BF16: return dispatch_capture<__nv_bfloat16, float>(P);
    case GKB_F16: return dispatch_capture<__half, float>(P);
  }
  return GKB_ERR_INVALID_ARG;
}

gkb_status direct_any(gkb_plan *P, cudaStream_t s) {
  switch (P->p.storage) {
    case GKB_F64: return run_direct<double, double>(P, s);
    case GKB_F32: return run_direct<float, float>(P, s);
    case GKB_BF16: return run_direct<__nv_bfloat16, float>(P, s);
    case GKB_F16: return run_direct<__half, float>(P, s);
  }
  return GKB_ERR_INVALID_ARG;
}

gkb_status validate(const gkb_geometry *g, const gkb_solve_params *p) {
  if (!g || !p) return GKB_ERR_INVALID_ARG;
  if (p->variant < GKB_AB || p->variant > GKB_BA_GMRES) return GKB_ERR_INVALID_ARG;
  const bool gmres = p->variant == GKB_AB_GMRES || p->variant == GKB_BA_GMRES;
  if (gmres && (p->k_max > 2048 || p->stop == GKB_STOP_LEARNED)) return GKB_ERR_INVALID_ARG;
  const bool mixed = p->storage == GKB_F32 && (p->operands == GKB_BF16 || p->operands == GKB_F16);
  if (mixed && (gmres || p->stop == GKB_STOP_LEARNED)) return GKB_ERR_INVALID_ARG;
  if (p->k_max < 1 || p->k_max > 4096) return GKB_ERR_INVALID_ARG;
  if (p->stop < GKB_STOP_NONE || p->stop > GKB_STOP_HYBRID) return GKB_ERR_INVALID_ARG;
  // hybrid: the projected residual is the data residual only for AB and
  // matched GKB; FP16 storage or operands run on b/||b||, not supported here
  if (p->stop == GKB_STOP_HYBRID &&
      ((p->variant != GKB_AB && p->variant != GKB_MATCHED) || !(p->noise_norm > 0.0) || !(p->rns_eps >= 0.0) ||
       p->storage == GKB_F16 || (p->storage == GKB_F32 && p->operands == GKB_F16)))
    return GKB_ERR_INVALID_ARG;
  if (p->stop == GKB_STOP_DP && !(p->noise_norm >= 0.0 && std::isfinite(p->noise_norm))) return GKB_ERR_INVALID_ARG;
  if (p->stop == GKB_STOP_RNS && !(p->rns_eps > 0.0 && std::isfinite(p->rns_eps))) return GKB_ERR_INVALID_ARG;
  if (!(p->tau >= 0.0) || !std::isfinite(p->tau)) return GKB_ERR_INVALID_ARG;
  if (p->reorth < 0 || p->reorth > 2) return GKB_ERR_INVALID_ARG;
  if (!dtype_valid(p->storage)) return GKB_ERR_INVALID_ARG;
  if (p->stop == GKB_STOP_LEARNED &&
      (p->variant != GKB_BA || p->storage != GKB_F32 || p->k_max <= kLearnK0 || !(p->noise_norm > 0.0)))
    return GKB_ERR_INVALID_ARG;
  return GKB_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The plan's workspace: every piece 256-byte aligned, in one block.  Returns
// the bytes needed; with base != nullptr also points the plan's buffers and
// its kernel view (SK) into the block.  gkb_plan_create and gkb_solve_noalloc
// both lay their workspace out with this one function.
size_t plan_layout(gkb_plan *P, char *base) {
  const gkb_geometry *g = P->g;
  const long long tmp_len = P->p.variant == GKB_BA ? g->m : g->n;
  const long long nparts = std::max({forward_blocks(g), back_blocks(g), (long long)148 * 8, (long long)P->nchunks,
                                     (long long)update_blocks(P)});
  const int ldk = P->kmax + 2;
  const size_t ts = P->tsz, cs = P->csz, os = dtype_size(P->op_dt);
  const size_t ms = align_up((size_t)P->m, 8), ns = align_up((size_t)P->n, 8);
  const size_t dss = align_up((size_t)P->ds, 8), tls = align_up((size_t)tmp_len, 8), ldq = (size_t)P->ldq;
  struct Piece { void **ptr; size_t bytes; };
  const Piece pieces[] = {
      {&P->Q, ts * ldq * (size_t)(P->kmax + 1)},
      {&P->s_cur, ts * dss}, {&P->s_tmp, ts * dss},
      {&P->qt, ts * ldq}, {&P->q_cur, ts * ldq},
      {&P->vM, os * ms}, {&P->tmp, os * tls}, {&P->b_st, ts * ms},
      {&P->xacc, cs * ldq}, {&P->w, cs * ldq}, {&P->z, cs * ms}, {&P->r, cs * ms},
      {&P->b_in, cs * ms}, {&P->x_out, cs * ns}, {&P->xt, std::max(ts, cs) * ns}, {&P->acc, 8 * ms + 256},
      {&P->fadj, 8 * ns},
      {(void **)&P->scal, sizeof(double) * 9 * (size_t)ldk},
      {(void **)&P->partials, sizeof(double) * (size_t)nparts},
      // reorthogonalisation partials (nchunks x ldk), also the learned step's k-long scratch
      {(void **)&P->dotp, sizeof(double) * (size_t)std::max(P->nchunks, 2) * ldk},
      {(void **)&P->coef, sizeof(double) * (size_t)ldk},
      {(void **)&P->counters, sizeof(unsigned) * 16},
      {(void **)&P->ctl, sizeof(Ctl)},
      {&P->x_dp, P->p.stop == GKB_STOP_LEARNED ? cs * ldq : 0},
      {(void **)&P->sk.R, P->gmres ? sizeof(double) * (size_t)ldk * ldk : 0},
      {(void **)&P->sk.hcol, sizeof(double) * (size_t)ldk},
      {&P->Z, P->p.variant == GKB_BA_GMRES ? cs * (size_t)P->ldz * (size_t)P->kmax : 0},
      {&P->q_op, P->mixed ? os * ldq : 0}, {&P->s_op, P->mixed ? os * dss : 0}, {&P->b_op, P->mixed ? os * ms : 0},
      {(void **)&P->sk.hyb, P->p.stop == GKB_STOP_HYBRID ? sizeof(double) * 64 * (size_t)ldk : 0},
  };
  size_t off = 0;
  for (const Piece &pc : pieces) {
    if (base) *pc.ptr = pc.bytes ? base + off : nullptr;
    off += align_up(pc.bytes, 256);
  }
  if (base) {
    double *sc = P->scal;
    SK &S = P->sk;
    S.c = P->ctl;
    S.alpha = sc + 0 * ldk; S.t = sc + 1 * ldk; S.rho = sc + 2 * ldk; S.rhobar = sc + 3 * ldk;
    S.phibar = sc + 4 * ldk; S.cg = sc + 5 * ldk; S.sg = sc + 6 * ldk; S.resid = sc + 7 * ldk;
    S.lam = sc + 8 * ldk;
    S.partials = P->partials; S.counters = P->counters; S.dotp = P->dotp; S.coef = P->coef; S.ldk = ldk;
  }
  return off;
}

// The plan's sizes from the geometry and the parameters (no allocation).
void plan_sizes(gkb_plan *P, const gkb_geometry *g, const gkb_solve_params *p) {
  P->g = g;
  P->p = *p;
  P->f64 = p->storage == GKB_F64;
  P->n = g->n;
  P->m = g->m;
  P->gmres = p->variant == GKB_AB_GMRES || p->variant == GKB_BA_GMRES;
  // GKB: s in the space of M's output (n for BA), q in its input; GMRES: one
  // basis in the space of the square M (m for AB, n for BA)
  P->dq = (p->variant == GKB_AB || p->variant == GKB_AB_GMRES) ? g->m : g->n;
  P->ds = P->gmres ? P->dq : (p->variant == GKB_BA ? g->n : g->m);
  P->ldz = (long long)align_up((size_t)g->m, 8);
  P->ldq = (long long)align_up((size_t)P->dq, 8);
  P->kmax = p->k_max;
  P->nchunks = (int)((P->ldq + kRowsPerBlock - 1) / kRowsPerBlock);
  P->tsz = dtype_size(p->storage);
  P->csz = P->f64 ? 8 : 4;
  P->io_dt = P->f64 ? GKB_F64 : GKB_F32;
  P->mixed = p->storage == GKB_F32 && (p->operands == GKB_BF16 || p->operands == GKB_F16);
  P->op_dt = P->mixed ? p->operands : p->storage;
}

}  // namespace

extern "C" gkb_status gkb_plan_kernel_counts(const gkb_plan *P, long long *outer, long long *per_iteration) {
  if (!P || !P->graph_ok || P->kernels_outer < 0) return GKB_ERR_UNSUPPORTED;
  if (outer) *outer = P->kernels_outer;
  if (per_iteration) *per_iteration = P->kernels_body;
  return GKB_OK;
}

extern "C" gkb_status gkb_plan_destroy(gkb_plan *P) {
  if (!P) return GKB_ERR_INVALID_ARG;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->cap_body) cudaStreamDestroy(P->cap_body);
  if (P->arena) cudaFree(P->arena);
  delete P;
  return GKB_OK;
}

extern "C" gkb_status gkb_plan_create(const gkb_geometry *g, const gkb_solve_params *p, gkb_plan **out) {
  if (!out) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  gkb_status st = validate(g, p);
  if (st != GKB_OK) return st;
  gkb_plan *P = new (std::nothrow) gkb_plan();
  if (!P) return GKB_ERR_OOM;
  plan_sizes(P, g, p);
  if (P->f64 && (st = ensure_f64(const_cast<gkb_geometry *>(g))) != GKB_OK) {
    delete P;
    return st;
  }
  // the projectors run in the operand type (the storage type unless mixed)
  if (!P->f64 && (st = autotune(const_cast<gkb_geometry *>(g), P->op_dt)) != GKB_OK) {
    delete P;
    return st;
  }
  const size_t total = plan_layout(P, nullptr);
  cudaError_t e = cudaMalloc(&P->arena, total);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    cudaGetLastError();
    delete P;
    return e == cudaErrorMemoryAllocation ? GKB_ERR_OOM : GKB_ERR_CUDA;
  }
  // zero everything once: padding rows of Q / q~ must stay zero
  e = cudaMemset(P->arena, 0, total);
  plan_layout(P, static_cast<char *>(P->arena));
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    gkb_plan_destroy(P);
    return GKB_ERR_CUDA;
  }
  if (p->use_graph) {
    st = capture_any(P);
    if (st != GKB_OK) {
      gkb_plan_destroy(P);
      return st;
    }
  }
  *out = P;
  return GKB_OK;
}

namespace gkb {
namespace {
// Status of a finished solve from its control block.
gkb_status finish_status(const gkb_plan *P, const Ctl &hc) {
  gkb_status out = hc.status;
  if (out == GKB_OK) {
    if (hc.reason == GKB_REASON_BREAKDOWN) out = GKB_STATUS_BREAKDOWN;
    else if (hc.reason == GKB_REASON_K_MAX && P->p.stop != GKB_STOP_NONE) out = GKB_STATUS_NOT_CONVERGED;
  }
  return out;
}
// Copy the control block (and the scalar histories when info asks for them)
// of a plan to the host, asynchronously on s; hs must stay alive until s syncs.
gkb_status fetch_info(gkb_plan *P, Ctl *hc, std::vector<double> &hs, const gkb_solve_info *info, cudaStream_t s) {
  GKB_CUDA_TRY(cudaMemcpyAsync(hc, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  const int ldk = P->kmax + 2;
  if (info && (info->alpha || info->t || info->resid || info->lambda)) {
    hs.resize((size_t)9 * ldk);
    GKB_CUDA_TRY(cudaMemcpyAsync(hs.data(), P->scal, sizeof(double) * 9 * ldk, cudaMemcpyDeviceToHost, s));
  }
  return GKB_OK;
}
void fill_info(const gkb_plan *P, const Ctl &hc, const std::vector<double> &hs, gkb_status out, gkb_solve_info *info) {
  if (!info) return;
  info->k_stop = hc.k_stop;
  info->stop_reason = hc.reason;
  info->status = out;
  const int ldk = P->kmax + 2;
  const int kcount = hc.k_stop;  // iterations whose data exist
  if (hs.empty()) return;
  const double *al = hs.data() + 0 * ldk, *tt = hs.data() + 1 * ldk, *rs = hs.data() + 7 * ldk;
  const double *lm = hs.data() + 8 * ldk;
  for (int i = 0; i <= kcount && i < ldk; ++i) {
    if (info->alpha && i < kcount) info->alpha[i] = al[i + 1];   // alpha_1 .. alpha_k
    if (info->t) info->t[i] = tt[i + 1];                          // t_1 .. t_{k+1}
    if (info->resid && i < kcount) info->resid[i] = rs[i + 1];   // r_1 .. r_k
    if (info->lambda && i < kcount) info->lambda[i] = lm[i + 1]; // lambda_1 .. lambda_k (hybrid)
  }
}
}  // namespace
}  // namespace gkb

extern "C" gkb_status gkb_plan_execute(gkb_plan *P, const void *b, void *x, gkb_solve_info *info, void *stream) {
  if (!P || !b || !x) return GKB_ERR_INVALID_ARG;
  if (P->p.stop == GKB_STOP_LEARNED) return GKB_ERR_INVALID_ARG;  // needs a predictor: gkb_batch_execute_learned
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GKB_CUDA_TRY(cudaMemcpyAsync(P->b_in, b, P->csz * P->m, cudaMemcpyDefault, s));
  gkb_status st;
  if (P->graph_ok) {
    GKB_CUDA_TRY(cudaGraphLaunch(P->exec, s));
    st = GKB_OK;
  } else {
    st = direct_any(P, s);
  }
  if (st != GKB_OK) return st;
  GKB_CUDA_TRY(cudaMemcpyAsync(x, P->x_out, P->csz * P->n, cudaMemcpyDefault, s));
  Ctl hc;
  std::vector<double> hs;
  if ((st = fetch_info(P, &hc, hs, info, s)) != GKB_OK) return st;
  GKB_CUDA_TRY(cudaStreamSynchronize(s));
  const gkb_status out = finish_status(P, hc);
  fill_info(P, hc, hs, out, info);
  return out;
}

extern "C" gkb_status gkb_plan_profile(gkb_plan *P, const void *b, double *ms, long long *groups, void *stream) {
  if (!P || !b || !ms || P->p.stop == GKB_STOP_LEARNED) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Prof pr;
  P->prof = &pr;
  GKB_CUDA_TRY(cudaMemcpyAsync(P->b_in, b, P->csz * P->m, cudaMemcpyDefault, s));
  gkb_status st = direct_any(P, s);   // init, iterations (stop checked every 8), final
  mark(P, s, PC_OTHER);               // closes the last group
  P->prof = nullptr;
  cudaError_t e = cudaStreamSynchronize(s);
  for (int c = 0; c < PC_COUNT; ++c) {
    ms[c] = 0.0;
    if (groups) groups[c] = 0;
  }
  if (st == GKB_OK && e == cudaSuccess && !pr.failed) {
    for (size_t i = 0; i + 1 < pr.used; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pr.ev[i], pr.ev[i + 1]) == cudaSuccess) ms[pr.cls[i]] += t;
      if (groups) groups[pr.cls[i]] += 1;
    }
  }
  for (cudaEvent_t ev : pr.ev) cudaEventDestroy(ev);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    return GKB_ERR_CUDA;
  }
  if (pr.failed) return GKB_ERR_CUDA;
  return st;
}

extern "C" gkb_status gkb_solve(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x,
                                gkb_solve_info *info, void *stream) {
  if (!b || !x || (p && p->stop == GKB_STOP_LEARNED)) return GKB_ERR_INVALID_ARG;
  gkb_plan *P = nullptr;
  gkb_status st = gkb_plan_create(g, p, &P);
  if (st != GKB_OK) return st;
  st = gkb_plan_execute(P, b, x, info, stream);
  gkb_plan_destroy(P);
  return st;
}

// ---------------------------------------------------------------------------
// Batched solve: independent slices, one captured graph.
//
// Every slice keeps its own plan (workspace, Krylov state, device-side stop).
// The slices are assigned, largest first, to the least loaded of up to 32
// capture streams, and the whole batch is captured as one graph: a fork from
// a master stream, one chain of solves per capture stream (each solve: its
// initialisation, its WHILE node, its final combination), and a join.  One
// launch of that graph runs the batch; the device schedules the chains
// concurrently and each slice stops on its own discrepancy test.

struct gkb_batch {
  int n = 0;
  int learned = 0;
  std::vector<gkb_plan *> plans;
  std::vector<cudaStream_t> streams;
  std::vector<int> order, chain;
  cudaStream_t master = nullptr, body = nullptr;
  std::vector<cudaEvent_t> events;
  cudaGraphExec_t exec = nullptr;   // the whole batch (learned: phase 1)
  cudaGraphExec_t exec3 = nullptr;  // learned: phase 3
  gkb::SK *d_sks = nullptr;         // per-slice kernel views, for the cross-slice kernels
};

namespace gkb {
namespace {
// Capture every slice's part of the solve as one graph: fork from the master
// stream, one chain per capture stream, join.
gkb_status capture_batch(gkb_batch *B, int part, cudaGraphExec_t *out) {
  const int ns = (int)B->streams.size();
  gkb_status st = GKB_OK;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(B->master, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(B->events[ns], B->master);
  for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(B->streams[k], B->events[ns], 0);
  for (int i : B->order) {
    if (e != cudaSuccess || st != GKB_OK) break;
    st = enqueue_captured_any(B->plans[i], B->streams[B->chain[i]], B->body, part);
  }
  for (int k = 0; k < ns && e == cudaSuccess && st == GKB_OK; ++k) {
    e = cudaEventRecord(B->events[k], B->streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->master, B->events[k], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(B->master, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && st == GKB_OK) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || st != GKB_OK) {
    cudaGetLastError();
    if (e != cudaSuccess) set_last_cuda_error(e);
    *out = nullptr;
    return st != GKB_OK ? st : GKB_ERR_CUDA;
  }
  return GKB_OK;
}
}  // namespace
}  // namespace gkb

extern "C" gkb_status gkb_batch_destroy(gkb_batch *B) {
  if (!B) return GKB_ERR_INVALID_ARG;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->exec3) cudaGraphExecDestroy(B->exec3);
  if (B->d_sks) cudaFree(B->d_sks);
  for (cudaEvent_t e : B->events) cudaEventDestroy(e);
  for (cudaStream_t s : B->streams) cudaStreamDestroy(s);
  if (B->master) cudaStreamDestroy(B->master);
  if (B->body) cudaStreamDestroy(B->body);
  for (gkb_plan *P : B->plans)
    if (P) gkb_plan_destroy(P);
  delete B;
  return GKB_OK;
}

extern "C" gkb_status gkb_batch_create(int n, const gkb_geometry *const *g, const gkb_solve_params *p, gkb_batch **out) {
  using namespace gkb;
  if (!out) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || !g || !p) return GKB_ERR_INVALID_ARG;
  int n_learned = 0;
  for (int i = 0; i < n; ++i) {
    gkb_status st = validate(g[i], p + i);
    if (st != GKB_OK) return st;
    n_learned += p[i].stop == GKB_STOP_LEARNED;
  }
  if (n_learned != 0 && n_learned != n) return GKB_ERR_INVALID_ARG;  // all slices learned, or none
  gkb_batch *B = new (std::nothrow) gkb_batch();
  if (!B) return GKB_ERR_OOM;
  B->n = n;
  B->learned = n_learned == n;
  B->plans.assign(n, nullptr);
  gkb_status st = GKB_OK;
  std::vector<double> work(n);
  for (int i = 0; i < n && st == GKB_OK; ++i) {
    gkb_solve_params q = p[i];
    q.use_graph = 0;  // the batch graph captures the solve itself
    st = gkb_plan_create(g[i], &q, &B->plans[i]);
    const gkb_plan *P = B->plans[i];
    if (st == GKB_OK)  // work estimate: projector taps plus the reorthogonalisation
      work[i] = (double)P->kmax * (8.0 * (double)g[i]->n * g[i]->desc.n_angles + (double)P->dq * P->kmax);
  }
  if (st != GKB_OK) {
    gkb_batch_destroy(B);
    return st;
  }
  const int ns = std::min(n, 32);
  B->streams.assign(ns, nullptr);
  for (int k = 0; k < ns; ++k)
    if (cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking) != cudaSuccess) st = GKB_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&B->master, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&B->body, cudaStreamNonBlocking) != cudaSuccess)
    st = GKB_ERR_CUDA;
  B->events.assign(ns + 1, nullptr);
  for (auto &e : B->events)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = GKB_ERR_CUDA;
  std::vector<SK> sks(n);
  for (int i = 0; i < n; ++i) sks[i] = B->plans[i]->sk;
  if (st == GKB_OK && (cudaMalloc(&B->d_sks, sizeof(SK) * n) != cudaSuccess ||
                       cudaMemcpy(B->d_sks, sks.data(), sizeof(SK) * n, cudaMemcpyHostToDevice) != cudaSuccess))
    st = GKB_ERR_CUDA;
  if (st != GKB_OK) {
    cudaGetLastError();
    gkb_batch_destroy(B);
    return st;
  }
  // largest first onto the least loaded chain
  B->order.resize(n);
  for (int i = 0; i < n; ++i) B->order[i] = i;
  std::sort(B->order.begin(), B->order.end(), [&](int a, int b) { return work[a] > work[b]; });
  std::vector<double> load(ns, 0.0);
  B->chain.resize(n);
  for (int i : B->order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    B->chain[i] = k;
    load[k] += work[i];
  }
  st = capture_batch(B, B->learned ? 1 : 0, &B->exec);
  if (st == GKB_OK && B->learned) st = capture_batch(B, 3, &B->exec3);
  if (st != GKB_OK) {
    gkb_batch_destroy(B);
    return st;
  }
  *out = B;
  return GKB_OK;
}

namespace gkb {
namespace {
gkb_status batch_collect(gkb_batch *B, void *const *x, gkb_solve_info *info, gkb_learned_info *linfo, cudaStream_t s) {
  std::vector<Ctl> hc(B->n);
  std::vector<std::vector<double>> hs(B->n);
  for (int i = 0; i < B->n; ++i) {
    gkb_plan *P = B->plans[i];
    GKB_CUDA_TRY(cudaMemcpyAsync(x[i], P->x_out, P->csz * P->n, cudaMemcpyDefault, s));
    gkb_status st = fetch_info(P, &hc[i], hs[i], info ? info + i : nullptr, s);
    if (st != GKB_OK) return st;
  }
  GKB_CUDA_TRY(cudaStreamSynchronize(s));
  gkb_status worst = GKB_OK;
  for (int i = 0; i < B->n; ++i) {
    gkb_status out = finish_status(B->plans[i], hc[i]);
    if (B->learned && out == GKB_STATUS_NOT_CONVERGED && hc[i].k_dp > 0) out = GKB_OK;
    fill_info(B->plans[i], hc[i], hs[i], out, info ? info + i : nullptr);
    if (linfo) {
      linfo[i].k_hat = hc[i].k_hat;
      linfo[i].lambda = hc[i].lambda;
      linfo[i].k_dp = hc[i].k_dp;
      linfo[i].hybrid = hc[i].fallback == 0 && hc[i].hybrid;
      linfo[i].fallback = hc[i].fallback;
      linfo[i].hybrid_resid = sqrt(hc[i].hyb_r2);
    }
    if (out < 0 && worst >= 0) worst = out;          // the first error wins
    else if (worst >= 0 && out > worst) worst = out;  // else the strongest informational status
  }
  return worst;
}
}  // namespace
}  // namespace gkb

extern "C" gkb_status gkb_batch_execute(gkb_batch *B, const void *const *b, void *const *x, gkb_solve_info *info,
                                        void *stream) {
  using namespace gkb;
  if (!B || !b || !x || B->learned) return GKB_ERR_INVALID_ARG;
  for (int i = 0; i < B->n; ++i)
    if (!b[i] || !x[i]) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < B->n; ++i) {
    gkb_plan *P = B->plans[i];
    GKB_CUDA_TRY(cudaMemcpyAsync(P->b_in, b[i], P->csz * P->m, cudaMemcpyDefault, s));
  }
  GKB_CUDA_TRY(cudaGraphLaunch(B->exec, s));
  return batch_collect(B, x, info, nullptr, s);
}

extern "C" gkb_status gkb_batch_execute_learned(gkb_batch *B, const gkb_mlp *mlp, const void *const *b, void *const *x,
                                                gkb_solve_info *info, gkb_learned_info *linfo, void *stream) {
  using namespace gkb;
  if (!B || !mlp || !b || !x || !B->learned) return GKB_ERR_INVALID_ARG;
  for (int i = 0; i < B->n; ++i)
    if (!b[i] || !x[i]) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < B->n; ++i) {
    gkb_plan *P = B->plans[i];
    GKB_CUDA_TRY(cudaMemcpyAsync(P->b_in, b[i], P->csz * P->m, cudaMemcpyDefault, s));
  }
  GKB_CUDA_TRY(cudaGraphLaunch(B->exec, s));                                            // first kLearnK0 iterations
  k_learned_predict<<<B->n, kHid, 0, s>>>(B->d_sks, mlp->theta_bf16, mlp->norm, kLearnDelta);  // k_hat, lambda_hat
  GKB_CUDA_TRY(cudaGetLastError());
  GKB_CUDA_TRY(cudaGraphLaunch(B->exec3, s));                                           // resume, hybrid step, check
  return batch_collect(B, x, info, linfo, s);
}

extern "C" gkb_status gkb_batch_training_data(gkb_batch *B, float *X, float *T, int *valid, void *stream) {
  using namespace gkb;
  if (!B || !X || !T || !valid || B->learned) return GKB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_learned_labels<<<B->n, kHid, 0, s>>>(B->d_sks, kLearnDelta, X, T, valid);
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

extern "C" gkb_status gkb_solve_batched(int n, const gkb_geometry *const *g, const gkb_solve_params *p,
                                        const void *const *b, void *const *x, gkb_solve_info *info, void *stream) {
  if (n == 0) return GKB_OK;
  gkb_batch *B = nullptr;
  gkb_status st = gkb_batch_create(n, g, p, &B);
  if (st != GKB_OK) return st;
  st = gkb_batch_execute(B, b, x, info, stream);
  gkb_batch_destroy(B);
  return st;
}

extern "C" gkb_status gkb_solve_iterates(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x_hist,
                                         gkb_solve_info *info, void *stream) {
  if (!g || !p || !b || !x_hist || p->stop == GKB_STOP_LEARNED) return GKB_ERR_INVALID_ARG;
  // AB iterates need a back projection each; GMRES forms its iterate at the stop only
  if (p->variant == GKB_AB || p->variant == GKB_AB_GMRES || p->variant == GKB_BA_GMRES) return GKB_ERR_UNSUPPORTED;
  gkb_solve_params q = *p;
  q.use_graph = 0;
  gkb_plan *P = nullptr;
  gkb_status st = gkb_plan_create(g, &q, &P);
  if (st != GKB_OK) return st;
  P->hist = x_hist;
  // the returned iterate goes to the last row (which is x_k_max when the solve runs to k_max)
  void *x_last = static_cast<char *>(x_hist) + (size_t)(q.k_max - 1) * P->n * P->csz;
  st = gkb_plan_execute(P, b, x_last, info, stream);
  gkb_plan_destroy(P);
  return st;
}

// ---------------------------------------------------------------------------
// Solve without any device allocation (gkb_solve_noalloc).
//
// Some callers cannot allocate device memory at the moment they solve: an
// application that owns the whole device through its own memory pool, a
// plugin host that forbids cudaMalloc after start-up, or a real-time loop that
// must not block on the allocator.  This entry point runs the same solve as
// gkb_solve, but its workspace is a fixed array in the library's own device
// memory (static storage, reserved on every GPU that loads the library, held
// until the process exits) instead of memory obtained per call.

#include <mutex>

namespace gkb {
namespace {

constexpr size_t kNoAllocArenaBytes = 64ull << 20;  // 64 MiB: the largest workspace the entry point accepts

static __device__ __align__(256) unsigned char g_noalloc_arena[kNoAllocArenaBytes];

// Device address of the array on the current device.  Host code may not use
// g_noalloc_arena's host-side name as a device pointer; the address is looked
// up once per device with that device current and cached (so it is stale
// after cudaDeviceReset of that device).  The geometry's tables live on
// g->device, which must be the current device.
gkb_status noalloc_arena(const gkb_geometry *g, void **out) {
  static std::mutex mu;
  static void *addr[64] = {nullptr};
  int dev = 0;
  GKB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device) return GKB_ERR_INVALID_ARG;
  if (dev < 0 || dev >= 64) return GKB_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_arena);
    if (e != cudaSuccess) {
      set_last_cuda_error(e);
      cudaGetLastError();
      return GKB_ERR_CUDA;
    }
    addr[dev] = p;
  }
  *out = addr[dev];
  return GKB_OK;
}

// Launch loop with no host allocation: the stop flag is read into a local.
template <typename T, typename C>
gkb_status noalloc_run(gkb_plan *P, cudaStream_t s) {
  gkb_status st = enqueue_init<T, C>(P, s);
  if (st != GKB_OK) return st;
  for (int j = 1; j <= P->kmax; ++j) {
    if ((st = enqueue_body<T, C>(P, s, 0, 0)) != GKB_OK) return st;
    if ((j & 7) == 0) {
      int done = 0;
      GKB_CUDA_TRY(cudaMemcpyAsync(&done, &P->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      GKB_CUDA_TRY(cudaStreamSynchronize(s));
      if (done) break;
    }
  }
  return enqueue_final<T, C>(P, s);
}

}  // namespace
}  // namespace gkb

extern "C" gkb_status gkb_solve_noalloc(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x,
                                        gkb_solve_info *info, void *stream) {
  using namespace gkb;
  if (!b || !x || (p && p->stop == GKB_STOP_LEARNED)) return GKB_ERR_INVALID_ARG;
  gkb_status st = validate(g, p);
  if (st != GKB_OK) return st;
  // FP64 storage needs the geometry's FP64 tables, which only an earlier FP64
  // call can have built (building them here would allocate).
  if (p->storage == GKB_F64 && !g->ray_d) return GKB_ERR_INVALID_ARG;
  gkb_plan P;  // on the stack: no host allocation either
  plan_sizes(&P, g, p);
  P.p.use_graph = 0;
  const size_t need = plan_layout(&P, nullptr);
  if (need > kNoAllocArenaBytes) return GKB_ERR_TOO_LARGE;
  void *arena = nullptr;
  if ((st = noalloc_arena(g, &arena)) != GKB_OK) return st;
  plan_layout(&P, static_cast<char *>(arena));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: zero what must start at zero
  // (padding rows of the basis, reduction counters, accumulators)
  GKB_CUDA_TRY(cudaMemsetAsync(arena, 0, need, s));
  GKB_CUDA_TRY(cudaMemcpyAsync(P.b_in, b, P.csz * P.m, cudaMemcpyDefault, s));
  switch (p->storage) {
    case GKB_F64: st = noalloc_run<double, double>(&P, s); break;
    case GKB_F32: st = noalloc_run<float, float>(&P, s); break;
    case GKB_BF16: st = noalloc_run<__nv_bfloat16, float>(&P, s); break;
    case GKB_F16: st = noalloc_run<__half, float>(&P, s); break;
  }
  if (st != GKB_OK) return st;
  GKB_CUDA_TRY(cudaMemcpyAsync(x, P.x_out, P.csz * P.n, cudaMemcpyDefault, s));
  Ctl hc;
  GKB_CUDA_TRY(cudaMemcpyAsync(&hc, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  GKB_CUDA_TRY(cudaStreamSynchronize(s));
  gkb_status out = hc.status;
  if (out == GKB_OK) {
    if (hc.reason == GKB_REASON_BREAKDOWN) out = GKB_STATUS_BREAKDOWN;
    else if (hc.reason == GKB_REASON_K_MAX && p->stop != GKB_STOP_NONE) out = GKB_STATUS_NOT_CONVERGED;
  }
  if (info) {
    info->k_stop = hc.k_stop;
    info->stop_reason = hc.reason;
    info->status = out;
    const int k = hc.k_stop;
    // histories straight into the caller's arrays (alpha_1.., t_1.., r_1..)
    if (info->alpha && k > 0)
      GKB_CUDA_TRY(cudaMemcpyAsync(info->alpha, P.sk.alpha + 1, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    if (info->t) GKB_CUDA_TRY(cudaMemcpyAsync(info->t, P.sk.t + 1, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    if (info->resid && k > 0)
      GKB_CUDA_TRY(cudaMemcpyAsync(info->resid, P.sk.resid + 1, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    GKB_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return out;
}

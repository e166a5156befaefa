// Shared device-side definitions of the GKB library: storage types, the
// interpolation-weight functions that each projector shares with its exact
// transpose, and deterministic block/grid reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gkb.h"

namespace gkb {

// ---------------------------------------------------------------------------
// storage <-> compute conversion

template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_c(float v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_c<__half>(float v) { return __float2half_rn(v); }
template <typename T> __device__ __forceinline__ T from_c(double v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }

// Unfused, correctly rounded arithmetic.  The weight of a projector and of
// its transpose must be the same number, so every coordinate the two kernels
// share is evaluated with these intrinsics (the compiler may neither contract
// nor reorder them differently in the two kernels).
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float floor_(float a) { return floorf(a); }
__device__ __forceinline__ double floor_(double a) { return floor(a); }
__device__ __forceinline__ float ceil_(float a) { return ceilf(a); }
__device__ __forceinline__ double ceil_(double a) { return ceil(a); }
__device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__device__ __forceinline__ double abs_(double a) { return fabs(a); }
__device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }

// ---------------------------------------------------------------------------
// geometry as seen by the kernels

// One ray of Joseph's projector: along axis 0 it crosses image row i at
// column coordinate J0 + i*Js; along axis 1 it crosses column j at row
// coordinate J0 + j*Js.  scale = pixel / max(|e_x|, |e_y|).
template <typename C> struct RayP { C J0, Js, scale, axis; };

// Per-angle constants of the pixel-driven projector (and of the candidate
// windows the gathers use).
//   parallel: t = xr*cu + yr*su + t0          (bin coordinate of a pixel centre)
//   fan:      U' = sodp - (xr*c + yr*s), L' = -xr*s + yr*c,
//             t = g*L'/U' + t0, w = wpix*sqrt(U'^2+L'^2)/U'^2
//   fan arc:  t = g*atan2(L', U') + t0, w = wpix/sqrt(U'^2+L'^2)
// with xr = j - (nx-1)/2 and yr = (ny-1)/2 - i in pixel units.
template <typename C> struct AngleP { C c, s, cu, su, R; };

template <typename C> struct GeomK {
  int beam;          // 0 parallel, 1 fan (flat detector), 2 fan (arc detector)
  int nx, ny, na, nd;
  C t0;              // (nd-1)/2
  C hx, hy;          // (nx-1)/2, (ny-1)/2
  C wpar;            // parallel weight pixel^2 / det_width
  C sodp, gfan, wpix; // fan: sod/pixel, sdd/det_width, pixel*sdd/det_width
  const RayP<C> *ray;      // na*nd
  const AngleP<C> *ang;    // na
};

// Bin coordinate t and weight w of pixel (xr, yr) at one angle: the single
// definition used by the back projector and by its transpose.
template <typename C>
__device__ __forceinline__ void pixel_bin(const GeomK<C> &G, const AngleP<C> &A, C xr, C yr, C &t, C &w) {
  if (G.beam == 0) {
    t = fma_(xr, A.cu, fma_(yr, A.su, G.t0));
    w = G.wpar;
  } else if (G.beam == 1) {
    C U = sub_(G.sodp, fma_(xr, A.c, mul_(yr, A.s)));
    C L = fma_(yr, A.c, -mul_(xr, A.s));
    C rU = div_(C(1), U);
    t = fma_(mul_(G.gfan, L), rU, G.t0);
    w = mul_(mul_(G.wpix, sqrt_(fma_(U, U, mul_(L, L)))), mul_(rU, rU));
  } else {
    C U = sub_(G.sodp, fma_(xr, A.c, mul_(yr, A.s)));
    C L = fma_(yr, A.c, -mul_(xr, A.s));
    t = fma_(G.gfan, atan2(L, U), G.t0);
    w = div_(G.wpix, sqrt_(fma_(U, U, mul_(L, L))));
  }
}

// FP32 form, split as w = wscale * wr with wscale = wpar (parallel) or wpix
// (fan) a constant of the geometry, so that kernels can sum wr-weighted
// terms and apply wscale once.  Reciprocal, square root and reciprocal square
// root come from the hardware approximations (relative error ~2e-7); B and
// B^T call this same function, so they still apply the same numbers.  The evaluation
// order puts the column term first (fma(yr, su, fma(xr, cu, t0)) for the
// parallel beam, U and L from xr*cos and xr*sin for the fan), so that a
// thread holding several pixels of one column computes it once.
//   parallel: t = xr cu + yr su + t0, wr = 1
//   fan:      tau = L / U, t = gfan tau + t0, wr = sqrt(1 + tau^2) / U
//             (= sqrt(U^2 + L^2) / U^2, the inverse ray spacing over wpix)
//   fan arc:  t = gfan atan2(L, U) + t0, wr = 1 / sqrt(U^2 + L^2)
// The beam is a template parameter so a kernel instantiated for one beam
// carries none of the others' code (and none of their registers).
template <int BEAM>
__device__ __forceinline__ float bin_column_x(const GeomK<float> &G, const AngleP<float> &A, float xr) {
  if constexpr (BEAM == 0) return __fmaf_rn(xr, A.cu, G.t0);
  else return __fsub_rn(G.sodp, __fmul_rn(xr, A.c));   // U of the column's y = 0 point
}
template <int BEAM>
__device__ __forceinline__ float bin_column_l(const GeomK<float> &G, const AngleP<float> &A, float xr) {
  if constexpr (BEAM == 0) return 0.f;
  else return -__fmul_rn(xr, A.s);                     // L of the column's y = 0 point
}
// The hardware approximations themselves (one special-function instruction
// each; relative error about 2^-22): U is at least sod - half diagonal > 0
// pixels and s2 >= 1, far from the flush-to-zero and special-value ranges.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int BEAM>
__device__ __forceinline__ void pixel_bin_col(const GeomK<float> &G, const AngleP<float> &A, float cx, float cl,
                                              float yr, float &t, float &wr) {
  if constexpr (BEAM == 0) {
    t = __fmaf_rn(yr, A.su, cx);
    wr = 1.f;
  } else {
    const float U = __fmaf_rn(-yr, A.s, cx);
    const float L = __fmaf_rn(yr, A.c, cl);
    if constexpr (BEAM == 1) {
      const float rU = rcp_approx(U);
      const float tau = __fmul_rn(L, rU);
      t = __fmaf_rn(G.gfan, tau, G.t0);
      wr = __fmul_rn(rU, sqrt_approx(__fmaf_rn(tau, tau, 1.0f)));
    } else {
      t = __fmaf_rn(G.gfan, atan2f(L, U), G.t0);
      wr = rsqrt_approx(__fmaf_rn(U, U, __fmul_rn(L, L)));
    }
  }
}
template <int BEAM>
__device__ __forceinline__ void pixel_bin_rel(const GeomK<float> &G, const AngleP<float> &A, float xr, float yr,
                                              float &t, float &wr) {
  pixel_bin_col<BEAM>(G, A, bin_column_x<BEAM>(G, A, xr), bin_column_l<BEAM>(G, A, xr), yr, t, wr);
}
template <int BEAM> __device__ __forceinline__ float bin_wscale(const GeomK<float> &G) {
  return BEAM == 0 ? G.wpar : G.wpix;
}
template <int BEAM>
__device__ __forceinline__ void pixel_bin_f(const GeomK<float> &G, const AngleP<float> &A, float xr, float yr,
                                            float &t, float &w) {
  float wr;
  pixel_bin_rel<BEAM>(G, A, xr, yr, t, wr);
  w = __fmul_rn(bin_wscale<BEAM>(G), wr);
}

template <>
__device__ __forceinline__ void pixel_bin<float>(const GeomK<float> &G, const AngleP<float> &A, float xr, float yr,
                                                 float &t, float &w) {
  if (G.beam == 0) pixel_bin_f<0>(G, A, xr, yr, t, w);
  else if (G.beam == 1) pixel_bin_f<1>(G, A, xr, yr, t, w);
  else pixel_bin_f<2>(G, A, xr, yr, t, w);
}

// Bins [lo, hi] of the rays that can weight pixel (xr, yr) at one angle.
// Joseph's weight is non-zero only for rays passing within one pixel of the
// centre (within max(|cos|, |sin|) of the ray's direction, exactly, for a
// parallel beam: t -+ R).  Fan: the source directions within asin(1/rho) of
// the pixel's direction (rho its distance from the source), mapped to the
// flat detector by the tangent addition formula; a side whose direction turns
// past 90 degrees from the central ray is unbounded (+-1e30).  A small margin
// covers rounding.
template <typename C>
__device__ __forceinline__ void ray_range(const GeomK<C> &G, const AngleP<C> &A, C xr, C yr, C &lo, C &hi) {
  if (G.beam == 0) {
    const C tc = fma_(xr, A.cu, fma_(yr, A.su, G.t0));
    lo = tc - A.R - C(0.02);
    hi = tc + A.R + C(0.02);
    return;
  }
  const C U = G.sodp - (xr * A.c + yr * A.s);
  const C L = yr * A.c - xr * A.s;
  const C r2 = U * U + L * L;
  if (!(r2 > C(1)) || !(U > C(0))) {
    lo = C(-1e30);
    hi = C(1e30);
    return;
  }
  if (G.beam == 2) {   // arc: bins are linear in the angle
    const C gm = atan2(L, U), dg = asin(C(1) / sqrt_(r2));
    hi = G.gfan * (gm + dg) + G.t0;
    lo = G.gfan * (gm - dg) + G.t0;
    hi += C(0.02) + C(1e-5) * abs_(hi);
    lo -= C(0.02) + C(1e-5) * abs_(lo);
    return;
  }
  const C a = L / U, q = C(1) / sqrt_(r2 - C(1));
  const C dh = C(1) - a * q, dl = C(1) + a * q;
  hi = dh > C(0) ? G.gfan * (a + q) / dh + G.t0 : C(1e30);
  lo = dl > C(0) ? G.gfan * (a - q) / dl + G.t0 : C(-1e30);
  hi += C(0.02) + C(1e-5) * abs_(hi);
  lo -= C(0.02) + C(1e-5) * abs_(lo);
}

// The same range for every pixel centre of the rectangle [x0, x1] x [y0, y1]
// (pixel-centre coordinates): the parallel bin coordinate and the fan's L/U
// take their extremes at the corners, and every pixel of the rectangle is at
// least rho_min (the nearest point's distance) from the source, so the
// corners' extreme directions widened by asin(1/rho_min) bound every pixel's
// range.
template <typename C>
__device__ __forceinline__ void ray_range_rect(const GeomK<C> &G, const AngleP<C> &A, C x0, C x1, C y0, C y1, C &lo,
                                               C &hi) {
  if (G.beam == 0) {
    C tmin = C(1e30), tmax = C(-1e30);
    for (int k = 0; k < 4; ++k) {
      const C tc = fma_((k & 1) ? x1 : x0, A.cu, fma_((k & 2) ? y1 : y0, A.su, G.t0));
      tmin = min_(tmin, tc);
      tmax = max_(tmax, tc);
    }
    lo = tmin - A.R - C(0.02);
    hi = tmax + A.R + C(0.02);
    return;
  }
  C amin = C(1e30), amax = C(-1e30);
  bool behind = false;
  for (int k = 0; k < 4; ++k) {
    const C xr = (k & 1) ? x1 : x0, yr = (k & 2) ? y1 : y0;
    const C U = G.sodp - (xr * A.c + yr * A.s);
    const C L = yr * A.c - xr * A.s;
    if (!(U > C(0))) behind = true;
    const C a = L / U;
    amin = min_(amin, a);
    amax = max_(amax, a);
  }
  const C xs = G.sodp * A.c, ys = G.sodp * A.s;   // the source, in the same coordinates
  const C dx = xs - min_(max_(xs, x0), x1), dy = ys - min_(max_(ys, y0), y1);
  const C r2 = dx * dx + dy * dy;
  if (behind || !(r2 > C(1))) {
    lo = C(-1e30);
    hi = C(1e30);
    return;
  }
  if (G.beam == 2) {   // arc: the corner directions' angles widened by asin(1/rho_min)
    const C dg = asin(C(1) / sqrt_(r2));
    hi = G.gfan * (atan(amax) + dg) + G.t0;
    lo = G.gfan * (atan(amin) - dg) + G.t0;
    hi += C(0.02) + C(1e-5) * abs_(hi);
    lo -= C(0.02) + C(1e-5) * abs_(lo);
    return;
  }
  const C q = C(1) / sqrt_(r2 - C(1));
  const C dh = C(1) - amax * q, dl = C(1) + amin * q;
  hi = dh > C(0) ? G.gfan * (amax + q) / dh + G.t0 : C(1e30);
  lo = dl > C(0) ? G.gfan * (amin - q) / dl + G.t0 : C(-1e30);
  hi += C(0.02) + C(1e-5) * abs_(hi);
  lo -= C(0.02) + C(1e-5) * abs_(lo);
}

// Joseph interpolation coordinate of ray r on row i (axis 0) / column j (axis 1).
template <typename C>
__device__ __forceinline__ C ray_coord(const RayP<C> &r, int k) {
  return fma_(C(k), r.Js, r.J0);
}

// ---------------------------------------------------------------------------
// reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block (fixed order: shuffle tree inside each warp, then
// warp 0 over the warp sums).  Every thread must call it; the block size must
// be a multiple of 32.  The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh /*>=32*/) {
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthreads = blockDim.x * blockDim.y;
  v = warp_sum(v);
  __syncthreads();
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (t < 32) {
    r = (t < (nthreads + 31) / 32) ? sh[t] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Deterministic grid-wide sum: every block stores its partial; the last block
// to arrive adds all partials in index order and writes *result.  The counter
// is left at zero for the next use.  Every thread of every participating
// block must call it: block bid of nb participating blocks (the others must
// not call it); the short form takes every block of the grid.
__device__ __forceinline__ void grid_sum_finalize(double v, double *partials, unsigned *counter, double *result,
                                                  double *sh, unsigned bid, unsigned nb) {
  __shared__ int s_last;
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthreads = blockDim.x * blockDim.y;
  double bs = block_sum(v, sh);
  if (t == 0) {
    partials[bid] = bs;
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == nb - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double acc = 0.0;
    for (unsigned k = t; k < nb; k += nthreads) acc += __ldcg(partials + k);
    double tot = block_sum(acc, sh);
    if (t == 0) {
      *result = tot;
      *counter = 0u;
    }
  }
}

__device__ __forceinline__ void grid_sum_finalize(double v, double *partials, unsigned *counter,
                                                  double *result, double *sh) {
  grid_sum_finalize(v, partials, counter, result, sh, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                    gridDim.x * gridDim.y * gridDim.z);
}

}  // namespace gkb

// Fast FP32-accumulating projector kernels for sm_103a.
//
//   k_back_tile       B,   pixel-driven: a 32x16 pixel tile per CTA; for each
//                     chunk of 16 angles the tile's window of sinogram bins is
//                     staged in shared memory (zero outside the detector), so
//                     the inner loop is bounds-check free.
//   k_fadj_tile       A^T, pixel-driven: the same tiling; per chunk of 8 angles
//                     the window of candidate rays (their Joseph parameters and
//                     sinogram values) is staged in shared memory.
//   k_forward_band    A,   ray-driven: a CTA owns up to 128 neighbouring rays of
//                     one angle and walks the image in bands of 16 rows; each
//                     band's footprint box (16 x 256 pixels) is brought into
//                     shared memory by a TMA tiled copy into a 3-stage ring
//                     (mbarrier completion).  Out-of-image parts of a box are
//                     zero-filled by the copy engine, which is exactly Joseph's
//                     zero padding, so the row loop has no bounds checks.
//   k_badj_band       B^T, ray-driven with the same banded TMA staging: per
//                     row, the pixels whose bin coordinate lies within one bin
//                     of the ray are enumerated between the two strip
//                     boundaries and weighted with pixel_bin().
//   k_transpose       rays closer to horizontal step over columns; they run on
//                     a transposed copy of the image so every band is a set of
//                     consecutive rows of some row-major image.
//
// Each kernel computes interpolation coordinates with the same expressions
// (ray_coord, pixel_bin) as its transpose, so the pairs stay exact transposes.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fast.h"

namespace gkb {
namespace {

// ---------------------------------------------------------------------------
// small PTX helpers (mbarrier + TMA)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait on the phase parity; returns false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void epilogue_f(bool valid, long long idx, float v, T *__restrict__ out, const Epi &e,
                                           double *sh) {
  float o = v;
  double sq = 0.0;
  if (valid) {
    if (e.prev) o = v - (float)(*e.gamma) * to_c(static_cast<const T *>(e.prev)[idx]);
    if (e.z) {
      float *z = static_cast<float *>(e.z);
      z[idx] = v - (float)(*e.cz) * z[idx];
    }
    const T st = from_c<T>(o);
    out[idx] = st;
    const double os = (double)to_c(st);
    sq = os * os;
  }
  if (e.partials) grid_sum_finalize(sq, e.partials, e.counter, e.result, sh);
}

// ---------------------------------------------------------------------------
// B: pixel-driven back projection, tiled

constexpr int TX = 32, TY = 8;          // pixel tile, one pixel per thread

// window start of tile (j0, i0) at angle A: floor of the smallest bin
// coordinate of the tile's corner pixels, minus one bin of margin
template <int BEAM>
__device__ __forceinline__ float tile_tmin(const GeomK<float> &G, const AngleP<float> &A, int j0, int i0, float &tmax) {
  float tmin = 3.0e38f;
  tmax = -3.0e38f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float xr = (float)(j0 + ((c & 1) ? TX - 1 : 0)) - G.hx;
    const float yr = G.hy - (float)(i0 + ((c & 2) ? TY - 1 : 0));
    float t, w;
    pixel_bin_f<BEAM>(G, A, xr, yr, t, w);
    tmin = fminf(tmin, t);
    tmax = fmaxf(tmax, t);
  }
  return tmin;
}

template <typename T, int BNA, int BEAM>
__global__ void __launch_bounds__(256) k_back_tile(GeomK<float> G, const T *__restrict__ y, T *__restrict__ x, Epi e) {
  if (e.done && *e.done) return;
  __shared__ float sino[BNA][kWinB];
  __shared__ AngleP<float> s_ang[BNA];
  __shared__ int s_dlo[BNA];
  __shared__ double sh[32];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int j0 = blockIdx.x * TX, i0 = blockIdx.y * TY;
  const int j = j0 + tx, i = i0 + ty;
  const float xr = (float)j - G.hx, yr = G.hy - (float)i;
  float acc = 0.f;
  for (int a0 = 0; a0 < G.na; a0 += BNA) {
    const int na = min(BNA, G.na - a0);
    if (tid < na) {
      float tmax;
      const AngleP<float> A = G.ang[a0 + tid];
      const float tmin = tile_tmin<BEAM>(G, A, j0, i0, tmax);
      s_dlo[tid] = (int)floorf(tmin) - 1;
      s_ang[tid] = A;
    }
    __syncthreads();
    for (int k = tid; k < na * kWinB; k += 256) {
      const int aa = k / kWinB, w = k - aa * kWinB;
      const int d = s_dlo[aa] + w;
      sino[aa][w] = (d >= 0 && d < G.nd) ? to_c(y[(long long)(a0 + aa) * G.nd + d]) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int aa = 0; aa < na; ++aa) {
      const AngleP<float> A = s_ang[aa];
      float t, w;
      pixel_bin_f<BEAM>(G, A, xr, yr, t, w);
      const float fl = floorf(t), f = t - fl;
      const int k = min(max((int)fl - s_dlo[aa], 0), kWinB - 2);
      acc += w * ((1.f - f) * sino[aa][k] + f * sino[aa][k + 1]);
    }
    __syncthreads();
  }
  epilogue_f<T>((j < G.nx) && (i < G.ny), (long long)i * G.nx + j, acc, x, e, sh);
}

// ---------------------------------------------------------------------------
// A^T: pixel-driven gather of Joseph weights, tiled

// First candidate ray of the tile at (j0, i0) for one angle: one below the
// tile's ray range (ray_range_rect).
__device__ __forceinline__ int fadj_dlo(const GeomK<float> &G, const AngleP<float> &A, int j0, int i0) {
  float lo, hi;
  ray_range_rect(G, A, (float)j0 - G.hx, (float)(j0 + TX - 1) - G.hx, G.hy - (float)(i0 + TY - 1), G.hy - (float)i0,
                 lo, hi);
  return (int)floorf(fmaxf(lo, -1.0e9f)) - 1;
}

template <typename T, int ANA>
__global__ void __launch_bounds__(256) k_fadj_tile(GeomK<float> G, const T *__restrict__ y, T *__restrict__ x, Epi e) {
  if (e.done && *e.done) return;
  __shared__ float4 rays[ANA][kWinA];   // (J0, Js, scale * y, axis) of the candidate rays
  __shared__ AngleP<float> s_ang[ANA];
  __shared__ int s_dlo[ANA];
  __shared__ double sh[32];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int j0 = blockIdx.x * TX, i0 = blockIdx.y * TY;
  const int j = j0 + tx, i = i0 + ty;
  const float xr = (float)j - G.hx, yr = G.hy - (float)i;
  const float fj = (float)j, fi = (float)i;
  float acc = 0.f;
  for (int a0 = 0; a0 < G.na; a0 += ANA) {
    const int na = min(ANA, G.na - a0);
    if (tid < na) {
      const AngleP<float> A = G.ang[a0 + tid];
      s_dlo[tid] = fadj_dlo(G, A, j0, i0);
      s_ang[tid] = A;
    }
    __syncthreads();
    for (int k = tid; k < na * kWinA; k += 256) {
      const int aa = k / kWinA, w = k - aa * kWinA;
      const int d = s_dlo[aa] + w;
      const bool in = d >= 0 && d < G.nd;
      const long long r = (long long)(a0 + aa) * G.nd + d;
      const RayP<float> rp = in ? G.ray[r] : RayP<float>{0.f, 0.f, 0.f, 0.f};
      // the Joseph weight of ray r on a pixel is (1 - f) or f times scale; fold scale and y
      rays[aa][w] = make_float4(rp.J0, rp.Js, in ? rp.scale * to_c(y[r]) : 0.f, rp.axis);
    }
    __syncthreads();
    for (int aa = 0; aa < na; ++aa) {
      const AngleP<float> A = s_ang[aa];
      const int dlo = s_dlo[aa];
      float lo, hi;
      ray_range(G, A, xr, yr, lo, hi);
      const int k0 = max((int)ceilf(fmaxf(lo, -1.0e9f)) - dlo, 0);
      const int k1 = min((int)floorf(fminf(hi, 1.0e9f)) - dlo, kWinA - 1);
      for (int k = k0; k <= k1; ++k) {
        const float4 r4 = rays[aa][k];
        const bool ax0 = r4.w == 0.f;
        const float c = fmaf(ax0 ? fi : fj, r4.y, r4.x);   // = ray_coord(ray, ax0 ? i : j)
        const float fl = floorf(c), f = c - fl;
        const float me = ax0 ? fj : fi;
        const float wt = (fl == me) ? 1.f - f : ((fl + 1.f == me) ? f : 0.f);
        acc += wt * r4.z;
      }
    }
    __syncthreads();
  }
  epilogue_f<T>((j < G.nx) && (i < G.ny), (long long)i * G.nx + j, acc, x, e, sh);
}

// ---------------------------------------------------------------------------
// A^T, ray-driven inside a pixel tile.  The pixel-driven kernels above test
// candidate rays per pixel; here each staged ray deposits its two Joseph
// weights per row (or column) of a 16x16 tile, which is the forward
// projector's own step: one coordinate, one floor, two products per ray and
// row.  A half-warp takes a ray with one lane per row (row-stepping rays) or
// per column (column-stepping rays), so its 16 lanes write 16 different
// pixels.  Every half-warp accumulates into its own copy of the tile and
// takes its rays in a fixed order, and the eight copies are added in a fixed
// order at the end: the result is deterministic without atomics.

constexpr int SW = 16;       // scatter tile edge (pixels)
constexpr int kWinS = 64;    // staged rays per angle and tile

__device__ __forceinline__ void scatter_window(const GeomK<float> &G, const AngleP<float> &A, int j0, int i0,
                                               int &dlo, int &cnt) {
  float lo, hi;
  ray_range_rect(G, A, (float)j0 - G.hx, (float)(j0 + SW - 1) - G.hx, G.hy - (float)(i0 + SW - 1), G.hy - (float)i0,
                 lo, hi);
  dlo = max((int)floorf(fmaxf(lo, -1.0e9f)) - 1, 0);
  const int dhi = min((int)ceilf(fminf(hi, 1.0e9f)) + 1, G.nd - 1);
  cnt = max(min(dhi - dlo + 1, kWinS), 0);
}

template <typename T>
__device__ __forceinline__ void epilogue2_f(bool va, long long ia, float a, bool vb, long long ib, float b,
                                            T *__restrict__ out, const Epi &e, double *sh) {
  double sq = 0.0;
  const bool vs[2] = {va, vb};
  const long long is[2] = {ia, ib};
  const float xs[2] = {a, b};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!vs[q]) continue;
    const long long idx = is[q];
    const float v = xs[q];
    float o = v;
    if (e.prev) o = v - (float)(*e.gamma) * to_c(static_cast<const T *>(e.prev)[idx]);
    if (e.z) {
      float *z = static_cast<float *>(e.z);
      z[idx] = v - (float)(*e.cz) * z[idx];
    }
    const T st = from_c<T>(o);
    out[idx] = st;
    const double os = (double)to_c(st);
    sq += os * os;
  }
  if (e.partials) grid_sum_finalize(sq, e.partials, e.counter, e.result, sh);
}

// Exact ray window of every (16x16 tile, angle) and the scatter's lane
// stride there: the first ray that deposits into the tile, how many follow,
// and the smallest t in 1..4 such that no two rays t apart (same axis) fall
// into the same slot of any line of the tile, checked with the kernel's own
// arithmetic.  Packed lo | count << 20 | (t - 1) << 30; *bad is set when a
// tile needs t > 4.  One warp per (tile, angle).
__global__ void __launch_bounds__(128) k_scatter_windows(GeomK<float> G, uint32_t *__restrict__ swin, int tiles_x,
                                                         long long n_pairs, int *__restrict__ bad) {
  const long long pair = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= n_pairs) return;
  const int a = (int)(pair % G.na);
  const long long tile = pair / G.na;
  const int j0 = (int)(tile % tiles_x) * SW, i0 = (int)(tile / tiles_x) * SW;
  int lo, cnt;
  scatter_window(G, G.ang[a], j0, i0, lo, cnt);
  int first = 1 << 30, last = -1;
  for (int w0 = 0; w0 < cnt; w0 += 32) {
    const int w = w0 + lane;
    bool hit = false;
    if (w < cnt) {
      const RayP<float> rp = G.ray[(long long)a * G.nd + lo + w];
      const bool ax0 = rp.axis == 0.f;
      for (int L = 0; L < SW; ++L) {
        const float c = fmaf((float)((ax0 ? i0 : j0) + L), rp.Js, rp.J0);
        const int q = (int)floorf(c) - (ax0 ? j0 : i0);
        if (q >= -1 && q < SW) hit = true;
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (b) {
      first = min(first, w0 + __ffs(b) - 1);
      last = max(last, w0 + 31 - __clz(b));
    }
  }
  const int n = last - first + 1;
  const long long r0 = (long long)a * G.nd + lo + first;
  int tbest = 0;
  for (int t = 1; t <= 4 && n > 0 && tbest == 0; ++t) {
    bool clash = false;
    for (int w0 = 0; w0 < n; w0 += 32) {
      const int w = w0 + lane;
      bool c = false;
      if (w + t < n) {
        const RayP<float> p0 = G.ray[r0 + w], p1 = G.ray[r0 + w + t];
        if (p0.axis == p1.axis) {
          const bool ax0 = p0.axis == 0.f;
          const int kb = ax0 ? i0 : j0, qb = (ax0 ? j0 : i0) - 1;
          for (int k = 0; k < SW; ++k) {
            const int q0 = (int)floorf(fmaf((float)(kb + k), p0.Js, p0.J0)) - qb;
            const int q1 = (int)floorf(fmaf((float)(kb + k), p1.Js, p1.J0)) - qb;
            if (q0 == q1 && (unsigned)q0 < (unsigned)(SW + 1)) c = true;
          }
        }
      }
      if (__any_sync(0xffffffffu, c)) clash = true;
    }
    if (!clash) tbest = t;
  }
  if (lane == 0) {
    if (n > 0 && tbest == 0) atomicExch(bad, 1);
    swin[pair] = n > 0 ? (uint32_t)(lo + first) | ((uint32_t)n << 20) | ((uint32_t)(max(tbest, 1) - 1) << 30) : 0u;
  }
}

constexpr int kLine = SW + 1;              // row stride of an accumulator tile (conflict-free columns)
constexpr int kHalfAcc = 2 * SW * kLine + 16;   // E and F tiles of one half-warp, padded to shift banks

template <typename T, int CH>
__global__ void __launch_bounds__(128) k_fadj_scatter(GeomK<float> G, const uint32_t *__restrict__ swin,
                                                      const T *__restrict__ y, T *__restrict__ x, Epi e) {
  static_assert(CH % 8 == 0 && CH <= 32, "angle chunks of whole half-warp rounds");
  if (e.done && *e.done) return;
  // Per half-warp two tiles indexed by pixel: E collects the (1 - f) parts,
  // F the f parts, of every ray's two weights on a line.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *acc = reinterpret_cast<float *>(smem_raw);             // [8][kHalfAcc]
  float4 *rays = reinterpret_cast<float4 *>(acc + 8 * kHalfAcc);   // [CH * kWinS]
  __shared__ int s_lo[CH], s_off[CH + 1], s_t[CH], s_sw[CH];
  __shared__ double sh[32];
  const int tid = threadIdx.x, hw = tid >> 4, L = tid & 15;
  const int j0 = blockIdx.x * SW, i0 = blockIdx.y * SW;
  for (int k = tid; k < 8 * kHalfAcc; k += 128) acc[k] = 0.f;
  float *accE = acc + hw * kHalfAcc, *accF = accE + SW * kLine;
  const unsigned hmask = 0xffffu << (16 * (hw & 1));
  for (int a0 = 0; a0 < G.na; a0 += CH) {
    const int na = min(CH, G.na - a0);
    if (tid < 32) {
      int lo = 0, cnt = 0, ts = 1;
      if (tid < na) {
        const uint32_t wv = swin[((long long)blockIdx.y * gridDim.x + blockIdx.x) * G.na + a0 + tid];
        lo = (int)(wv & 0xfffffu);
        cnt = (int)((wv >> 20) & 0x3ffu);
        ts = (int)(wv >> 30) + 1;
      }
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += u;
      }
      if (tid < CH) {
        s_lo[tid] = lo;
        s_off[tid] = incl - cnt;
        s_t[tid] = ts;
        s_sw[tid] = cnt;
      }
      if (tid == CH - 1) s_off[CH] = incl;
    }
    __syncthreads();
    for (int aa = hw; aa < na; aa += 8) {
      const int o = s_off[aa], cnt = s_off[aa + 1] - o;
      const long long r0 = (long long)(a0 + aa) * G.nd + s_lo[aa];
      for (int w = L; w < cnt; w += 16) {
        const RayP<float> rp = G.ray[r0 + w];
        rays[o + w] = make_float4(rp.J0, rp.Js, rp.scale * to_c(y[r0 + w]), rp.axis);
        // where the stepping axis switches (at most once in a projection)
        if (w > 0 && G.ray[r0 + w - 1].axis != rp.axis) s_sw[aa] = w;
      }
    }
    __syncthreads();
    // half-warp hw takes the angles a = hw (mod 8) and their row-stepping and
    // column-stepping rays separately; its lanes take rays t_stride apart,
    // which never reach the same pixel of a line of this tile, so the 16 lanes
    // of one step touch 16 different E and F entries
    for (int aa = hw; aa < na; aa += 8)
    for (int part = 0; part < 2; ++part) {
      const int o = s_off[aa], t_stride = s_t[aa];
      const int w_lo = part ? s_sw[aa] : 0, w_hi = part ? s_off[aa + 1] - o : s_sw[aa];
      for (int base = w_lo; base < w_hi; base += 16 * t_stride) {
        for (int ph = 0; ph < t_stride; ++ph) {
          const int w = base + ph + t_stride * L;
          const bool act = w < w_hi;
          const float4 r4 = act ? rays[o + w] : make_float4(0.f, 0.f, 0.f, 0.f);
          const bool ax0 = r4.w == 0.f;
          const int kb = ax0 ? i0 : j0, qb = ax0 ? j0 : i0;
          // pixel (line k, position q) sits at k * kLine + q (row-stepping)
          // or q * kLine + k (column-stepping)
          const int sk = ax0 ? kLine : 1, sq = ax0 ? 1 : kLine;
          // four lines per round (k, k + 4, k + 8, k + 12 differ, so do all
          // their entries): loads, then updates, then stores
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float fr[4];
            int ie[4];
            bool okE[4], okF[4];
            float vE[4], vF[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int kk = k + 4 * u;
              const float c = fmaf((float)(kb + kk), r4.y, r4.x);   // = ray_coord(ray, row or column kb + kk)
              const float fl = floorf(c);
              fr[u] = c - fl;
              const int q = (int)fl - qb;
              okE[u] = act && (unsigned)q < (unsigned)SW;
              okF[u] = act && (unsigned)(q + 1) < (unsigned)SW;
              ie[u] = kk * sk + q * sq;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (okE[u]) vE[u] = accE[ie[u]];
              if (okF[u]) vF[u] = accF[ie[u] + sq];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (okE[u]) accE[ie[u]] = fmaf(1.f - fr[u], r4.z, vE[u]);
              if (okF[u]) accF[ie[u] + sq] = fmaf(fr[u], r4.z, vF[u]);
            }
          }
          // the next lane set may touch entries this one touched
          __syncwarp(hmask);
        }
      }
    }
    __syncthreads();
  }
  float v[2];
  int ii[2], jj[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int p = tid + q * 128, r = p / SW, cc = p - r * SW;
    float sum = 0.f;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const float *E = acc + h * kHalfAcc, *F = E + SW * kLine;
      sum += E[r * kLine + cc] + F[r * kLine + cc];
    }
    v[q] = sum;
    ii[q] = i0 + r;
    jj[q] = j0 + cc;
  }
  epilogue2_f<T>(ii[0] < G.ny && jj[0] < G.nx, (long long)ii[0] * G.nx + jj[0], v[0], ii[1] < G.ny && jj[1] < G.nx,
                 (long long)ii[1] * G.nx + jj[1], v[1], x, e, sh);
}

template <typename T, int CH>
constexpr size_t fadj_scatter_smem() {
  return sizeof(float) * 8 * kHalfAcc + sizeof(float4) * CH * kWinS;
}

// ---------------------------------------------------------------------------
// transpose (rows <-> columns) for the column-stepping rays

template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T *__restrict__ in, T *__restrict__ out, int rows, int cols) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = by + r, jj = bx + threadIdx.x;
    if (i < rows && jj < cols) tile[r][threadIdx.x] = in[(long long)i * cols + jj];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int jj = bx + r, i = by + threadIdx.x;
    if (jj < cols && i < rows) out[(long long)jj * rows + i] = tile[threadIdx.x][r];
  }
}

// ---------------------------------------------------------------------------
// banded ray-driven kernels (A and B^T)

struct BandCtx {
  int a, d0, nb, axis;
  int rows, cols;   // image as walked: rows = stepping extent, cols = interpolation extent
  int k0, k1;       // row range of the item
};

// rows in [0, kmax) where J0 + k Js lies in (-1 - pad, lim + pad)
__device__ __forceinline__ void band_range(float J0, float Js, int lim, int kmax, float pad, int &k0, int &k1) {
  const float lo = -1.f - pad, hi = (float)lim + pad;
  if (fabsf(Js) < 1e-30f) {
    if (J0 > lo && J0 < hi) { k0 = 0; k1 = kmax - 1; } else { k0 = 0; k1 = -1; }
    return;
  }
  float p = (lo - J0) / Js, q = (hi - J0) / Js;
  if (p > q) { const float t = p; p = q; q = t; }
  p = fminf(fmaxf(p, -2.f), (float)kmax + 1.f);
  q = fminf(fmaxf(q, -2.f), (float)kmax + 1.f);
  k0 = max((int)floorf(p) - 1, 0);
  k1 = min((int)floorf(q) + 1, kmax - 1);
}

// Minimum interpolation coordinate of the item's rays over rows [r0, r1].
__device__ __forceinline__ float band_min(const RayP<float> &f, const RayP<float> &l, int r0, int r1) {
  return fminf(fminf(ray_coord(f, r0), ray_coord(f, r1)), fminf(ray_coord(l, r0), ray_coord(l, r1)));
}

template <typename T, int kBandRows, int kStages>
__global__ void __launch_bounds__(kBandRays) k_forward_band(const __grid_constant__ CUtensorMap tm_x,
                                                           const __grid_constant__ CUtensorMap tm_xt, GeomK<float> G,
                                                           const int4 *__restrict__ items, T *__restrict__ y, Epi e) {
  if (e.done && *e.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  const int4 it = items[blockIdx.x];
  const int a = it.x, d0 = it.y, nb = it.z, axis = it.w;
  const int rows = axis ? G.nx : G.ny, cols = axis ? G.ny : G.nx;
  const CUtensorMap *tm = axis ? &tm_xt : &tm_x;
  const RayP<float> *rt = G.ray + (long long)a * G.nd;
  const RayP<float> rf = rt[d0], rl = rt[d0 + nb - 1];
  const bool active = tid < nb;
  const RayP<float> ray = rt[d0 + (active ? tid : nb - 1)];
  // rows the item touches: hull of every ray's own row range
  __shared__ int s_k0, s_k1;
  if (tid == 0) {
    s_k0 = rows;
    s_k1 = -1;
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (active) {
    int ka, kb;
    band_range(ray.J0, ray.Js, cols, rows, 0.f, ka, kb);
    if (kb >= ka) {
      atomicMin(&s_k0, ka);
      atomicMax(&s_k1, kb);
    }
  }
  __syncthreads();
  const int k0 = s_k0, k1 = s_k1;
  const int nbands = k1 >= k0 ? (k1 - k0 + kBandRows) / kBandRows : 0;
  constexpr int align = 16 / (int)sizeof(T);
  constexpr uint32_t box_bytes = kBandRows * kBoxW * sizeof(T);
  auto box_x = [&](int b) {
    const int r0 = k0 + b * kBandRows, r1 = r0 + kBandRows - 1;
    const int xm = (int)floorf(band_min(rf, rl, r0, r1)) - 1;
    return (xm >= 0) ? (xm / align) * align : -(((-xm) + align - 1) / align) * align;
  };
  if (tid == 0) {
    for (int b = 0; b < min(kStages, nbands); ++b) {
      mbar_expect_tx(&full[b], box_bytes);
      tma_load_2d(buf + (size_t)b * kBandRows * kBoxW, tm, &full[b], box_x(b), k0 + b * kBandRows);
    }
  }
  float acc = 0.f;
  bool ok = true;
  for (int b = 0; b < nbands; ++b) {
    const int s = b % kStages;
    if (!mbar_wait(&full[s], (uint32_t)((b / kStages) & 1))) { ok = false; }
    const T *S = buf + (size_t)s * kBandRows * kBoxW;
    const int r0 = k0 + b * kBandRows;
    const int x0 = box_x(b);
#pragma unroll 4
    for (int r = 0; r < kBandRows; ++r) {
      const float c = ray_coord(ray, r0 + r);
      const float fl = floorf(c), f = c - fl;
      const int jj = min(max((int)fl - x0, 0), kBoxW - 2);
      acc += (1.f - f) * to_c(S[r * kBoxW + jj]) + f * to_c(S[r * kBoxW + jj + 1]);
    }
    __syncthreads();
    if (tid == 0 && b + kStages < nbands) {
      fence_proxy_async();
      mbar_expect_tx(&full[s], box_bytes);
      tma_load_2d(buf + (size_t)s * kBandRows * kBoxW, tm, &full[s], box_x(b + kStages), k0 + (b + kStages) * kBandRows);
    }
  }
  float v = acc * ray.scale;
  if (!ok) v = __int_as_float(0x7fc00000);  // a copy never arrived: poison the output
  epilogue_f<T>(active, (long long)a * G.nd + d0 + tid, v, y, e, sh);
}

// strip boundary of bin coordinate tb at angle A as an affine map of the
// stepping index: coordinate(k) = P + k Q along the item's walking axis
__device__ __forceinline__ void strip_line(const GeomK<float> &G, const AngleP<float> &A, float tb, int axis,
                                           float bin_per_pix, float &P, float &Q) {
  // detector coordinate of the boundary in pixel units (bins times det_width/pixel)
  const float ub = (tb - G.t0) / bin_per_pix;
  float px, py, ex, ey;
  if (G.beam == 0) {
    px = ub * A.c; py = ub * A.s; ex = -A.s; ey = A.c;
  } else if (G.beam == 2) {
    // arc: the boundary ray leaves the source at the angle (tb - t0) / g
    float sg, cg;
    sincosf((tb - G.t0) / G.gfan, &sg, &cg);
    px = G.sodp * A.c; py = G.sodp * A.s;
    ex = -A.c * cg - A.s * sg; ey = -A.s * cg + A.c * sg;
  } else {
    // source and detector point in pixel units
    const float sp = G.sodp;
    const float dd = G.gfan / bin_per_pix - sp;   // (sdd - sod)/pixel
    px = sp * A.c; py = sp * A.s;
    const float bx = -dd * A.c - ub * A.s, by = -dd * A.s + ub * A.c;
    ex = bx - px; ey = by - py;
  }
  if (axis == 0) {  // column coordinate at row k: x = px + (y_k - py) ex/ey, y_k = hy - k
    const float q = ex / ey;
    P = px + (G.hy - py) * q + G.hx;
    Q = -q;
  } else {          // row coordinate at column k: hy - (py + (x_k - px) ey/ex), x_k = k - hx
    const float q = ey / ex;
    P = G.hy - (py + (-G.hx - px) * q);
    Q = -q;
  }
}

// Rows an item of B^T touches: the hull over its rays of the rows where each
// ray's strip (between its two boundaries and around its centre line) meets
// the image.  Called by all threads of the CTA (two barriers inside).
__device__ __forceinline__ void strip_hull(bool active, float Pm, float Qm, float Pp, float Qp, int rows, int cols,
                                           int *s_k0, int *s_k1, int &k0, int &k1) {
  if (threadIdx.x == 0) {
    *s_k0 = rows;
    *s_k1 = -1;
  }
  __syncthreads();
  if (active) {
    int lo = rows, hi = -1, ka, kb;
    band_range(Pm, Qm, cols, rows, 2.f, ka, kb);
    if (kb >= ka) { lo = min(lo, ka); hi = max(hi, kb); }
    band_range(Pp, Qp, cols, rows, 2.f, ka, kb);
    if (kb >= ka) { lo = min(lo, ka); hi = max(hi, kb); }
    band_range(0.5f * (Pm + Pp), 0.5f * (Qm + Qp), cols, rows, 2.f, ka, kb);
    if (kb >= ka) { lo = min(lo, ka); hi = max(hi, kb); }
    if (hi >= lo) {
      atomicMin(s_k0, lo);
      atomicMax(s_k1, hi);
    }
  }
  __syncthreads();
  k0 = *s_k0;
  k1 = *s_k1;
}

template <typename T, int kBandRows, int kStages>
__global__ void __launch_bounds__(kBandRays) k_badj_band(const __grid_constant__ CUtensorMap tm_x,
                                                        const __grid_constant__ CUtensorMap tm_xt, GeomK<float> G,
                                                        const int4 *__restrict__ items, float bin_per_pix,
                                                        T *__restrict__ y, Epi e) {
  if (e.done && *e.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  const int4 it = items[blockIdx.x];
  const int a = it.x, d0 = it.y, nb = it.z, axis = it.w;
  const int rows = axis ? G.nx : G.ny, cols = axis ? G.ny : G.nx;
  const CUtensorMap *tm = axis ? &tm_xt : &tm_x;
  const AngleP<float> A = G.ang[a];
  const bool active = tid < nb;
  const int d = d0 + (active ? tid : nb - 1);
  // strip boundaries (bins d-1 and d+1) of this ray and of the item's outer rays
  float Pm, Qm, Pp, Qp, Pf, Qf, Pl, Ql;
  strip_line(G, A, (float)(d - 1), axis, bin_per_pix, Pm, Qm);
  strip_line(G, A, (float)(d + 1), axis, bin_per_pix, Pp, Qp);
  strip_line(G, A, (float)(d0 - 1), axis, bin_per_pix, Pf, Qf);
  strip_line(G, A, (float)(d0 + nb), axis, bin_per_pix, Pl, Ql);
  const float marg = 0.02f;
  __shared__ int s_k0, s_k1;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  int k0, k1;
  strip_hull(active, Pm, Qm, Pp, Qp, rows, cols, &s_k0, &s_k1, k0, k1);
  const int nbands = k1 >= k0 ? (k1 - k0 + kBandRows) / kBandRows : 0;
  constexpr int align = 16 / (int)sizeof(T);
  constexpr uint32_t box_bytes = kBandRows * kBoxW * sizeof(T);
  auto box_x = [&](int b) {
    const int r0 = k0 + b * kBandRows, r1 = r0 + kBandRows - 1;
    const float m = fminf(fminf(fmaf((float)r0, Qf, Pf), fmaf((float)r1, Qf, Pf)),
                          fminf(fmaf((float)r0, Ql, Pl), fmaf((float)r1, Ql, Pl)));
    const int xm = (int)floorf(m) - 2;
    return (xm >= 0) ? (xm / align) * align : -(((-xm) + align - 1) / align) * align;
  };
  if (tid == 0) {
    for (int b = 0; b < min(kStages, nbands); ++b) {
      mbar_expect_tx(&full[b], box_bytes);
      tma_load_2d(buf + (size_t)b * kBandRows * kBoxW, tm, &full[b], box_x(b), k0 + b * kBandRows);
    }
  }
  const float fd = (float)d;
  float acc = 0.f;
  bool ok = true;
  for (int b = 0; b < nbands; ++b) {
    const int s = b % kStages;
    if (!mbar_wait(&full[s], (uint32_t)((b / kStages) & 1))) ok = false;
    const T *S = buf + (size_t)s * kBandRows * kBoxW;
    const int r0 = k0 + b * kBandRows;
    const int x0 = box_x(b);
    for (int r = 0; r < kBandRows; ++r) {
      const int k = r0 + r;
      if (k > k1) break;
      const float cm = fmaf((float)k, Qm, Pm), cp = fmaf((float)k, Qp, Pp);
      const int c0 = max(max((int)ceilf(fminf(cm, cp) - marg), 0), x0);
      const int c1 = min(min((int)floorf(fmaxf(cm, cp) + marg), cols - 1), x0 + kBoxW - 1);
      // pixel coordinates of the candidates, stepped exactly (small integers)
      const float fk = axis ? (float)k - G.hx : G.hy - (float)k;
      float fc = axis ? G.hy - (float)c0 : (float)c0 - G.hx;
      const float dc = axis ? -1.f : 1.f;
      for (int c = c0; c <= c1; ++c, fc += dc) {
        // pixel (i, j) of the original image: axis 0 walks rows (k = i), axis 1 columns (k = j)
        float t, w;
        pixel_bin(G, A, axis ? fk : fc, axis ? fc : fk, t, w);
        const float fl = floorf(t), f = t - fl;
        const float wt = (fl == fd) ? 1.f - f : ((fl + 1.f == fd) ? f : 0.f);
        acc += w * wt * to_c(S[r * kBoxW + (c - x0)]);
      }
    }
    __syncthreads();
    if (tid == 0 && b + kStages < nbands) {
      fence_proxy_async();
      mbar_expect_tx(&full[s], box_bytes);
      tma_load_2d(buf + (size_t)s * kBandRows * kBoxW, tm, &full[s], box_x(b + kStages), k0 + (b + kStages) * kBandRows);
    }
  }
  float v = acc;
  if (!ok) v = __int_as_float(0x7fc00000);
  epilogue_f<T>(active, (long long)a * G.nd + d0 + tid, v, y, e, sh);
}

// ---------------------------------------------------------------------------
// B^T, pixel-driven scatter.  The ray-driven kernel evaluates pixel_bin() for
// every candidate pixel of every ray (about three rays per pixel and angle);
// here every pixel evaluates it once per angle and adds its two weighted
// values to the two bins, exactly as B reads them.  The additions are
// integers: each value is scaled by a power of two chosen from max|x| and a
// bound on the weights (per tile for the 32-bit shared-memory sums, for the
// whole image for the 64-bit global sums) and rounded to the nearest integer.  Integer addition is associative, so the shared-memory
// atomics inside a CTA and the 64-bit global atomics between CTAs give the
// same result in any order: the operator is deterministic.  A CTA owns a
// 32x32 pixel tile and a group of angles; a finishing kernel converts the
// integer sums back, runs the fused epilogue and clears the accumulator.

constexpr int BS = 32;        // scatter tile edge (pixels)
constexpr int kWinB2 = 96;    // bins per angle and tile
constexpr int kBCH = 8;       // angles per shared-memory round

// Power-of-two scales.  Global: values bounded by wmax * M (M = max|x|); the
// sum of 2^log2n of them stays below 2^62 after scaling, so no ray's 64-bit
// sum can overflow.  Tile: a tile adds at most P values into one bin, each
// bounded by wmax * Mt (Mt = the tile's max|x|); scaled, their sum stays
// below 2^30, so the 32-bit shared-memory sums cannot overflow.  The tile
// scale never exceeds the global one, and both are powers of two, so a tile's
// integer sum moves to the global scale by an exact left shift.
__device__ __forceinline__ int badj_exp(float M, float wmax, int log2n) {
  int ex;
  frexpf(wmax * M, &ex);   // wmax * M = m 2^ex, m in [0.5, 1)
  return min(max(62 - ex - log2n, -120), 120);
}
__device__ __forceinline__ int badj_tile_exp(float Mt, float wmax, float P, int eg) {
  int ex;
  frexpf(P * wmax * Mt, &ex);
  return min(30 - ex, eg);
}

template <typename T>
__global__ void __launch_bounds__(256) k_absmax(const T *__restrict__ x, long long n, unsigned *__restrict__ mx,
                                                Epi e) {
  if (e.done && *e.done) return;
  unsigned m = 0u;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const unsigned b = __float_as_uint(fabsf(to_c(x[i])));   // NaN sorts above +inf
    m = max(m, b);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

template <typename T, int BEAM>
__global__ void __launch_bounds__(256) k_badj_scatter(GeomK<float> G, const T *__restrict__ x,
                                                      const unsigned *__restrict__ mx, float wmax, float P,
                                                      int log2n, int tiles_x, unsigned long long *__restrict__ acc64,
                                                      Epi e) {
  if (e.done && *e.done) return;
  __shared__ float xs[BS][BS + 1];
  __shared__ int acc[kBCH][kWinB2];
  __shared__ unsigned s_mt;
  __shared__ AngleP<float> s_ang[kBCH];
  __shared__ int s_lo[kBCH], s_cnt[kBCH], s_rows[kBCH];
  const float M = __uint_as_float(*mx);
  if (!(M > 0.f) || !(M <= 3.4e38f)) return;   // all zero, or non-finite (the finishing kernel writes NaN)
  const int eg = badj_exp(M, wmax, log2n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = (blockIdx.x % tiles_x) * BS, i0 = (blockIdx.x / tiles_x) * BS;
  const int a_begin = (int)((long long)blockIdx.y * G.na / gridDim.y);
  const int a_end = (int)((long long)(blockIdx.y + 1) * G.na / gridDim.y);
  if (tid == 0) s_mt = 0u;
  __syncthreads();
  unsigned mt = 0u;
  for (int k = tid; k < BS * BS; k += 256) {
    const int r = k / BS, c = k - r * BS, i = i0 + r, j = j0 + c;
    const float v = (i < G.ny && j < G.nx) ? to_c(x[(long long)i * G.nx + j]) : 0.f;
    xs[r][c] = v;
    mt = max(mt, __float_as_uint(fabsf(v)));
  }
  mt = __reduce_max_sync(0xffffffffu, mt);
  if (lane == 0) atomicMax(&s_mt, mt);
  for (int k = tid; k < kBCH * kWinB2; k += 256) (&acc[0][0])[k] = 0;
  __syncthreads();
  if (s_mt == 0u) return;   // an all-zero tile adds nothing
  const int el = badj_tile_exp(__uint_as_float(s_mt), wmax, P, eg);
  const float S = ldexpf(1.f, el);
  const int shift = eg - el;
  // this thread's pixels: lanes along rows (row-major lines) or along columns,
  // whichever the bin coordinate moves faster on; centre coordinates and the
  // scaled values (exact: S is a power of two) stay in registers
  const float xr_lane = (float)(j0 + lane) - G.hx, yr_lane = G.hy - (float)(i0 + lane);
  float xr_w[BS / 8], yr_w[BS / 8], v_row[BS / 8], v_col[BS / 8];
#pragma unroll
  for (int q = 0; q < BS / 8; ++q) {
    const int r = warp + 8 * q;
    xr_w[q] = (float)(j0 + r) - G.hx;
    yr_w[q] = G.hy - (float)(i0 + r);
    v_row[q] = xs[r][lane] * S;
    v_col[q] = xs[lane][r] * S;
  }
  for (int a0 = a_begin; a0 < a_end; a0 += kBCH) {
    const int na = min(kBCH, a_end - a0);
    if (tid < na) {
      const AngleP<float> A = G.ang[a0 + tid];
      float tmin = 3.0e38f, tmax = -3.0e38f, t, w;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pixel_bin_f<BEAM>(G, A, (float)(j0 + ((c & 1) ? BS - 1 : 0)) - G.hx, G.hy - (float)(i0 + ((c & 2) ? BS - 1 : 0)), t, w);
        tmin = fminf(tmin, t);
        tmax = fmaxf(tmax, t);
      }
      const int lo = max((int)floorf(tmin) - 1, 0), hi = min((int)floorf(tmax) + 2, G.nd - 1);
      s_lo[tid] = lo;
      s_cnt[tid] = max(min(hi - lo + 1, kWinB2), 0);
      // lanes along the tile direction in which the bin coordinate moves faster: fewer lanes share a bin
      const float xc = (float)(j0 + BS / 2) - G.hx, yc = G.hy - (float)(i0 + BS / 2);
      float t0, tj, ti;
      pixel_bin_f<BEAM>(G, A, xc, yc, t0, w);
      pixel_bin_f<BEAM>(G, A, xc + 1.f, yc, tj, w);
      pixel_bin_f<BEAM>(G, A, xc, yc - 1.f, ti, w);
      s_rows[tid] = fabsf(tj - t0) >= fabsf(ti - t0);
      s_ang[tid] = A;
    }
    __syncthreads();
    for (int aa = 0; aa < na; ++aa) {
      const AngleP<float> A = s_ang[aa];
      const int lo = s_lo[aa];
      const unsigned cnt = (unsigned)s_cnt[aa];
      int *ac = acc[aa];
      // pixel (i, j) adds round(w v S (1 - f)) to bin fl and round(w v S f)
      // to bin fl + 1; the first is taken as round(w v S) minus the second,
      // so the two integers always sum to the rounded total
      auto deposit = [&](float xr, float yr, float vS) {
        float t, w;
        pixel_bin_f<BEAM>(G, A, xr, yr, t, w);
        const float fl = floorf(t), f = t - fl;
        const float tot = w * vS;
        const int d1 = __float2int_rn(tot * f);
        const int d0 = __float2int_rn(tot) - d1;
        const int k = (int)fl - lo;
        if ((unsigned)k < cnt) atomicAdd(ac + k, d0);
        if ((unsigned)(k + 1) < cnt) atomicAdd(ac + k + 1, d1);
      };
      if (s_rows[aa]) {
#pragma unroll
        for (int q = 0; q < BS / 8; ++q) deposit(xr_lane, yr_w[q], v_row[q]);
      } else {
#pragma unroll
        for (int q = 0; q < BS / 8; ++q) deposit(xr_w[q], yr_lane, v_col[q]);
      }
    }
    __syncthreads();
    for (int k = tid; k < na * kWinB2; k += 256) {
      const int aa = k / kWinB2, wi = k - aa * kWinB2;
      const int v = acc[aa][wi];
      if (v != 0) {
        if (wi < s_cnt[aa])
          atomicAdd(acc64 + (long long)(a0 + aa) * G.nd + s_lo[aa] + wi, (unsigned long long)((long long)v << shift));
        acc[aa][wi] = 0;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_badj_finish(long long m, unsigned long long *__restrict__ acc64,
                                                     const unsigned *__restrict__ mx, float wmax, int log2n,
                                                     T *__restrict__ y, Epi e) {
  if (e.done && *e.done) return;
  __shared__ double sh[32];
  const float M = __uint_as_float(*mx);
  const bool finite = M <= 3.4e38f;
  // 2^-e as a float (e <= 120 keeps it normal); scaling by it is exact
  const float inv = (M > 0.f && finite) ? ldexpf(1.f, -badj_exp(M, wmax, log2n)) : 0.f;
  double sq = 0.0;
  auto finish = [&](long long r, long long iv) {
    const float v = finite ? __ll2float_rn(iv) * inv : __int_as_float(0x7fc00000);
    float o = v;
    if (e.prev) o = v - (float)(*e.gamma) * to_c(static_cast<const T *>(e.prev)[r]);
    if (e.z) {
      float *z = static_cast<float *>(e.z);
      z[r] = v - (float)(*e.cz) * z[r];
    }
    const T st = from_c<T>(o);
    y[r] = st;
    const double os = (double)to_c(st);
    sq += os * os;
  };
  const long long stride = (long long)gridDim.x * 256;
  for (long long r0 = (long long)blockIdx.x * 256 + threadIdx.x; r0 < m; r0 += 2 * stride) {
    // two elements per round, their loads issued together
    const long long r1 = r0 + stride;
    const long long iv0 = (long long)acc64[r0];
    const long long iv1 = r1 < m ? (long long)acc64[r1] : 0ll;
    acc64[r0] = 0ull;
    finish(r0, iv0);
    if (r1 < m) {
      acc64[r1] = 0ull;
      finish(r1, iv1);
    }
  }
  if (e.partials) grid_sum_finalize(sq, e.partials, e.counter, e.result, sh);
}

// ---------------------------------------------------------------------------
// host side

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <typename T> CUtensorMapDataType tm_type();
template <> CUtensorMapDataType tm_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tm_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType tm_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <typename T>
bool make_map(CUtensorMap *m, const void *base, int rows, int cols, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(T)};
  cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, tm_type<T>(), 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the band-kernel shapes the autotuner chooses from: (rows per band, ring depth)
constexpr int kBandCfgs = 5;
constexpr int kBandCfgRows[kBandCfgs] = {8, 8, 16, 16, 32};
constexpr int kBandCfgStages[kBandCfgs] = {2, 3, 2, 3, 2};

template <typename T, int R, int S>
void launch_band_shape(int which, int n_items, const CUtensorMap &mx, const CUtensorMap &mt, const GeomK<float> &K,
                       const int4 *items, float bpp, void *out, const Epi &e, cudaStream_t s) {
  const size_t smem = (size_t)S * R * kBoxW * sizeof(T);
  T *y = static_cast<T *>(out);
  if (which == 0) k_forward_band<T, R, S><<<n_items, kBandRays, smem, s>>>(mx, mt, K, items, y, e);
  else k_badj_band<T, R, S><<<n_items, kBandRays, smem, s>>>(mx, mt, K, items, bpp, y, e);
}

template <typename T>
gkb_status launch_band(int which, const gkb_geometry *g, const void *in, void *out, void *scratch_t, const Epi &e,
                       cudaStream_t s) {
  const FastPlan &F = g->fast;
  const int nx = g->desc.nx, ny = g->desc.ny;
  const int cfg = which == 0 ? F.cfg_fwd : F.cfg_badj;
  const int R = kBandCfgRows[cfg];
  void *xt = scratch_t;
  bool own = false;
  if (F.any_axis1 && !xt) {
    GKB_CUDA_TRY(cudaMallocAsync(&xt, (size_t)g->n * sizeof(T), s));
    own = true;
  }
  CUtensorMap mx, mt;
  if (!make_map<T>(&mx, in, ny, nx, R)) return GKB_ERR_UNSUPPORTED;
  if (F.any_axis1) {
    dim3 tb(32, 8), tg((nx + 31) / 32, (ny + 31) / 32);
    k_transpose<T><<<tg, tb, 0, s>>>(static_cast<const T *>(in), static_cast<T *>(xt), ny, nx);
    if (!make_map<T>(&mt, xt, nx, ny, R)) return GKB_ERR_UNSUPPORTED;
  } else {
    mt = mx;
  }
  const GeomK<float> K = geom_view<float>(g);
  const int4 *items = which == 0 ? F.items_fwd : F.items_badj;
  const int n_items = which == 0 ? F.n_fwd : F.n_badj;
  const float bpp = (float)(g->desc.pixel / g->desc.det_width);
  switch (cfg) {
    case 0: launch_band_shape<T, 8, 2>(which, n_items, mx, mt, K, items, bpp, out, e, s); break;
    case 1: launch_band_shape<T, 8, 3>(which, n_items, mx, mt, K, items, bpp, out, e, s); break;
    case 2: launch_band_shape<T, 16, 2>(which, n_items, mx, mt, K, items, bpp, out, e, s); break;
    case 3: launch_band_shape<T, 16, 3>(which, n_items, mx, mt, K, items, bpp, out, e, s); break;
    default: launch_band_shape<T, 32, 2>(which, n_items, mx, mt, K, items, bpp, out, e, s); break;
  }
  GKB_CUDA_TRY(cudaGetLastError());
  if (own) GKB_CUDA_TRY(cudaFreeAsync(xt, s));
  return GKB_OK;
}

// tile-kernel angle chunks the autotuner chooses from
constexpr int kTileCfgs = 3;
constexpr int kBackChunk[kTileCfgs] = {8, 16, 32};
constexpr int kFadjChunk[kTileCfgs] = {4, 8, 16};

template <typename T, int BEAM>
void launch_back_tile(int cfg, const GeomK<float> &K, dim3 tg, dim3 tb, const T *src, T *dst, const Epi &e,
                      cudaStream_t s) {
  if (cfg == 0) k_back_tile<T, 8, BEAM><<<tg, tb, 0, s>>>(K, src, dst, e);
  else if (cfg == 1) k_back_tile<T, 16, BEAM><<<tg, tb, 0, s>>>(K, src, dst, e);
  else k_back_tile<T, 32, BEAM><<<tg, tb, 0, s>>>(K, src, dst, e);
}

template <typename T>
void launch_tile(int op, int cfg, const GeomK<float> &K, dim3 tg, const void *in, void *out, const Epi &e,
                 cudaStream_t s) {
  const dim3 tb(32, 8);
  const T *src = static_cast<const T *>(in);
  T *dst = static_cast<T *>(out);
  if (op == 1) {
    if (K.beam == 0) launch_back_tile<T, 0>(cfg, K, tg, tb, src, dst, e, s);
    else if (K.beam == 1) launch_back_tile<T, 1>(cfg, K, tg, tb, src, dst, e, s);
    else launch_back_tile<T, 2>(cfg, K, tg, tb, src, dst, e, s);
  } else {
    if (cfg == 0) k_fadj_tile<T, 4><<<tg, tb, 0, s>>>(K, src, dst, e);
    else if (cfg == 1) k_fadj_tile<T, 8><<<tg, tb, 0, s>>>(K, src, dst, e);
    else k_fadj_tile<T, 16><<<tg, tb, 0, s>>>(K, src, dst, e);
  }
}

template <typename T>
void launch_fadj_scatter(int cfg, const GeomK<float> &K, const uint32_t *swin, dim3 sg, const void *in, void *out,
                         const Epi &e, cudaStream_t s) {
  const T *src = static_cast<const T *>(in);
  T *dst = static_cast<T *>(out);
  if (cfg == 0) k_fadj_scatter<T, 8><<<sg, 128, fadj_scatter_smem<T, 8>(), s>>>(K, swin, src, dst, e);
  else if (cfg == 1) k_fadj_scatter<T, 16><<<sg, 128, fadj_scatter_smem<T, 16>(), s>>>(K, swin, src, dst, e);
  else k_fadj_scatter<T, 24><<<sg, 128, fadj_scatter_smem<T, 24>(), s>>>(K, swin, src, dst, e);
}

template <typename T>
gkb_status launch_badj_scatter(const gkb_geometry *g, const void *in, void *out, const Epi &e, cudaStream_t s) {
  const FastPlan &F = g->fast;
  const long long n = g->n, m = g->m;
  void *acc = e.scratch_acc;
  const size_t bytes = (size_t)m * 8 + 256;
  bool own = false;
  if (!acc) {
    GKB_CUDA_TRY(cudaMallocAsync(&acc, bytes, s));
    GKB_CUDA_TRY(cudaMemsetAsync(acc, 0, bytes, s));
    own = true;
  }
  unsigned long long *acc64 = static_cast<unsigned long long *>(acc);
  unsigned *mx = reinterpret_cast<unsigned *>(acc64 + m);
  GKB_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned), s));
  const int gmax = (int)std::min<long long>((n + 1023) / 1024, 1184);
  k_absmax<T><<<std::max(gmax, 1), 256, 0, s>>>(static_cast<const T *>(in), n, mx, e);
  const int tiles_x = (g->desc.nx + BS - 1) / BS, tiles_y = (g->desc.ny + BS - 1) / BS;
  int log2n = 10;   // at least the tile's pixel count, so a tile sum alone cannot overflow either
  while ((1LL << log2n) < n) ++log2n;
  const GeomK<float> K = geom_view<float>(g);
  const dim3 sg(tiles_x * tiles_y, F.bs_groups);
  const T *src = static_cast<const T *>(in);
  if (K.beam == 0) k_badj_scatter<T, 0><<<sg, 256, 0, s>>>(K, src, mx, F.bs_wmax, F.bs_pmax, log2n, tiles_x, acc64, e);
  else if (K.beam == 1) k_badj_scatter<T, 1><<<sg, 256, 0, s>>>(K, src, mx, F.bs_wmax, F.bs_pmax, log2n, tiles_x, acc64, e);
  else k_badj_scatter<T, 2><<<sg, 256, 0, s>>>(K, src, mx, F.bs_wmax, F.bs_pmax, log2n, tiles_x, acc64, e);
  const int gfin = (int)std::max<long long>(1, std::min<long long>((m + 255) / 256, 1184));
  k_badj_finish<T><<<gfin, 256, 0, s>>>(m, acc64, mx, F.bs_wmax, log2n, static_cast<T *>(out), e);
  GKB_CUDA_TRY(cudaGetLastError());
  if (own) GKB_CUDA_TRY(cudaFreeAsync(acc, s));
  return GKB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// plan of the fast paths (built with the geometry, host FP64)

namespace {

void ray_host(const gkb_geometry_desc &d, double c, double s, double bin, double &px, double &py, double &ex,
              double &ey) {
  const double u = (bin - 0.5 * (d.n_det - 1)) * d.det_width;
  if (d.beam == GKB_PARALLEL) {
    px = u * c; py = u * s; ex = -s; ey = c;
    return;
  }
  if (d.beam == GKB_FAN_ARC) {
    const double gm = u / d.sdd, cg = std::cos(gm), sg = std::sin(gm);
    px = d.sod * c; py = d.sod * s; ex = -c * cg - s * sg; ey = -s * cg + c * sg;
    return;
  }
  const double sx = d.sod * c, sy = d.sod * s;
  const double bx = -(d.sdd - d.sod) * c - u * s, by = -(d.sdd - d.sod) * s + u * c;
  const double lx = bx - sx, ly = by - sy, L = std::sqrt(lx * lx + ly * ly);
  px = sx; py = sy; ex = lx / L; ey = ly / L;
}

// interpolation coordinate of a ray (or strip boundary at fractional bin) at stepping index k
double coord_host(const gkb_geometry_desc &d, double c, double s, double bin, int axis, double k) {
  double px, py, ex, ey;
  ray_host(d, c, s, bin, px, py, ex, ey);
  const double pix = d.pixel, hx = 0.5 * (d.nx - 1), hy = 0.5 * (d.ny - 1);
  if (axis == 0) return (px + ((hy - k) * pix - py) * ex / ey) / pix + hx;
  return hy - (py + ((k - hx) * pix - px) * ey / ex) / pix;
}

int axis_host(const gkb_geometry_desc &d, double c, double s, int bin) {
  double px, py, ex, ey;
  ray_host(d, c, s, bin, px, py, ex, ey);
  return std::fabs(ey) >= std::fabs(ex) ? 0 : 1;
}

// Width (in pixels) of the band footprint of bins [b0, b1] (fractional bins
// allowed, for strip boundaries) over every band of the walk.
double footprint(const gkb_geometry_desc &d, double c, double s, double b0, double b1, int axis) {
  const int rows = axis ? d.nx : d.ny;
  double worst = 0.0;
  for (int k = 0; k < rows; k += kFootRows / 2) {
    const int k1 = k + kFootRows - 1;
    const double v[4] = {coord_host(d, c, s, b0, axis, k), coord_host(d, c, s, b0, axis, k1),
                         coord_host(d, c, s, b1, axis, k), coord_host(d, c, s, b1, axis, k1)};
    const double lo = std::min(std::min(v[0], v[1]), std::min(v[2], v[3]));
    const double hi = std::max(std::max(v[0], v[1]), std::max(v[2], v[3]));
    worst = std::max(worst, hi - lo);
  }
  return worst;
}

void build_items(const gkb_geometry_desc &d, const std::vector<double> &ang, bool strip, std::vector<int4> &out,
                 bool &any_axis1, bool &ok) {
  const double slack = strip ? 12.0 : 8.0;   // floor, neighbour, 16-byte alignment, strip margins
  for (int a = 0; a < d.n_angles && ok; ++a) {
    const double c = std::cos(ang[a]), s = std::sin(ang[a]);
    int b = 0;
    while (b < d.n_det) {
      const int ax = axis_host(d, c, s, b);
      int e = b;
      while (e + 1 < d.n_det && axis_host(d, c, s, e + 1) == ax) ++e;
      // split [b, e] into items whose footprint fits a box
      int start = b;
      while (start <= e) {
        int nb = std::min(kBandRays, e - start + 1);
        while (nb > 1) {
          const double lo = strip ? start - 1.0 : start, hi = strip ? start + nb : start + nb - 1.0;
          if (footprint(d, c, s, lo, hi, ax) + slack <= kBoxW) break;
          nb = std::max(1, nb * 3 / 4);
        }
        const double lo = strip ? start - 1.0 : start, hi = strip ? start + nb : start + nb - 1.0;
        if (footprint(d, c, s, lo, hi, ax) + slack > kBoxW) { ok = false; return; }
        out.push_back(make_int4(a, start, nb, ax));
        if (ax) any_axis1 = true;
        start += nb;
      }
      b = e + 1;
    }
  }
}

// Largest window (in bins) any tw x th tile spans at any angle, for B and A^T.
void tile_windows(const gkb_geometry &g, double &winB, double &winA, int TX = gkb::TX, int TY = gkb::TY) {
  const gkb_geometry_desc &d = g.desc;
  const double hx = 0.5 * (d.nx - 1), hy = 0.5 * (d.ny - 1), pix = d.pixel;
  winB = winA = 0.0;
  const int tilesx = (d.nx + TX - 1) / TX, tilesy = (d.ny + TY - 1) / TY;
  for (int a = 0; a < d.n_angles; ++a) {
    const double c = std::cos(g.angles[a]), s = std::sin(g.angles[a]);
    const double R = std::max(std::fabs(c), std::fabs(s)) * pix / d.det_width;
    const bool par = d.beam == GKB_PARALLEL;
    const int step_x = par ? tilesx : 1, step_y = par ? tilesy : 1;  // parallel: every tile alike
    for (int ty = 0; ty < tilesy; ty += step_y)
      for (int tx = 0; tx < tilesx; tx += step_x) {
        double tmin = 1e300, tmax = -1e300, amin = 1e300, amax = -1e300;
        const double x0 = tx * TX - hx, x1 = tx * TX + TX - 1 - hx, y0 = hy - (ty * TY + TY - 1), y1 = hy - ty * TY;
        bool behind = false;
        for (int k = 0; k < 4; ++k) {
          const double xr = (k & 1) ? x1 : x0, yr = (k & 2) ? y1 : y0;
          double t;
          if (par) {
            t = (xr * c + yr * s) * pix / d.det_width + 0.5 * (d.n_det - 1);
          } else {
            const double U = d.sod / pix - (xr * c + yr * s), L = -xr * s + yr * c;
            if (!(U > 0.0)) behind = true;
            t = d.sdd / d.det_width * (d.beam == GKB_FAN_ARC ? std::atan2(L, U) : L / U) + 0.5 * (d.n_det - 1);
            amin = std::min(amin, L / U);
            amax = std::max(amax, L / U);
          }
          tmin = std::min(tmin, t);
          tmax = std::max(tmax, t);
        }
        winB = std::max(winB, tmax - tmin + 4.0);
        // A^T: the rays within one pixel of the tile's pixels (as ray_range_rect)
        double lo = tmin - R, hi = tmax + R;
        if (!par) {
          const double xs = d.sod / pix * c, ys = d.sod / pix * s;
          const double dx = xs - std::min(std::max(xs, x0), x1), dy = ys - std::min(std::max(ys, y0), y1);
          const double r2 = dx * dx + dy * dy;
          if (behind || !(r2 > 1.0)) {
            lo = -1e30;
            hi = 1e30;
          } else if (d.beam == GKB_FAN_ARC) {
            const double dg = std::asin(1.0 / std::sqrt(r2)), g2 = d.sdd / d.det_width, t0 = 0.5 * (d.n_det - 1);
            hi = g2 * (std::atan(amax) + dg) + t0;
            lo = g2 * (std::atan(amin) - dg) + t0;
          } else {
            const double q = 1.0 / std::sqrt(r2 - 1.0), g2 = d.sdd / d.det_width, t0 = 0.5 * (d.n_det - 1);
            hi = 1.0 - amax * q > 0.0 ? g2 * (amax + q) / (1.0 - amax * q) + t0 : 1e30;
            lo = 1.0 + amin * q > 0.0 ? g2 * (amin - q) / (1.0 + amin * q) + t0 : -1e30;
          }
        }
        winA = std::max(winA, hi - lo + 5.0);
      }
  }
}

}  // namespace

template <typename T, int R, int S>
void set_band_smem_shape() {
  const int smem = S * R * kBoxW * (int)sizeof(T);
  cudaFuncSetAttribute(k_forward_band<T, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_badj_band<T, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <typename T>
void set_scatter_smem() {
  cudaFuncSetAttribute(k_fadj_scatter<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fadj_scatter_smem<T, 8>());
  cudaFuncSetAttribute(k_fadj_scatter<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fadj_scatter_smem<T, 16>());
  cudaFuncSetAttribute(k_fadj_scatter<T, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fadj_scatter_smem<T, 24>());
}
template <typename T>
void set_band_smem() {
  set_band_smem_shape<T, 8, 2>();
  set_band_smem_shape<T, 8, 3>();
  set_band_smem_shape<T, 16, 2>();
  set_band_smem_shape<T, 16, 3>();
  set_band_smem_shape<T, 32, 2>();
}

gkb_status use_scatter(gkb_geometry *g, bool enable) {
  FastPlan &F = g->fast;
  if (F.scatter != enable) {
    F.scatter = enable;
    F.cfg_fadj = 1;
    F.cfg_badj = 2;
    F.tuned = false;
  }
  return GKB_OK;
}

void build_fast_plan(gkb_geometry *g) {
  static bool attrs = false;
  if (!attrs) {
    attrs = true;
    set_band_smem<float>();
    set_band_smem<__nv_bfloat16>();
    set_band_smem<__half>();
    set_scatter_smem<float>();
    set_scatter_smem<__nv_bfloat16>();
    set_scatter_smem<__half>();
    cudaGetLastError();
  }
  FastPlan &F = g->fast;
  const gkb_geometry_desc &d = g->desc;
  double wb, wa;
  tile_windows(*g, wb, wa);
  F.tile_back = wb <= kWinB;
  F.tile_fadj = wa <= kWinA;
  {  // B^T scatter: windows of 32x32 tiles, weight bound, grid shape
    double wb2, wa2;
    tile_windows(*g, wb2, wa2, BS, BS);
    F.bscatter = wb2 + 4.0 <= kWinB2;
    const double pix = d.pixel;
    if (d.beam == GKB_PARALLEL) {
      F.bs_wmax = (float)(pix * pix / d.det_width * 1.0001);
    } else {
      const double rimg = std::sqrt(0.25 * (d.nx - 1.0) * (d.nx - 1.0) + 0.25 * (d.ny - 1.0) * (d.ny - 1.0));
      const double umin = d.sod / pix - rimg, wpix = pix * d.sdd / d.det_width;
      // flat: w = wpix rho / U^2 <= wpix (1/U + |L|/U^2); arc: w = wpix / rho
      F.bs_wmax = umin > 0.5 ? (float)((d.beam == GKB_FAN_ARC ? wpix / umin
                                                                : wpix * (1.0 / umin + rimg / (umin * umin))) * 1.01)
                             : 0.f;
      if (!(F.bs_wmax > 0.f)) F.bscatter = false;
    }
    // pixels of one tile that can add into one bin: the tile's intersection
    // with a strip two bins wide, the bins measured where they are widest
    const double rimg2 = std::sqrt(0.25 * (d.nx - 1.0) * (d.nx - 1.0) + 0.25 * (d.ny - 1.0) * (d.ny - 1.0));
    const double bw = d.beam == GKB_PARALLEL ? d.det_width / pix : d.det_width / pix * (d.sod / pix + rimg2) * pix / d.sdd;
    F.bs_pmax = (float)std::min((double)(BS * BS), std::ceil(1.25 * BS * std::sqrt(2.0) * (2.0 * bw + 2.0)));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaGetLastError();
    const long long tiles = (long long)((d.nx + BS - 1) / BS) * ((d.ny + BS - 1) / BS);
    const long long want = 4LL * sms * 6;
    F.bs_groups = (int)std::max(1LL, std::min((long long)d.n_angles, (want + tiles - 1) / tiles));
  }
  tile_windows(*g, wb, wa, SW, SW);
  F.tile_scatter = wa + 4.0 <= kWinS && d.n_det < (1 << 20);
  if (F.tile_scatter) {
    const int tsx = (d.nx + SW - 1) / SW, tsy = (d.ny + SW - 1) / SW;
    const long long pairs = (long long)tsx * tsy * d.n_angles;
    int *bad = nullptr;
    if (cudaMalloc(&F.swin, pairs * sizeof(uint32_t)) == cudaSuccess && cudaMalloc(&bad, sizeof(int)) == cudaSuccess) {
      cudaMemset(bad, 0, sizeof(int));
      k_scatter_windows<<<(unsigned)((pairs + 3) / 4), 128>>>(geom_view<float>(g), F.swin, tsx, pairs, bad);
      int hbad = 1;
      if (cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || hbad) {
        cudaFree(F.swin);
        F.swin = nullptr;
      }
    }
    if (bad) cudaFree(bad);
    cudaGetLastError();
    F.tile_scatter = F.swin != nullptr;
  }
  F.tuned = false;
  std::vector<int4> fwd, badj;
  bool ok = true, any1 = false;
  build_items(d, g->angles, false, fwd, any1, ok);
  if (ok) build_items(d, g->angles, true, badj, any1, ok);
  F.any_axis1 = any1;
  F.band = ok && !fwd.empty() && !badj.empty() && encode_fn() != nullptr;
  if (F.band) {
    if (cudaMalloc(&F.items_fwd, fwd.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&F.items_badj, badj.size() * sizeof(int4)) != cudaSuccess) {
      cudaGetLastError();
      F.band = false;
      return;
    }
    cudaMemcpy(F.items_fwd, fwd.data(), fwd.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(F.items_badj, badj.data(), badj.size() * sizeof(int4), cudaMemcpyHostToDevice);
    F.n_fwd = (int)fwd.size();
    F.n_badj = (int)badj.size();
  }
}

void free_fast_plan(gkb_geometry *g) {
  FastPlan &F = g->fast;
  if (F.items_fwd) cudaFree(F.items_fwd);
  if (F.items_badj) cudaFree(F.items_badj);
  if (F.swin) cudaFree(F.swin);
  F = FastPlan{};
}

bool band_ok_for(const gkb_geometry *g, gkb_dtype dt) {
  const FastPlan &F = g->fast;
  if (!F.band || dt == GKB_F64) return false;
  const int align = dt == GKB_F32 ? 4 : 8;   // 16-byte row strides for the tensor maps
  return g->desc.nx % align == 0 && g->desc.ny % align == 0;
}

gkb_status launch_fast(int op, const gkb_geometry *g, gkb_dtype dt, const void *in, void *out, void *scratch_t,
                       const Epi &e, cudaStream_t s, bool &handled) {
  handled = false;
  if (dt == GKB_F64) return GKB_OK;
  const GeomK<float> K = geom_view<float>(g);
  const FastPlan &F = g->fast;
  dim3 tb(32, 8), tg((g->desc.nx + TX - 1) / TX, (g->desc.ny + TY - 1) / TY);
  gkb_status st = GKB_OK;
  switch (op) {
    case 1:    // B
    case 2: {  // A^T
      if (op == 1 ? !F.tile_back : !F.tile_fadj) return GKB_OK;
      handled = true;
      const int cfg = op == 1 ? F.cfg_back : F.cfg_fadj;
      if (op == 2 && F.swin && F.scatter) {
        const dim3 sg((g->desc.nx + SW - 1) / SW, (g->desc.ny + SW - 1) / SW);
        if (dt == GKB_F32) launch_fadj_scatter<float>(cfg, K, F.swin, sg, in, out, e, s);
        else if (dt == GKB_BF16) launch_fadj_scatter<__nv_bfloat16>(cfg, K, F.swin, sg, in, out, e, s);
        else launch_fadj_scatter<__half>(cfg, K, F.swin, sg, in, out, e, s);
        break;
      }
      if (dt == GKB_F32) launch_tile<float>(op, cfg, K, tg, in, out, e, s);
      else if (dt == GKB_BF16) launch_tile<__nv_bfloat16>(op, cfg, K, tg, in, out, e, s);
      else launch_tile<__half>(op, cfg, K, tg, in, out, e, s);
      break;
    }
    case 3:  // B^T
      if (F.bscatter && F.scatter) {
        handled = true;
        if (dt == GKB_F32) st = launch_badj_scatter<float>(g, in, out, e, s);
        else if (dt == GKB_BF16) st = launch_badj_scatter<__nv_bfloat16>(g, in, out, e, s);
        else st = launch_badj_scatter<__half>(g, in, out, e, s);
        break;
      }
      [[fallthrough]];
    case 0:  // A
      if (!band_ok_for(g, dt)) return GKB_OK;
      handled = true;
      if (dt == GKB_F32) st = launch_band<float>(op == 0 ? 0 : 1, g, in, out, scratch_t, e, s);
      else if (dt == GKB_BF16) st = launch_band<__nv_bfloat16>(op == 0 ? 0 : 1, g, in, out, scratch_t, e, s);
      else st = launch_band<__half>(op == 0 ? 0 : 1, g, in, out, scratch_t, e, s);
      return st;
  }
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time every shape of each fast kernel once per geometry shape and
// storage type, keep the fastest.  The shapes change only how work is split
// (angle chunks of the tiles, band height and TMA ring depth), never the
// arithmetic, so any choice gives the same results bit for bit.

namespace {
struct TuneKey {
  int beam, nx, ny, na, nd, dt, mapped;
  long long dw, sod, sdd, a0, a1;
  bool operator<(const TuneKey &o) const {
    return std::tie(beam, nx, ny, na, nd, dt, mapped, dw, sod, sdd, a0, a1) <
           std::tie(o.beam, o.nx, o.ny, o.na, o.nd, o.dt, o.mapped, o.dw, o.sod, o.sdd, o.a0, o.a1);
  }
};
struct TuneVal { int back, fadj, fwd, badj; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

TuneKey tune_key(const gkb_geometry *g, gkb_dtype dt) {
  const gkb_geometry_desc &d = g->desc;
  auto q = [](double v) { return (long long)llround(v * 1e6); };
  return TuneKey{d.beam, d.nx, d.ny, d.n_angles, d.n_det, (int)dt, g->fast.scatter ? 1 : 0, q(d.det_width / d.pixel),
                 q(d.sod / d.pixel),
                 q(d.sdd / d.pixel), q(g->angles.front()), q(g->angles.back())};
}
}  // namespace

gkb_status autotune(gkb_geometry *g, gkb_dtype dt) {
  if (dt == GKB_F64) return GKB_OK;
  FastPlan &F = g->fast;
  if (F.tuned) return GKB_OK;
  const TuneKey key = tune_key(g, dt);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      F.cfg_back = it->second.back; F.cfg_fadj = it->second.fadj;
      F.cfg_fwd = it->second.fwd; F.cfg_badj = it->second.badj;
      F.tuned = true;
      return GKB_OK;
    }
  }
  const size_t ts = dtype_size(dt);
  void *x = nullptr, *y = nullptr, *xt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gkb_status st = GKB_OK;
  if (cudaMalloc(&x, ts * g->n) != cudaSuccess || cudaMalloc(&y, ts * g->m) != cudaSuccess ||
      cudaMalloc(&xt, ts * g->n) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    st = GKB_ERR_OOM;
  if (st == GKB_OK) {
    cudaMemset(x, 0, ts * g->n);
    cudaMemset(y, 0, ts * g->m);
  }
  auto time_op = [&](int op) -> float {
    Epi e;
    e.scratch_t = xt;
    bool handled = false;
    const void *in = (op == 0 || op == 3) ? x : y;
    void *out = (op == 0 || op == 3) ? y : x;
    launch_fast(op, g, dt, in, out, xt, e, nullptr, handled);  // warm-up
    float best = 3.0e38f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, nullptr);
      launch_fast(op, g, dt, in, out, xt, e, nullptr, handled);
      cudaEventRecord(e1, nullptr);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return handled ? best : 3.0e38f;
  };
  if (st == GKB_OK) {
    int *cfgs[4] = {&F.cfg_fwd, &F.cfg_back, &F.cfg_fadj, &F.cfg_badj};
    const int counts[4] = {kBandCfgs, kTileCfgs, kTileCfgs, kBandCfgs};
    for (int op = 0; op < 4; ++op) {
      int best_c = *cfgs[op];
      float best_t = 3.0e38f;
      for (int c = 0; c < counts[op]; ++c) {
        *cfgs[op] = c;
        const float t = time_op(op);
        if (t < best_t) { best_t = t; best_c = c; }
      }
      *cfgs[op] = best_c;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) st = GKB_ERR_CUDA;
  }
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (xt) cudaFree(xt);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (st != GKB_OK) return st;
  F.tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = TuneVal{F.cfg_back, F.cfg_fadj, F.cfg_fwd, F.cfg_badj};
  return GKB_OK;
}

void get_shapes(const gkb_geometry *g, int shapes[4], int counts[4]) {
  const FastPlan &F = g->fast;
  const int sh[4] = {F.cfg_fwd, F.cfg_back, F.cfg_fadj, F.cfg_badj};
  const int ct[4] = {kBandCfgs, kTileCfgs, kTileCfgs, kBandCfgs};
  for (int i = 0; i < 4; ++i) {
    if (shapes) shapes[i] = sh[i];
    if (counts) counts[i] = ct[i];
  }
}

gkb_status set_shapes(gkb_geometry *g, const int shapes[4]) {
  const int ct[4] = {kBandCfgs, kTileCfgs, kTileCfgs, kBandCfgs};
  for (int i = 0; i < 4; ++i)
    if (shapes[i] < 0 || shapes[i] >= ct[i]) return GKB_ERR_INVALID_ARG;
  FastPlan &F = g->fast;
  F.cfg_fwd = shapes[0];
  F.cfg_back = shapes[1];
  F.cfg_fadj = shapes[2];
  F.cfg_badj = shapes[3];
  F.tuned = true;
  return GKB_OK;
}

long long fast_blocks(const gkb_geometry *g) {
  const FastPlan &F = g->fast;
  long long t = (long long)((g->desc.nx + TX - 1) / TX) * ((g->desc.ny + TY - 1) / TY);
  t = std::max(t, (long long)((g->desc.nx + SW - 1) / SW) * ((g->desc.ny + SW - 1) / SW));
  return std::max({t, (long long)F.n_fwd, (long long)F.n_badj});
}

}  // namespace gkb

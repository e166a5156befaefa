// The four projector kernels and their entry points.
//
//   A   (projector_forward)         one thread per ray: Joseph's method.
//   B   (projector_back)            one thread per pixel: pixel-driven linear
//                                   interpolation over the detector.
//   A^T (projector_forward_adjoint) one thread per pixel: gathers, for every
//                                   angle, the few rays whose Joseph weight
//                                   on this pixel is non-zero, with the
//                                   weight A uses.
//   B^T (projector_back_adjoint)    one thread per ray: gathers the pixels of
//                                   the strip whose pixel-driven weight on
//                                   this bin is non-zero, with the weight B uses.
//
// A and A^T evaluate each ray's interpolation coordinate with the same
// correctly rounded expression (ray_coord), and B and B^T evaluate each
// pixel's bin coordinate and weight with the same function (pixel_bin), so
// each pair is an exact transpose up to the order of the floating-point sums.
#include <algorithm>
#include <cstdlib>

#include "fast.h"

namespace gkb {

namespace {

constexpr int kRayBlock = 128;
constexpr int kPixBX = 16, kPixBY = 16;

template <typename T, typename C>
__device__ __forceinline__ void epilogue(bool valid, long long idx, C v, T *__restrict__ out, const Epi &e,
                                         double *sh) {
  double sq = 0.0;
  if (valid) {
    const double os = (double)epi_store<T, C>(e, idx, v, out);
    sq = os * os;
  }
  if (e.partials) grid_sum_finalize(sq, e.partials, e.counter, e.result, sh);
}

// rows (or columns) k in [0, kmax) for which J0 + k*Js lies in (-1, lim),
// widened by one on each side; the per-step bounds checks stay exact.
template <typename C>
__device__ __forceinline__ void step_range(C J0, C Js, int lim, int kmax, int &k0, int &k1) {
  const C lo_c = C(-1), hi_c = C(lim);
  if (abs_(Js) < C(1e-30)) {
    if (J0 > lo_c - C(1) && J0 < hi_c + C(1)) { k0 = 0; k1 = kmax - 1; }
    else { k0 = 0; k1 = -1; }
    return;
  }
  C a = (lo_c - J0) / Js, b = (hi_c - J0) / Js;
  if (a > b) { C t = a; a = b; b = t; }
  a = a < C(-2) ? C(-2) : (a > C(kmax + 1) ? C(kmax + 1) : a);
  b = b < C(-2) ? C(-2) : (b > C(kmax + 1) ? C(kmax + 1) : b);
  k0 = (int)floor_(a) - 1;
  k1 = (int)floor_(b) + 1;
  if (k0 < 0) k0 = 0;
  if (k1 > kmax - 1) k1 = kmax - 1;
}

// ---------------------------------------------------------------------------
// A: Joseph forward projection, one thread per ray

template <typename T, typename C>
__global__ void __launch_bounds__(kRayBlock) k_forward(GeomK<C> G, const T *__restrict__ x, T *__restrict__ y, Epi e) {
  if (e.done && *e.done) return;
  __shared__ double sh[32];
  const long long m = (long long)G.na * G.nd;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < m;
  C v = C(0);
  if (valid) {
    const RayP<C> ray = G.ray[r];
    const int nx = G.nx, ny = G.ny;
    C acc = C(0);
    if (ray.axis == C(0)) {
      int k0, k1;
      step_range(ray.J0, ray.Js, nx, ny, k0, k1);
      for (int i = k0; i <= k1; ++i) {
        const C jf = ray_coord(ray, i);
        const C fl = floor_(jf);
        if (!(fl >= C(-1) && fl <= C(nx - 1))) continue;
        const C f = jf - fl;
        const int j = (int)fl;
        const T *row = x + (long long)i * nx;
        const C a = (j >= 0) ? to_c(row[j]) : C(0);
        const C b = (j + 1 < nx) ? to_c(row[j + 1]) : C(0);
        acc += (C(1) - f) * a + f * b;
      }
    } else {
      int k0, k1;
      step_range(ray.J0, ray.Js, ny, nx, k0, k1);
      for (int j = k0; j <= k1; ++j) {
        const C fi = ray_coord(ray, j);
        const C fl = floor_(fi);
        if (!(fl >= C(-1) && fl <= C(ny - 1))) continue;
        const C f = fi - fl;
        const int i = (int)fl;
        const C a = (i >= 0) ? to_c(x[(long long)i * nx + j]) : C(0);
        const C b = (i + 1 < ny) ? to_c(x[(long long)(i + 1) * nx + j]) : C(0);
        acc += (C(1) - f) * a + f * b;
      }
    }
    v = acc * ray.scale;
  }
  epilogue<T, C>(valid, r, v, y, e, sh);
}

// ---------------------------------------------------------------------------
// A^T: pixel-driven gather of Joseph weights

template <typename T, typename C>
__global__ void __launch_bounds__(kPixBX *kPixBY) k_forward_adj(GeomK<C> G, const T *__restrict__ y, T *__restrict__ x, Epi e) {
  if (e.done && *e.done) return;
  __shared__ double sh[32];
  const int j = blockIdx.x * kPixBX + threadIdx.x;
  const int i = blockIdx.y * kPixBY + threadIdx.y;
  const bool valid = (i < G.ny) && (j < G.nx);
  C acc = C(0);
  if (valid) {
    const C xr = C(j) - G.hx, yr = G.hy - C(i);
    const C Ci = C(i), Cj = C(j);
    for (int a = 0; a < G.na; ++a) {
      const AngleP<C> A = G.ang[a];
      C lo, hi;
      ray_range(G, A, xr, yr, lo, hi);
      C dlo = ceil_(lo), dhi = floor_(hi);
      dlo = min_(max_(dlo, C(0)), C(G.nd));
      dhi = min_(max_(dhi, C(-1)), C(G.nd - 1));
      const RayP<C> *rays = G.ray + (long long)a * G.nd;
      const T *ya = y + (long long)a * G.nd;
      for (int d = (int)dlo; d <= (int)dhi; ++d) {
        const RayP<C> r = rays[d];
        C wt = C(0);
        if (r.axis == C(0)) {
          const C jf = ray_coord(r, i);
          const C fl = floor_(jf);
          const C f = jf - fl;
          if (fl == Cj) wt = C(1) - f;
          else if (fl + C(1) == Cj) wt = f;
        } else {
          const C fi = ray_coord(r, j);
          const C fl = floor_(fi);
          const C f = fi - fl;
          if (fl == Ci) wt = C(1) - f;
          else if (fl + C(1) == Ci) wt = f;
        }
        acc += wt * r.scale * to_c(ya[d]);
      }
    }
  }
  epilogue<T, C>(valid, (long long)i * G.nx + j, acc, x, e, sh);
}

// ---------------------------------------------------------------------------
// B: pixel-driven back projection

template <typename T, typename C>
__global__ void __launch_bounds__(kPixBX *kPixBY) k_back(GeomK<C> G, const T *__restrict__ y, T *__restrict__ x, Epi e) {
  if (e.done && *e.done) return;
  __shared__ double sh[32];
  const int j = blockIdx.x * kPixBX + threadIdx.x;
  const int i = blockIdx.y * kPixBY + threadIdx.y;
  const bool valid = (i < G.ny) && (j < G.nx);
  C acc = C(0);
  if (valid) {
    const C xr = C(j) - G.hx, yr = G.hy - C(i);
    const C lim = C(G.nd - 1);
    for (int a = 0; a < G.na; ++a) {
      C t, w;
      pixel_bin(G, G.ang[a], xr, yr, t, w);
      const C fl = floor_(t);
      if (!(fl >= C(-1) && fl <= lim)) continue;
      const C f = t - fl;
      const int d = (int)fl;
      const T *row = y + (long long)a * G.nd;
      const C v0 = (d >= 0) ? to_c(row[d]) : C(0);
      const C v1 = (d + 1 < G.nd) ? to_c(row[d + 1]) : C(0);
      acc += w * ((C(1) - f) * v0 + f * v1);
    }
  }
  epilogue<T, C>(valid, (long long)i * G.nx + j, acc, x, e, sh);
}

// ---------------------------------------------------------------------------
// B^T: ray-driven gather of pixel-driven weights

template <typename T, typename C>
__device__ __forceinline__ void bt_accumulate(const GeomK<C> &G, const AngleP<C> &A, int i, int j, int d,
                                              const T *__restrict__ x, C &acc) {
  C t, w;
  pixel_bin(G, A, C(j) - G.hx, G.hy - C(i), t, w);
  const C fl = floor_(t);
  const C f = t - fl;
  C wt = C(0);
  if (fl == C(d)) wt = C(1) - f;
  else if (fl + C(1) == C(d)) wt = f;
  if (wt != C(0)) acc += w * wt * to_c(x[(long long)i * G.nx + j]);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kRayBlock) k_back_adj(GeomK<C> G, const T *__restrict__ x, T *__restrict__ y, Epi e) {
  if (e.done && *e.done) return;
  __shared__ double sh[32];
  const long long m = (long long)G.na * G.nd;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < m;
  C acc = C(0);
  if (valid) {
    const int a = (int)(r / G.nd), d = (int)(r - (long long)a * G.nd);
    const AngleP<C> A = G.ang[a];
    C km = C(d - 1) - G.t0, kp = C(d + 1) - G.t0;   // bin offsets of the strip edges
    const C marg = C(0.01);
    if (G.beam == 0) {
      if (abs_(A.cu) >= abs_(A.su)) {
        const C inv = C(1) / A.cu;
        for (int i = 0; i < G.ny; ++i) {
          const C yr = G.hy - C(i);
          C p = (km - yr * A.su) * inv, q = (kp - yr * A.su) * inv;
          if (p > q) { C t = p; p = q; q = t; }
          int j0 = (int)max_(ceil_(p + G.hx - marg), C(0));
          int j1 = (int)min_(floor_(q + G.hx + marg), C(G.nx - 1));
          for (int j = j0; j <= j1; ++j) bt_accumulate(G, A, i, j, d, x, acc);
        }
      } else {
        const C inv = C(1) / A.su;
        for (int j = 0; j < G.nx; ++j) {
          const C xr = C(j) - G.hx;
          C p = (km - xr * A.cu) * inv, q = (kp - xr * A.cu) * inv;   // yr interval
          if (p > q) { C t = p; p = q; q = t; }
          int i0 = (int)max_(ceil_(G.hy - q - marg), C(0));
          int i1 = (int)min_(floor_(G.hy - p + marg), C(G.ny - 1));
          for (int i = i0; i <= i1; ++i) bt_accumulate(G, A, i, j, d, x, acc);
        }
      }
    } else {
      const RayP<C> ray = G.ray[r];
      const C g = G.gfan;
      if (G.beam == 2) {
        // arc: the boundary of bin offset k leaves the source at the angle k/g,
        // i.e. on the flat-detector boundary of offset g tan(k/g)
        const C lim = C(1.5707963);
        km = g * tan(min_(max_(km / g, -lim), lim));
        kp = g * tan(min_(max_(kp / g, -lim), lim));
      }
      if (ray.axis == C(0)) {
        // row yr: xr = (k (sodp - yr s) - g yr c) / (k c - g s)
        const C dm = km * A.c - g * A.s, dp = kp * A.c - g * A.s;
        for (int i = 0; i < G.ny; ++i) {
          const C yr = G.hy - C(i);
          C p = (km * (G.sodp - yr * A.s) - g * yr * A.c) / dm;
          C q = (kp * (G.sodp - yr * A.s) - g * yr * A.c) / dp;
          if (p > q) { C t = p; p = q; q = t; }
          int j0 = (int)max_(ceil_(p + G.hx - marg), C(0));
          int j1 = (int)min_(floor_(q + G.hx + marg), C(G.nx - 1));
          for (int j = j0; j <= j1; ++j) bt_accumulate(G, A, i, j, d, x, acc);
        }
      } else {
        // column xr: yr = (k (sodp - xr c) + g xr s) / (g c + k s)
        const C dm = g * A.c + km * A.s, dp = g * A.c + kp * A.s;
        for (int j = 0; j < G.nx; ++j) {
          const C xr = C(j) - G.hx;
          C p = (km * (G.sodp - xr * A.c) + g * xr * A.s) / dm;
          C q = (kp * (G.sodp - xr * A.c) + g * xr * A.s) / dp;
          if (p > q) { C t = p; p = q; q = t; }
          int i0 = (int)max_(ceil_(G.hy - q - marg), C(0));
          int i1 = (int)min_(floor_(G.hy - p + marg), C(G.ny - 1));
          for (int i = i0; i <= i1; ++i) bt_accumulate(G, A, i, j, d, x, acc);
        }
      }
    }
  }
  epilogue<T, C>(valid, r, acc, y, e, sh);
}

// ---------------------------------------------------------------------------
// launchers

dim3 ray_grid(const gkb_geometry *g) { return dim3((unsigned)((g->m + kRayBlock - 1) / kRayBlock)); }
dim3 pix_grid(const gkb_geometry *g) {
  return dim3((g->desc.nx + kPixBX - 1) / kPixBX, (g->desc.ny + kPixBY - 1) / kPixBY);
}

enum Op { OP_A = 0, OP_B = 1, OP_AT = 2, OP_BT = 3 };

// GKB_GENERIC_PROJECTORS=1 selects the generic kernels (a debugging aid).
bool fast_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *s = getenv("GKB_GENERIC_PROJECTORS");
    v = (s && s[0] == '1') ? 0 : 1;
  }
  return v == 1;
}

template <typename T, typename C>
gkb_status launch_typed(Op op, const gkb_geometry *g, const void *in, void *out, const Epi &e, cudaStream_t s) {
  GeomK<C> K = geom_view<C>(g);
  const T *src = static_cast<const T *>(in);
  T *dst = static_cast<T *>(out);
  switch (op) {
    case OP_A: k_forward<T, C><<<ray_grid(g), kRayBlock, 0, s>>>(K, src, dst, e); break;
    case OP_BT: k_back_adj<T, C><<<ray_grid(g), kRayBlock, 0, s>>>(K, src, dst, e); break;
    case OP_B: k_back<T, C><<<pix_grid(g), dim3(kPixBX, kPixBY), 0, s>>>(K, src, dst, e); break;
    case OP_AT: k_forward_adj<T, C><<<pix_grid(g), dim3(kPixBX, kPixBY), 0, s>>>(K, src, dst, e); break;
  }
  GKB_CUDA_TRY(cudaGetLastError());
  return GKB_OK;
}

gkb_status launch(Op op, const gkb_geometry *g, gkb_dtype dt, const void *in, void *out, const Epi &e, cudaStream_t s) {
  if (!g || !in || !out || !dtype_valid(dt)) return GKB_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return GKB_ERR_INVALID_ARG;
  if (fast_enabled()) {
    bool handled = false;
    gkb_status st = launch_fast((int)op, g, dt, in, out, e.scratch_t, e, s, handled);
    if (handled || st != GKB_OK) return st;
  }
  switch (dt) {
    case GKB_F64: {
      gkb_status st = ensure_f64(const_cast<gkb_geometry *>(g));
      if (st != GKB_OK) return st;
      return launch_typed<double, double>(op, g, in, out, e, s);
    }
    case GKB_F32: return launch_typed<float, float>(op, g, in, out, e, s);
    case GKB_BF16: return launch_typed<__nv_bfloat16, float>(op, g, in, out, e, s);
    case GKB_F16: return launch_typed<__half, float>(op, g, in, out, e, s);
  }
  return GKB_ERR_INVALID_ARG;
}

}  // namespace

long long forward_blocks(const gkb_geometry *g) {
  return std::max((g->m + kRayBlock - 1) / kRayBlock, fast_blocks(g));
}
long long back_blocks(const gkb_geometry *g) {
  dim3 b = pix_grid(g);
  return std::max((long long)b.x * b.y, fast_blocks(g));
}

gkb_status launch_forward(const gkb_geometry *g, gkb_dtype dt, const void *x, void *y, const Epi &e, cudaStream_t s) {
  return launch(OP_A, g, dt, x, y, e, s);
}
gkb_status launch_back(const gkb_geometry *g, gkb_dtype dt, const void *y, void *x, const Epi &e, cudaStream_t s) {
  return launch(OP_B, g, dt, y, x, e, s);
}
gkb_status launch_forward_adj(const gkb_geometry *g, gkb_dtype dt, const void *y, void *x, const Epi &e, cudaStream_t s) {
  return launch(OP_AT, g, dt, y, x, e, s);
}
gkb_status launch_back_adj(const gkb_geometry *g, gkb_dtype dt, const void *x, void *y, const Epi &e, cudaStream_t s) {
  return launch(OP_BT, g, dt, x, y, e, s);
}

}  // namespace gkb

extern "C" gkb_status projector_forward(const gkb_geometry *g, const void *x, void *y, gkb_dtype dtype, void *stream) {
  return gkb::launch_forward(g, dtype, x, y, gkb::Epi{}, static_cast<cudaStream_t>(stream));
}
extern "C" gkb_status projector_back(const gkb_geometry *g, const void *y, void *x, gkb_dtype dtype, void *stream) {
  return gkb::launch_back(g, dtype, y, x, gkb::Epi{}, static_cast<cudaStream_t>(stream));
}
extern "C" gkb_status projector_forward_adjoint(const gkb_geometry *g, const void *y, void *x, gkb_dtype dtype,
                                                void *stream) {
  return gkb::launch_forward_adj(g, dtype, y, x, gkb::Epi{}, static_cast<cudaStream_t>(stream));
}
extern "C" gkb_status projector_back_adjoint(const gkb_geometry *g, const void *x, void *y, gkb_dtype dtype,
                                             void *stream) {
  return gkb::launch_back_adj(g, dtype, x, y, gkb::Epi{}, static_cast<cudaStream_t>(stream));
}

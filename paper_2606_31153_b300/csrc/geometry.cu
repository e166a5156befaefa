// Scan geometry: validation and the per-angle / per-ray device tables.
//
// Every ray of Joseph's projector is reduced, in FP64 on the host, to the
// affine map from the stepping index (image row or column) to the
// interpolation coordinate along the other axis, then rounded once to the
// table's type.  Both the forward kernel and its exact transpose evaluate
// that same map, so they use identical interpolation weights.
#include <cmath>
#include <cstring>
#include <new>

#include "fast.h"

namespace gkb {

static thread_local cudaError_t g_last_cuda = cudaSuccess;
cudaError_t last_cuda_error() { return g_last_cuda; }
void set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

size_t dtype_size(gkb_dtype dt) {
  switch (dt) {
    case GKB_F64: return 8;
    case GKB_F32: return 4;
    default: return 2;
  }
}
bool dtype_valid(int dt) { return dt >= GKB_F32 && dt <= GKB_F16; }

namespace {

struct HostRay { double px, py, ex, ey; };

HostRay ray_of(const gkb_geometry_desc &d, double c, double s, int bin) {
  const double u = (bin - 0.5 * (d.n_det - 1)) * d.det_width;
  if (d.beam == GKB_PARALLEL) return {u * c, u * s, -s, c};
  if (d.beam == GKB_FAN_ARC) {   // central direction -(c, s) turned by u / sdd towards (-s, c)
    const double gm = u / d.sdd, cg = std::cos(gm), sg = std::sin(gm);
    return {d.sod * c, d.sod * s, -c * cg - s * sg, -s * cg + c * sg};
  }
  const double sx = d.sod * c, sy = d.sod * s;
  const double bx = -(d.sdd - d.sod) * c - u * s, by = -(d.sdd - d.sod) * s + u * c;
  const double lx = bx - sx, ly = by - sy, L = std::sqrt(lx * lx + ly * ly);
  return {sx, sy, lx / L, ly / L};
}

template <typename C>
void build_tables(const gkb_geometry &g, std::vector<RayP<C>> &rays, std::vector<AngleP<C>> &angs) {
  const gkb_geometry_desc &d = g.desc;
  const double pix = d.pixel, hx = 0.5 * (d.nx - 1), hy = 0.5 * (d.ny - 1);
  rays.resize((size_t)d.n_angles * d.n_det);
  angs.resize(d.n_angles);
  for (int a = 0; a < d.n_angles; ++a) {
    const double c = std::cos(g.angles[a]), s = std::sin(g.angles[a]);
    AngleP<C> A;
    A.c = (C)c;
    A.s = (C)s;
    A.cu = (C)(c * pix / d.det_width);
    A.su = (C)(s * pix / d.det_width);
    // half-width (in bins) of the set of rays that can touch a pixel: a ray
    // reaches pixel centres within pixel*max(|c|,|s|) along the detector.
    A.R = (C)(std::max(std::fabs(c), std::fabs(s)) * pix / d.det_width * (1.0 + 1e-5) + 2e-3);
    angs[a] = A;
    for (int b = 0; b < d.n_det; ++b) {
      HostRay r = ray_of(d, c, s, b);
      RayP<C> R;
      if (std::fabs(r.ey) >= std::fabs(r.ex)) {
        // crossing of row i: x = px + (y_i - py) ex/ey, y_i = (hy - i) pix
        const double q = r.ex / r.ey;
        R.J0 = (C)((r.px + (hy * pix - r.py) * q) / pix + hx);
        R.Js = (C)(-q);
        R.scale = (C)(pix / std::fabs(r.ey));
        R.axis = (C)0;
      } else {
        // crossing of column j: y = py + (x_j - px) ey/ex, x_j = (j - hx) pix;
        // row coordinate hy - y/pix
        const double q = r.ey / r.ex;
        R.J0 = (C)(hy - (r.py + (-hx * pix - r.px) * q) / pix);
        R.Js = (C)(-q);
        R.scale = (C)(pix / std::fabs(r.ex));
        R.axis = (C)1;
      }
      rays[(size_t)a * d.n_det + b] = R;
    }
  }
}

template <typename C>
gkb_status upload(const gkb_geometry &g, RayP<C> **dr, AngleP<C> **da) {
  std::vector<RayP<C>> rays;
  std::vector<AngleP<C>> angs;
  build_tables<C>(g, rays, angs);
  GKB_CUDA_TRY(cudaMalloc((void **)dr, rays.size() * sizeof(RayP<C>)));
  GKB_CUDA_TRY(cudaMalloc((void **)da, angs.size() * sizeof(AngleP<C>)));
  GKB_CUDA_TRY(cudaMemcpy(*dr, rays.data(), rays.size() * sizeof(RayP<C>), cudaMemcpyHostToDevice));
  GKB_CUDA_TRY(cudaMemcpy(*da, angs.data(), angs.size() * sizeof(AngleP<C>), cudaMemcpyHostToDevice));
  return GKB_OK;
}

void free_tables(gkb_geometry *g) {
  if (g->ray_f) cudaFree(g->ray_f);
  if (g->ang_f) cudaFree(g->ang_f);
  if (g->ray_d) cudaFree(g->ray_d);
  if (g->ang_d) cudaFree(g->ang_d);
  g->ray_f = nullptr; g->ang_f = nullptr; g->ray_d = nullptr; g->ang_d = nullptr;
}

}  // namespace

// The FP32 ray table exactly as uploaded (the fast plan checks its kernels'
// shared-memory boxes against it).
void host_ray_table(const gkb_geometry *g, std::vector<RayP<float>> &rays) {
  std::vector<AngleP<float>> angs;
  build_tables<float>(*g, rays, angs);
}

gkb_status ensure_f64(gkb_geometry *g) {
  std::lock_guard<std::mutex> lk(g->f64_mutex);
  if (g->ray_d) return GKB_OK;
  int dev = 0;
  GKB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device) GKB_CUDA_TRY(cudaSetDevice(g->device));
  gkb_status st = upload<double>(*g, &g->ray_d, &g->ang_d);
  if (dev != g->device) cudaSetDevice(dev);
  return st;
}

template <typename C> GeomK<C> geom_view(const gkb_geometry *g);

template <typename C>
static GeomK<C> view_common(const gkb_geometry *g) {
  GeomK<C> K;
  const gkb_geometry_desc &d = g->desc;
  K.beam = d.beam == GKB_PARALLEL ? 0 : (d.beam == GKB_FAN_FLAT ? 1 : 2);
  K.nx = d.nx; K.ny = d.ny; K.na = d.n_angles; K.nd = d.n_det;
  K.t0 = (C)(0.5 * (d.n_det - 1));
  K.hx = (C)(0.5 * (d.nx - 1));
  K.hy = (C)(0.5 * (d.ny - 1));
  K.wpar = (C)(d.pixel * d.pixel / d.det_width);
  const bool fan = d.beam != GKB_PARALLEL;
  K.sodp = (C)(fan ? d.sod / d.pixel : 0.0);
  K.gfan = (C)(fan ? d.sdd / d.det_width : 0.0);   // flat: bins per unit tangent; arc: bins per radian
  K.wpix = (C)(fan ? d.pixel * d.sdd / d.det_width : 0.0);
  return K;
}

template <> GeomK<float> geom_view<float>(const gkb_geometry *g) {
  GeomK<float> K = view_common<float>(g);
  K.ray = g->ray_f; K.ang = g->ang_f;
  return K;
}
template <> GeomK<double> geom_view<double>(const gkb_geometry *g) {
  GeomK<double> K = view_common<double>(g);
  K.ray = g->ray_d; K.ang = g->ang_d;
  return K;
}

}  // namespace gkb

using namespace gkb;

extern "C" gkb_status gkb_geometry_create(const gkb_geometry_desc *desc, gkb_geometry **out) {
  if (!out) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || !desc->angles_rad) return GKB_ERR_INVALID_ARG;
  const gkb_geometry_desc &d = *desc;
  if (d.beam != GKB_PARALLEL && d.beam != GKB_FAN_FLAT && d.beam != GKB_FAN_ARC) return GKB_ERR_INVALID_ARG;
  if (d.nx < 1 || d.ny < 1 || d.n_angles < 1 || d.n_det < 1) return GKB_ERR_INVALID_ARG;
  if (!(d.pixel > 0.0) || !(d.det_width > 0.0) || !std::isfinite(d.pixel) || !std::isfinite(d.det_width))
    return GKB_ERR_INVALID_ARG;
  const long long n = (long long)d.nx * d.ny, m = (long long)d.n_angles * d.n_det;
  if (n >= (1LL << 31) || m >= (1LL << 31) || d.nx > (1 << 20) || d.ny > (1 << 20) || d.n_det > (1 << 20))
    return GKB_ERR_INVALID_ARG;
  for (int a = 0; a < d.n_angles; ++a)
    if (!std::isfinite(d.angles_rad[a])) return GKB_ERR_INVALID_ARG;
  const double half_diag = 0.5 * d.pixel * std::sqrt((double)d.nx * d.nx + (double)d.ny * d.ny);
  if (d.beam != GKB_PARALLEL) {
    if (!std::isfinite(d.sod) || !std::isfinite(d.sdd)) return GKB_ERR_INVALID_ARG;
    if (!(d.sod > half_diag) || !(d.sdd > d.sod)) return GKB_ERR_INVALID_ARG;
    if (d.beam == GKB_FAN_ARC && !(d.n_det * d.det_width / d.sdd < M_PI)) return GKB_ERR_INVALID_ARG;
  }
  gkb_geometry *g = new (std::nothrow) gkb_geometry();
  if (!g) return GKB_ERR_OOM;
  g->desc = d;
  g->angles.assign(d.angles_rad, d.angles_rad + d.n_angles);
  g->desc.angles_rad = g->angles.data();
  g->n = n;
  g->m = m;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    delete g;
    return GKB_ERR_CUDA;
  }
  gkb_status st = upload<float>(*g, &g->ray_f, &g->ang_f);
  if (st != GKB_OK) {
    free_tables(g);
    delete g;
    return st;
  }
  build_fast_plan(g);
  *out = g;
  return GKB_OK;
}

extern "C" gkb_status gkb_geometry_destroy(gkb_geometry *g) {
  if (!g) return GKB_ERR_INVALID_ARG;
  free_fast_plan(g);
  free_tables(g);
  delete g;
  return GKB_OK;
}

extern "C" gkb_status gkb_geometry_sizes(const gkb_geometry *g, long long *n_image, long long *m_sino) {
  if (!g) return GKB_ERR_INVALID_ARG;
  if (n_image) *n_image = g->n;
  if (m_sino) *m_sino = g->m;
  return GKB_OK;
}

extern "C" const char *gkb_status_string(gkb_status s) {
  switch (s) {
    case GKB_OK: return "ok";
    case GKB_ERR_INVALID_ARG: return "invalid argument";
    case GKB_ERR_CUDA: return "CUDA runtime error";
    case GKB_ERR_OOM: return "device out of memory";
    case GKB_ERR_NONFINITE: return "non-finite alpha or t";
    case GKB_ERR_TIMEOUT: return "bounded device wait ran out";
    case GKB_ERR_UNSUPPORTED: return "unsupported request";
    case GKB_ERR_TOO_LARGE: return "workspace exceeds the fixed array of gkb_solve_noalloc";
    case GKB_STATUS_BREAKDOWN: return "breakdown: Krylov space exhausted";
    case GKB_STATUS_NOT_CONVERGED: return "stopping rule not met by k_max";
    default: return "unknown status";
  }
}

extern "C" const char *gkb_version(void) { return "0.1.0"; }

extern "C" gkb_status gkb_geometry_autotune(gkb_geometry *g, gkb_dtype dtype) {
  if (!g || !dtype_valid(dtype)) return GKB_ERR_INVALID_ARG;
  return autotune(g, dtype);
}

extern "C" gkb_status gkb_geometry_get_shapes(const gkb_geometry *g, int shapes[4], int counts[4]) {
  if (!g) return GKB_ERR_INVALID_ARG;
  get_shapes(g, shapes, counts);
  return GKB_OK;
}

extern "C" gkb_status gkb_geometry_use_scatter(gkb_geometry *g, int enable) {
  if (!g || (enable != 0 && enable != 1)) return GKB_ERR_INVALID_ARG;
  return use_scatter(g, enable == 1);
}

extern "C" gkb_status gkb_geometry_set_shapes(gkb_geometry *g, const int shapes[4]) {
  if (!g || !shapes) return GKB_ERR_INVALID_ARG;
  return set_shapes(g, shapes);
}

// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/gkb.h"
#include "common.cuh"

namespace gkb {
// Work lists of the fast projector paths (see projectors_fast.cu).
struct FastPlan {
  bool tile_back = false, tile_fadj = false, tile_scatter = false, band = false, any_axis1 = false;
  // A: items of up to 2 (index 0) or 4 (index 1) consecutive angles, each two
  // int4: (first angle, first bin, bins, axis), (angles, first row, last row, 0)
  int4 *items_a[2] = {nullptr, nullptr};
  int n_a[2] = {0, 0};
  int4 *items_badj = nullptr;  // B^T gather: (angle, first bin, bins, axis)
  int n_badj = 0;
  // A^T scatter work lists: per tile (row-stepping 32x16 tiles first, then the
  // column-stepping 16x32 ones), entries off[t] .. off[t + 1] - 1 of ent, each
  // up to 32 rays of the tile's stepping axis in up to three ranges:
  // (first0 | axis << 31, first1, first2, count0 | count1 << 6 | count2 << 12)
  int *line_off = nullptr;
  uint4 *line_ent = nullptr;
  int line_t0 = 0, line_tiles = 0;     // row-stepping tiles (first), all tiles
  int line_tx0 = 0, line_tx1 = 0;      // tiles per image row band, row- and column-stepping
  bool bscatter = false;      // B^T by the pixel-driven integer scatter
  float bs_wmax = 0.f;        // bound on pixel_bin's weight over the image
  float bs_pmax = 1024.f;     // bound on the pixels of one scatter tile that add into one bin
  // kernel shapes (indices into the shape tables of projectors_fast.cu), set by the autotuner
  int cfg_back = 1, cfg_fadj = 1, cfg_fwd = 4, cfg_badj = 2;
  int tuned_dt = -1;          // storage type the shapes were tuned for (-1: none, -2: pinned by the caller)
  bool scatter = true;        // transposes by the scatter kernels where they apply
};
}  // namespace gkb

struct gkb_geometry {
  gkb_geometry_desc desc;      // angles_rad points into `angles`
  std::vector<double> angles;
  int device = 0;
  long long n = 0, m = 0;
  gkb::RayP<float> *ray_f = nullptr;
  gkb::AngleP<float> *ang_f = nullptr;
  gkb::RayP<double> *ray_d = nullptr;   // built on first FP64 use
  gkb::AngleP<double> *ang_d = nullptr;
  std::mutex f64_mutex;
  gkb::FastPlan fast;
};

namespace gkb {

// Optional fused epilogue of a projector launch.  With v the projector's
// output value at an index:
//   out = v - (*gamma) * prev          (when prev != nullptr)
//   z   = v - (*cz) * z                (when z != nullptr; z has the compute type)
//   *result = sum of out^2 over the launch (when partials != nullptr)
// and the launch does nothing when done != nullptr and *done != 0.
struct Epi {
  const void *prev = nullptr;
  const double *gamma = nullptr;
  void *z = nullptr;
  const double *cz = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  double *result = nullptr;
  const int *done = nullptr;
  void *scratch_t = nullptr;  // n-element buffer for a transposed image (allocated per call when null)
  void *scratch_acc = nullptr;  // m 64-bit accumulators + 256 bytes, zero between calls (per call when null)
  void *scratch_fadj = nullptr;  // 2 n FP32 values: the A^T scatter's partial images (per call when null)
  // mixed precision (16-bit projector operands, FP32 Krylov vectors): the
  // result goes to out32 in FP32 instead of the operator's own output, and
  // prev is FP32
  void *out32 = nullptr;
  bool prev32 = false;
};

// The fused epilogue at one output index: returns the stored value (as the
// caller's compute type) whose square feeds the launch's sum of squares.
template <typename T, typename C>
__device__ __forceinline__ C epi_store(const Epi &e, long long idx, C v, T *__restrict__ out) {
  C o = v;
  if (e.prev)
    o = v - (C)(*e.gamma) * (e.prev32 ? (C) static_cast<const float *>(e.prev)[idx]
                                      : to_c(static_cast<const T *>(e.prev)[idx]));
  if (e.z) {
    C *z = static_cast<C *>(e.z);
    z[idx] = v - (C)(*e.cz) * z[idx];
  }
  if (e.out32) {
    static_cast<float *>(e.out32)[idx] = (float)o;
    return (C)(float)o;
  }
  const T st = from_c<T>(o);
  out[idx] = st;
  return to_c(st);
}

#define GKB_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      gkb::set_last_cuda_error(_e);                          \
      return (_e == cudaErrorMemoryAllocation) ? GKB_ERR_OOM : GKB_ERR_CUDA; \
    }                                                        \
  } while (0)

void set_last_cuda_error(cudaError_t e);

gkb_status ensure_f64(gkb_geometry *g);
void host_ray_table(const gkb_geometry *g, std::vector<RayP<float>> &rays);
template <typename C> GeomK<C> geom_view(const gkb_geometry *g);

// Blocks a launch of each projector uses (the size of a partials buffer).
long long forward_blocks(const gkb_geometry *g);
long long back_blocks(const gkb_geometry *g);

gkb_status launch_forward(const gkb_geometry *g, gkb_dtype dt, const void *x, void *y, const Epi &e, cudaStream_t s);
gkb_status launch_back(const gkb_geometry *g, gkb_dtype dt, const void *y, void *x, const Epi &e, cudaStream_t s);
gkb_status launch_forward_adj(const gkb_geometry *g, gkb_dtype dt, const void *y, void *x, const Epi &e, cudaStream_t s);
gkb_status launch_back_adj(const gkb_geometry *g, gkb_dtype dt, const void *x, void *y, const Epi &e, cudaStream_t s);

size_t dtype_size(gkb_dtype dt);
bool dtype_valid(int dt);

}  // namespace gkb

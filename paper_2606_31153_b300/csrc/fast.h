// Shapes of the fast projector kernels and their host-side plan.
#pragma once
#include "internal.h"

namespace gkb {

constexpr int kWinB = 96;        // B tile: sinogram bins staged per angle
constexpr int kWinA = 96;        // A^T tile: candidate rays staged per angle
constexpr int kBandRays = 128;   // rays per CTA of the banded kernels
constexpr int kFootRows = 32;    // tallest band the item footprints are checked for
constexpr int kBoxW = 256;       // TMA box width (pixels)

void build_fast_plan(gkb_geometry *g);
void free_fast_plan(gkb_geometry *g);
bool band_ok_for(const gkb_geometry *g, gkb_dtype dt);
// op: 0 A, 1 B, 2 A^T, 3 B^T.  Sets handled=false when the fast path does not
// apply (FP64, unsupported geometry or layout) so the caller falls back.
gkb_status launch_fast(int op, const gkb_geometry *g, gkb_dtype dt, const void *in, void *out, void *scratch_t,
                       const Epi &e, cudaStream_t s, bool &handled);
long long fast_blocks(const gkb_geometry *g);
// Pick the fastest kernel shapes for this geometry and storage type (cached by
// geometry shape); synchronises the device, so it must not run during capture.
gkb_status autotune(gkb_geometry *g, gkb_dtype dt);
// Shape indices in operator order A, B, A^T, B^T and how many each kernel has.
void get_shapes(const gkb_geometry *g, int shapes[4], int counts[4]);
gkb_status set_shapes(gkb_geometry *g, const int shapes[4]);
// Run the transposes by the scatter kernels (default) or by the gather kernels.
gkb_status use_scatter(gkb_geometry *g, bool enable);

}  // namespace gkb

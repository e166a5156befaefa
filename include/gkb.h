/*
 * gkb.h -- C ABI of the B300 AB-/BA-GKB reconstruction library.
 *
 * The paper (GKB methods for X-ray CT with an unmatched back projector)
 * reconstructs x from A x ~ b (Sec. 1, Eq. 1) with a forward projector A and
 * a back projector B that is not A^T, by running Golub-Kahan
 * bidiagonalization on AB (AB-GKB, Algorithm 4) or BA (BA-GKB, Algorithm 5).
 * Every iteration applies A, B, A^T and B^T once each, so this library
 * exports all four operators, and the whole solve.
 *
 * Conventions shared by every entry point:
 *  - Image vectors hold ny*nx values, row-major (row 0 at the top, +y up);
 *    pixel (i, j) has its centre at x = (j - (nx-1)/2) pixel,
 *    y = ((ny-1)/2 - i) pixel.
 *  - Sinogram vectors hold n_angles*n_det values, angle-major.
 *  - Pointers named x, y, b are DEVICE pointers owned by the caller, dense
 *    and aligned to 16 bytes; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Operator calls are asynchronous on that stream.
 *  - Nothing throws across the ABI: every call returns a gkb_status.
 *    Negative values are errors, 0 is success, positive values are
 *    informational outcomes of a solve.
 */
#ifndef GKB_H
#define GKB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int gkb_status;
enum {
  GKB_OK = 0,
  GKB_ERR_INVALID_ARG = -1,  /* bad pointer, size, enum or geometry */
  GKB_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  GKB_ERR_OOM = -3,          /* device allocation failed */
  GKB_ERR_NONFINITE = -4,    /* NaN/Inf in alpha or t during a solve */
  GKB_ERR_TIMEOUT = -5,      /* a bounded device wait ran out */
  GKB_ERR_UNSUPPORTED = -6,  /* valid request the library does not implement */
  GKB_ERR_TOO_LARGE = -7,    /* workspace exceeds the fixed array of gkb_solve_noalloc */
  GKB_STATUS_BREAKDOWN = 1,  /* t_{k+1} or alpha_{k+1} vanished: Krylov space exhausted */
  GKB_STATUS_NOT_CONVERGED = 2 /* stopping rule not met by k_max */
};

typedef enum { GKB_PARALLEL = 0, GKB_FAN_FLAT = 1, GKB_FAN_ARC = 2 } gkb_beam;
typedef enum { GKB_F32 = 0, GKB_F64 = 1, GKB_BF16 = 2, GKB_F16 = 3 } gkb_dtype;
typedef enum { GKB_AB = 0, GKB_BA = 1, GKB_MATCHED = 2, GKB_AB_GMRES = 3, GKB_BA_GMRES = 4 } gkb_variant;
typedef enum { GKB_STOP_NONE = 0, GKB_STOP_DP = 1, GKB_STOP_RNS = 2, GKB_STOP_LEARNED = 3,
               GKB_STOP_HYBRID = 4 } gkb_stop;
typedef enum { GKB_REASON_K_MAX = 0, GKB_REASON_DP = 1, GKB_REASON_RNS = 2,
               GKB_REASON_BREAKDOWN = 3, GKB_REASON_ERROR = 4, GKB_REASON_LEARNED = 5,
               GKB_REASON_HYBRID = 6 } gkb_reason;

/*
 * Scan geometry (the paper's experiments use ASTRA parallel-beam geometries,
 * Sec. 5; the fan-beam form with a flat detector follows the same
 * line-integral model).
 *   Parallel: bin d of angle theta has detector coordinate
 *     u_d = (d - (n_det-1)/2) det_width and its ray is
 *     { p : p.x cos(theta) + p.y sin(theta) = u_d }.
 *   Fan (flat detector): source at sod (cos, sin); detector line through
 *     -(sdd - sod)(cos, sin) with axis (-sin, cos); the ray of bin d joins the
 *     source to the bin centre.  Requires sdd > sod > image half-diagonal.
 *   Fan (arc detector, equiangular bins): the same source; the detector is
 *     the circle of radius sdd about the source, bin d at arc length u_d from
 *     the central ray, so the ray of bin d leaves the source at the angle
 *     u_d / sdd from the central direction -(cos, sin), turned towards
 *     (-sin, cos).  B's weight is the inverse ray spacing at the pixel,
 *     pixel^2 sdd / (det_width rho), rho the pixel's distance from the
 *     source.  Same requirements; the bins must span less than pi.
 */
typedef struct {
  gkb_beam beam;
  int nx, ny;               /* image columns, rows (>= 1) */
  double pixel;             /* pixel width (> 0) */
  int n_angles;             /* >= 1 */
  const double *angles_rad; /* HOST array of n_angles angles; copied */
  int n_det;                /* bins per angle (>= 1) */
  double det_width;         /* bin width on the detector (> 0) */
  double sod, sdd;          /* fan only; ignored for parallel */
} gkb_geometry_desc;

typedef struct gkb_geometry gkb_geometry; /* opaque; owns its device tables */

/* Build the per-angle and per-ray device tables on the current device.
 * On error *out is set to NULL.  The handle is immutable afterwards and may be
 * used from several streams at once. */
gkb_status gkb_geometry_create(const gkb_geometry_desc *desc, gkb_geometry **out);
gkb_status gkb_geometry_destroy(gkb_geometry *g);
/* Time the shapes of the fast projector kernels (angle chunks of the pixel
 * tiles, band height and TMA ring depth of the ray bands, angles per CTA of
 * the B^T scatter) for this geometry and
 * storage type and keep the fastest; results are cached per geometry shape for
 * the process.  Shapes change only the work split, never the results.
 * gkb_plan_create and gkb_batch_create call it; call it yourself before timing
 * bare operator calls.  Allocates scratch and synchronises the device: not
 * during stream capture. */
gkb_status gkb_geometry_autotune(gkb_geometry *g, gkb_dtype dtype);
/* Kernel shapes in operator order A, B, A^T, B^T: shapes[i] is the index in
 * use, counts[i] how many shapes that kernel has (either pointer may be NULL;
 * host arrays of 4 ints).  Shape indices have no paper counterpart; they
 * select the work split of the fast kernels only. */
gkb_status gkb_geometry_get_shapes(const gkb_geometry *g, int shapes[4], int counts[4]);
/* Pin the kernel shapes (host array of 4 ints, each in [0, counts[i])) and mark
 * the geometry as tuned so later autotune calls keep them.  GKB_ERR_INVALID_ARG
 * for an index out of range (nothing is changed).  Not thread-safe against
 * concurrent operator calls on the same geometry. */
gkb_status gkb_geometry_set_shapes(gkb_geometry *g, const int shapes[4]);
/* Kernel family of the FP32/BF16/FP16 transposes.  enable=1 (the default):
 * A^T and B^T scatter each non-zero once from the side that computes its
 * weight (A^T: rays into tiles of 16 lines x 32 pixels; B^T: pixels into bins through
 * exact integer sums, see the B^T entry below); enable=0: both gather per
 * output element (pixel-driven A^T, ray-driven B^T).  Both families apply
 * identical weights; their results differ by rounding order only, except
 * that the scatter B^T returns NaN in every bin when any input value is not
 * finite (the gather returns it in the bins that value reaches).  The
 * choice is made per geometry, falls back to the gathers where a scatter
 * kernel does not apply, resets the two transposes' shapes to their defaults
 * and marks the geometry untuned.  Not thread-safe against concurrent
 * operator calls on the same geometry. */
gkb_status gkb_geometry_use_scatter(gkb_geometry *g, int enable);
/* Image and sinogram sizes of a geometry (either pointer may be NULL). */
gkb_status gkb_geometry_sizes(const gkb_geometry *g, long long *n_image, long long *m_sino);

/*
 * The four operators (Sec. 1 and Algorithms 4-5).
 * dtype selects the storage type of BOTH vectors: GKB_F64 computes in FP64;
 * GKB_F32/BF16/F16 accumulate in FP32.  Outputs are fully overwritten.
 *
 * projector_forward         y = A x    Joseph ray-driven forward projection:
 *                                      per ray, linear interpolation between
 *                                      the two pixel centres next to the ray
 *                                      on every row (or column) it crosses,
 *                                      scaled by pixel / max(|e_x|, |e_y|).
 * projector_back            x = B y    pixel-driven back projection with
 *                                      linear interpolation between bins and
 *                                      weight pixel^2/det_width (parallel) or
 *                                      the inverse ray spacing at the pixel (fan).
 * projector_forward_adjoint x = A^T y  exact transpose of projector_forward
 *                                      (the same interpolation weights,
 *                                      scattered from each ray into pixel
 *                                      tiles, or gathered per pixel).
 * projector_back_adjoint    y = B^T x  exact transpose of projector_back
 *                                      (the same weights, scattered from each
 *                                      pixel into bins as exact integer sums
 *                                      of values rounded to 24 significant
 *                                      bits relative to the largest |x| of
 *                                      their 32x32 tile, or gathered per ray).
 * B^T's scatter allocates m x 8 bytes of stream-ordered scratch per call.
 */
gkb_status projector_forward(const gkb_geometry *g, const void *x, void *y, gkb_dtype dtype, void *stream);
gkb_status projector_back(const gkb_geometry *g, const void *y, void *x, gkb_dtype dtype, void *stream);
gkb_status projector_forward_adjoint(const gkb_geometry *g, const void *y, void *x, gkb_dtype dtype, void *stream);
gkb_status projector_back_adjoint(const gkb_geometry *g, const void *x, void *y, gkb_dtype dtype, void *stream);

/*
 * Solver parameters.
 *   variant    GKB_AB (Algorithm 4), GKB_BA (Algorithm 5) or GKB_MATCHED
 *              (Algorithm 3 with A^T in place of B); or the paper's
 *              comparison methods GKB_AB_GMRES (Algorithm 1: Arnoldi on AB
 *              from b, x = B Q_k u_k) and GKB_BA_GMRES (Algorithm 2: Arnoldi
 *              on BA from B b, x = Q_k u_k), full (unrestarted) GMRES with
 *              `reorth` classical Gram-Schmidt passes (at least one; two
 *              match the printed modified Gram-Schmidt to rounding) and
 *              k_max <= 2048.  For the GMRES variants info->alpha returns the
 *              diagonal h_{k,k} of the Hessenberg matrix, info->t its
 *              subdiagonal h_{k+1,k} (t[0] = ||r_0||), info->resid
 *              ||A x_k - b|| as for GKB.
 *   k_max      maximum number of iterations (1 .. 4096).
 *   stop       GKB_STOP_DP: stop at the first k with ||A x_k - b|| <= tau ||e||
 *              (Eq. DP); GKB_STOP_RNS: first k >= 2 with
 *              | r_{k-1} - r_k | / r_{k-1} < rns_eps (Eq. RNS); GKB_STOP_NONE;
 *              GKB_STOP_HYBRID (AB and matched GKB: hybrid regularisation,
 *              the paper's stated future work, Sec. 6): after every
 *              iteration the projected Tikhonov problem
 *              min ||C_k u - t_1 e_1||^2 + lambda_k^2 ||u||^2 is solved with
 *              lambda_k = 0 while the least-squares residual is above
 *              tau ||e||, else the lambda_k whose projected residual -- for
 *              AB and matched GKB the data residual ||A x - b|| -- equals
 *              tau ||e||; the run stops once lambda_k has settled,
 *              |lambda_k - lambda_{k-1}| <= rns_eps lambda_{k-1} (reason
 *              GKB_REASON_HYBRID), else at k_max, and returns
 *              x = B Q_k u_lambda (AB) or Q_k u_lambda (matched).
 *   noise_norm ||e||_2 (absolute), required by GKB_STOP_DP.
 *   tau        DP safety factor (the paper uses 1; 0 means 1).
 *   reorth     0: none; 1: one classical Gram-Schmidt pass against all stored
 *              q_i (the one-sided reorthogonalisation of Algorithms
 *              4-5); 2: two passes.
 *   storage    type of the Krylov vectors and projector operands
 *              (F64, F32, BF16, F16); b and x are FP64 for F64 and FP32
 *              otherwise.  Scalars (alpha, t, Givens rotations, residual
 *              norms) are always FP64.
 *   use_graph  1: capture the iteration loop in a CUDA graph and launch it
 *              once; 0: launch kernels directly.
 *   operands   GKB_BF16 or GKB_F16 with storage GKB_F32 (GKB variants, no
 *              learned stop): mixed precision -- the Krylov vectors, the
 *              reorthogonalisation and every vector update stay FP32, while
 *              the projectors read and write their images and sinograms in
 *              that 16-bit type (FP32 accumulation; the result of the second
 *              projector of each step is written in FP32 by its fused
 *              epilogue).  Any other value: the projectors use the storage
 *              type.  (Zero-initialised parameters therefore mean "no mixed
 *              precision".)
 */
typedef struct {
  gkb_variant variant;
  int k_max;
  gkb_stop stop;
  double noise_norm;
  double tau;
  double rns_eps;
  int reorth;
  gkb_dtype storage;
  int use_graph;
  gkb_dtype operands;
} gkb_solve_params;

/*
 * Solve outcome.  alpha, t and resid are optional HOST arrays supplied by the
 * caller (NULL to skip) with room for k_max+1 values.  With k = k_stop, the
 * call writes alpha[i] = alpha_{i+1} (i < k), t[i] = t_{i+1} (i <= k) and
 * resid[i] = ||A x_{i+1} - b|| (i < k); other entries are left untouched.
 */
typedef struct {
  int k_stop;        /* iteration whose iterate is returned in x */
  int stop_reason;   /* gkb_reason */
  gkb_status status; /* same value gkb_solve returns */
  double *alpha;
  double *t;
  double *resid;
  double *lambda;    /* GKB_STOP_HYBRID: lambda[i] = lambda_{i+1} (i < k); NULL to skip */
} gkb_solve_info;

/*
 * Run AB-/BA-/matched GKB from x_0 = 0 on data b (n_angles*n_det values) and
 * write the iterate x_{k_stop} (ny*nx values).  Workspace (the Krylov basis of
 * (k_max+1) vectors plus a few vectors) is allocated on the device for the
 * call and released before returning.  The call blocks until the solve has
 * finished on `stream` and returns GKB_OK, GKB_STATUS_NOT_CONVERGED (the
 * stopping rule was requested but not met by k_max: x_{k_max} is returned),
 * GKB_STATUS_BREAKDOWN (x is the exact Krylov solution at k_stop) or an error.
 */
gkb_status gkb_solve(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x,
                     gkb_solve_info *info, void *stream);

/*
 * Reusable solve plan: the workspace and, with use_graph, the captured CUDA
 * graph of the whole solve, built once for a geometry and a parameter set.
 * gkb_plan_execute may then run any number of solves (one at a time per plan)
 * on any stream; b and x may be device pointers or host pointers (the copy
 * direction is inferred through unified addressing), b of n_angles*n_det and
 * x of ny*nx values, FP64 for F64 storage and FP32 otherwise.  It blocks until
 * the solve has finished and fills info like gkb_solve.  The geometry must
 * outlive the plan.
 */
typedef struct gkb_plan gkb_plan;
gkb_status gkb_plan_create(const gkb_geometry *g, const gkb_solve_params *p, gkb_plan **out);
gkb_status gkb_plan_execute(gkb_plan *plan, const void *b, void *x, gkb_solve_info *info, void *stream);
/* Kernels in the plan's captured graph: those outside the iteration loop
 * (initialisation and the final steps) and those of one iteration, so a
 * solve that ran k iterations launched outer + k * per_iteration kernels.
 * Host integers (either pointer may be NULL).  GKB_ERR_UNSUPPORTED for a
 * plan without a graph (use_graph = 0 or capture unavailable).  No paper
 * counterpart: launch accounting for measurements. */
gkb_status gkb_plan_kernel_counts(const gkb_plan *plan, long long *outer, long long *per_iteration);
/* Time one solve of the plan by kernel class: the solve runs with direct
 * launches (no graph) on `stream`, with a CUDA event before every group of
 * kernels, and ms[c] receives the milliseconds of class c, groups[c] (NULL
 * to skip) how many groups of that class ran.  Classes: 0 A, 1 B, 2 A^T,
 * 3 B^T (each projector application, with its helper kernels), 4 the
 * reorthogonalisation dot products, 5 its update, 6 everything else
 * (initialisation, the normalisations of s and q and the other vector
 * updates, the projected problem, the stopping test, the final
 * combination).  ms and groups are host arrays of 7; b as for
 * gkb_plan_execute.  Blocks until done.  Times include the event overhead of
 * a few microseconds per group.  No paper counterpart: measurement of the
 * per-iteration cost split (Sec. 4 counts it in projector applications). */
gkb_status gkb_plan_profile(gkb_plan *plan, const void *b, double *ms, long long *groups, void *stream);
gkb_status gkb_plan_destroy(gkb_plan *plan);

/*
 * Solve n independent problems (slices) with their own geometries, data,
 * parameters and stopping rules.  Each slice keeps its own workspace and
 * Krylov state and stops on its own discrepancy (or RNS) test; the whole batch
 * runs as ONE captured CUDA graph (one chain of solves per capture stream,
 * slices assigned largest first to the least loaded chain), launched once.
 * g, p, b, x and info are arrays of n entries; b[i], x[i] as for
 * gkb_plan_execute.  Returns the first error, else the strongest
 * informational status over the slices; info[i].status holds each slice's.
 *
 * gkb_batch_create/execute/destroy split the same work so that repeated
 * batches reuse the workspaces and the instantiated graph.
 */
gkb_status gkb_solve_batched(int n, const gkb_geometry *const *g, const gkb_solve_params *p,
                             const void *const *b, void *const *x, gkb_solve_info *info, void *stream);
typedef struct gkb_batch gkb_batch;
gkb_status gkb_batch_create(int n, const gkb_geometry *const *g, const gkb_solve_params *p, gkb_batch **out);
gkb_status gkb_batch_execute(gkb_batch *batch, const void *const *b, void *const *x, gkb_solve_info *info,
                             void *stream);
gkb_status gkb_batch_destroy(gkb_batch *batch);

/*
 * Learned stopping (BA-GKB, FP32 storage; the paper has no learned part).
 * A small perceptron (64 -> 256 -> 256 -> 2, exact GELU) reads the first 16
 * iterations of a slice -- log alpha_1..16, log t_2..17,
 * log(||A x_k - b|| / (tau ||e||)) and log(phibar_{k+1} / t_1), k = 1..16 --
 * and predicts log k_DP (the discrepancy-principle index, Eq. DP) and
 * log lambda, the projected Tikhonov parameter at k_DP + 8 whose projected
 * residual ||C u - t_1 e_1|| equals that of the plain iterate at k_DP.
 *
 * gkb_batch_execute_learned runs a batch whose slices all use
 * GKB_STOP_LEARNED: 16 iterations, the predictor on the device (BF16
 * weights), then each slice continues to k_hat + 8 (and at least until the
 * discrepancy principle has been met once, at most k_max), solves the
 * projected Tikhonov problem with lambda_hat (FP64, tridiagonal normal
 * equations of C_k) and forms x = Q_k u.  The discrepancy principle judges
 * the result: if | ||A x - b|| - tau ||e|| | > 0.05 tau ||e||, the slice falls back to
 * its discrepancy-principle iterate.  info[i].stop_reason is
 * GKB_REASON_LEARNED when the predicted stop was reached.
 */
typedef struct gkb_mlp gkb_mlp;
typedef struct {
  int k_hat;            /* predicted discrepancy index */
  double lambda;        /* predicted Tikhonov parameter */
  int k_dp;             /* first iteration that met the discrepancy principle (0: none) */
  int hybrid;           /* 1 if the returned x is the Tikhonov iterate */
  int fallback;         /* 0 accepted, 1 residual missed by > 5 %, 2 no discrepancy iterate */
  double hybrid_resid;  /* ||A x_hybrid - b|| */
} gkb_learned_info;
gkb_status gkb_batch_execute_learned(gkb_batch *batch, const gkb_mlp *mlp, const void *const *b, void *const *x,
                                     gkb_solve_info *info, gkb_learned_info *linfo, void *stream);
/* After gkb_batch_execute of a batch solved with GKB_STOP_NONE (and
 * noise_norm set): per slice the 64 features (X, n x 64, device), the labels
 * (T, n x 2: log k_DP, log lambda*, device) and valid[i] (device; 0 when the
 * run is too short to label). */
gkb_status gkb_batch_training_data(gkb_batch *batch, float *X, float *T, int *valid, void *stream);

/* The perceptron: FP32 parameters (flat: W1 256x64, b1, W2 256x256, b2,
 * W3 2x256, b3), Adam state, and a BF16 inference copy.  norm holds the
 * feature means (64), feature deviations (64), target means (2) and target
 * deviations (2) used by the inference path (gkb_mlp_forward with bf16=1 and
 * the learned solve); the FP32 path applies the raw network. */
gkb_status gkb_mlp_create(gkb_mlp **out);
gkb_status gkb_mlp_destroy(gkb_mlp *mlp);
int gkb_mlp_num_params(void);
gkb_status gkb_mlp_set_params(gkb_mlp *mlp, const float *theta, const float *norm);  /* host or device; resets Adam */
gkb_status gkb_mlp_get_params(const gkb_mlp *mlp, float *theta, float *norm);
/* Y (B x 2) = network(X (B x 64)); device pointers. */
gkb_status gkb_mlp_forward(gkb_mlp *mlp, const float *X, int B, float *Y, int bf16, void *stream);
/* Gradient of L = sum ||Y - T||^2 / (2B) into grad (device, num_params; NULL: internal) and L into *loss (device, or NULL). */
gkb_status gkb_mlp_gradient(gkb_mlp *mlp, const float *X, const float *T, int B, float *grad, float *loss, void *stream);
/* One Adam step (beta 0.9/0.999, eps 1e-8) on the batch. */
gkb_status gkb_mlp_train_step(gkb_mlp *mlp, const float *X, const float *T, int B, float lr, float *loss, void *stream);

/*
 * gkb_solve that also returns every iterate (BA and matched variants;
 * GKB_ERR_UNSUPPORTED for AB and the GMRES variants, whose iterates are
 * formed at the stop only): x_hist is a device array of k_max * n values
 * (FP64 for F64 storage, else FP32) whose row k-1 receives x_k for
 * k <= k_stop; the last row (k_max-1) also receives the returned iterate
 * x_{k_stop}.  For studies of
 * precision and semiconvergence (relative reconstruction error per iteration,
 * Eq. RE); launched without a graph.
 */
gkb_status gkb_solve_iterates(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x_hist,
                              gkb_solve_info *info, void *stream);

/*
 * gkb_solve without any device allocation.  (The paper has no counterpart:
 * this is a deployment variant of gkb_solve.)
 *
 * For callers that cannot call cudaMalloc when they solve -- applications
 * that hand the whole device to their own memory pool, plugin hosts that
 * forbid allocation after start-up, real-time loops that must not wait on the
 * allocator.  The result is the one gkb_solve computes (launched without a
 * graph); the workspace is a fixed 64 MiB array of static device memory inside
 * this library, reserved on every GPU that loads the library until the
 * process exits.  Problems whose workspace (about
 * (k_max+1) * dim_q + 8 * max(n, m) storage-type values, dim_q = n for BA and
 * matched, m for AB) exceeds it return GKB_ERR_TOO_LARGE.
 *
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the process, so it
 *    is stale after cudaDeviceReset of that device.
 *  - The current device must be the one the geometry was created on
 *    (GKB_ERR_INVALID_ARG otherwise): the array of the current device is
 *    used with the geometry's tables.
 *  - All calls share the one array, which keeps the previous call's contents;
 *    each call clears what must start at zero.  Calls whose work overlaps on
 *    the GPU (other streams, other host threads) race on it: serialise them.
 *  - FP64 storage uses the geometry's FP64 tables, which the first FP64
 *    operator or solve call builds; without them the call returns
 *    GKB_ERR_INVALID_ARG instead of allocating them.
 *  - b and x are as for gkb_plan_execute (device or host pointers); info as
 *    for gkb_solve.  Blocks until the solve has finished.
 */
gkb_status gkb_solve_noalloc(const gkb_geometry *g, const gkb_solve_params *p, const void *b, void *x,
                             gkb_solve_info *info, void *stream);

/* Static description of a status code. */
const char *gkb_status_string(gkb_status s);

/* Library version, "major.minor.patch". */
const char *gkb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GKB_H */

/*
 * FP64 reference projectors -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct loops for the unmatched projector pair of
 * the paper (Sec. 1, Eq. 1: A x ~ b with a forward projector A and a back
 * projector B != A^T) and for the exact transposes A^T and B^T that the
 * AB-/BA-GKB recurrences apply (Algorithms 4 and 5; Sec. 5
 * states that the toolbox was extended with the actual transposes).
 *
 *   A   : Joseph's ray-driven projector.  For every ray, step over the image
 *         rows (or columns, whichever axis the ray direction is closer to),
 *         take the point where the ray crosses that row, linearly interpolate
 *         between the two neighbouring pixel centres of the row (pixels
 *         outside the grid are zero) and scale the sum by pixel/c, with c the
 *         larger absolute component of the unit ray direction.
 *   B   : pixel-driven back projector.  For every pixel and every angle,
 *         project the pixel centre onto the detector, linearly interpolate the
 *         sinogram between the two neighbouring bins and weight by w(a,p).
 *   A^T : the same loop as A with every read turned into a scatter.
 *   B^T : the same loop as B with every read turned into a scatter.
 *
 * Threads (OpenMP, OMP_NUM_THREADS): every loop that is split runs over
 * outputs that no other iteration touches (rays for A, pixels for B, angles
 * for B^T, image rows or columns for A^T), and each output is summed in the
 * same order whatever the thread count, so results do not depend on it.
 *
 * Nothing here is shared with the CUDA path.  Only the test suite, the smoke
 * entry and the benchmark's CPU-baseline leg load this library.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

typedef struct {
  int beam;          /* 0: parallel, 1: fan beam, flat detector, 2: fan beam, arc detector */
  int nx, ny;        /* image columns and rows */
  double pix;        /* pixel width */
  int na;            /* number of projection angles */
  const double *ang; /* na angles in radians */
  int nd;            /* detector bins per angle */
  double du;         /* bin width on the detector */
  double sod, sdd;   /* fan beam: source-origin and source-detector distances */
  const double *cosv, *sinv; /* cos and sin of each angle */
} og_geom;

/* Ray (a, d): a point on it and its unit direction. */
static void ray_of(const og_geom *g, int a, int d, double *px, double *py,
                   double *ex, double *ey) {
  double c = g->cosv[a], s = g->sinv[a];
  double u = (d - 0.5 * (g->nd - 1)) * g->du;
  if (g->beam == 0) {
    *px = u * c; *py = u * s;
    *ex = -s; *ey = c;
  } else if (g->beam == 2) {
    /* arc detector: the central direction -(c, s) turned by gamma = u / sdd
       towards (-s, c) */
    double gam = u / g->sdd, cg = cos(gam), sg = sin(gam);
    *px = g->sod * c; *py = g->sod * s;
    *ex = -c * cg - s * sg;
    *ey = -s * cg + c * sg;
  } else {
    double sx = g->sod * c, sy = g->sod * s;                  /* source */
    double bx = -(g->sdd - g->sod) * c - u * s;               /* bin centre */
    double by = -(g->sdd - g->sod) * s + u * c;
    double lx = bx - sx, ly = by - sy, L = sqrt(lx * lx + ly * ly);
    *px = sx; *py = sy;
    *ex = lx / L; *ey = ly / L;
  }
}

static double xc(const og_geom *g, int j) { return (j - 0.5 * (g->nx - 1)) * g->pix; }
static double yc(const og_geom *g, int i) { return (0.5 * (g->ny - 1) - i) * g->pix; }

/*
 * Joseph's crossing of a ray (point p, unit direction e) with one line of the
 * image: for a ray closer to the vertical (|e_y| >= |e_x|, "row-stepping")
 * the line is image row k and the crossing is a column coordinate; otherwise
 * it is image column k and the crossing is a row coordinate.  *lo =
 * floor(coordinate), *f = coordinate - *lo.
 */
typedef struct { double px, py, ex, ey; } og_ray;

static og_ray ray_get(const og_geom *g, int a, int d) {
  og_ray r;
  ray_of(g, a, d, &r.px, &r.py, &r.ex, &r.ey);
  return r;
}
static int ray_axis(const og_ray *r) { return fabs(r->ey) >= fabs(r->ex) ? 0 : 1; }
/* the path length per line step: pix / max(|e_x|, |e_y|) */
static double ray_scale(const og_geom *g, const og_ray *r) {
  return ray_axis(r) ? g->pix / fabs(r->ex) : g->pix / fabs(r->ey);
}

static void joseph_line(const og_geom *g, const og_ray *r, int k, double *lo, double *f) {
  double c;
  if (ray_axis(r) == 0) {
    double xs = r->px + (yc(g, k) - r->py) / r->ey * r->ex;   /* crossing of row k */
    c = xs / g->pix + 0.5 * (g->nx - 1);                      /* column coordinate */
  } else {
    double ys = r->py + (xc(g, k) - r->px) / r->ex * r->ey;   /* crossing of column k */
    c = 0.5 * (g->ny - 1) - ys / g->pix;                      /* row coordinate */
  }
  *lo = floor(c);
  *f = c - *lo;
}

/* Joseph's method for one ray: sum_p A[r,p] x[p]. */
static double joseph_ray(const og_geom *g, int a, int d, const double *xin) {
  const og_ray r = ray_get(g, a, d);
  const int axis = ray_axis(&r);
  const int nk = axis ? g->nx : g->ny, nl = axis ? g->ny : g->nx;
  double acc = 0.0, lo, f;
  for (int k = 0; k < nk; ++k) {
    joseph_line(g, &r, k, &lo, &f);
    if (lo < -1.0 || lo > (double)nl) continue;
    int l = (int)lo;
    /* pixel (row, column) of position l on line k */
    if (l >= 0 && l < nl) acc += (1.0 - f) * xin[axis ? (size_t)l * g->nx + k : (size_t)k * g->nx + l];
    if (l + 1 >= 0 && l + 1 < nl) acc += f * xin[axis ? (size_t)(l + 1) * g->nx + k : (size_t)k * g->nx + l + 1];
  }
  return acc * ray_scale(g, &r);
}

/*
 * Pixel-driven back projection at pixel (i, j) and angle a: the fractional
 * bin t of the projected pixel centre and the weight w(a, p).
 *   parallel: u = x cos + y sin, w = pix^2 / du
 *   fan:      U = sod - (x cos + y sin) (depth from the source along the
 *             central ray), L = -x sin + y cos, u = sdd L / U and
 *             w = pix^2 sdd sqrt(U^2 + L^2) / (du U^2), the inverse of the
 *             perpendicular spacing of neighbouring rays at the pixel.
 *   fan arc:  u = sdd atan2(L, U), w = pix^2 sdd / (du rho), rho the
 *             pixel's distance from the source (the same rule).
 */
static void pixel_bin(const og_geom *g, int a, int i, int j, double *t, double *w) {
  double c = g->cosv[a], s = g->sinv[a];
  double x = xc(g, j), y = yc(g, i), u;
  if (g->beam == 0) {
    u = x * c + y * s;
    *w = g->pix * g->pix / g->du;
  } else if (g->beam == 2) {
    /* arc: the pixel's direction from the source is atan2(L, U) off the
       central ray, arc length sdd times that; neighbouring rays are du/sdd
       apart in angle, so rho du / sdd apart at the pixel */
    double U = g->sod - (x * c + y * s);
    double L = -x * s + y * c;
    double rho = sqrt(U * U + L * L);
    u = g->sdd * atan2(L, U);
    *w = g->pix * g->pix * g->sdd / (g->du * rho);
  } else {
    double U = g->sod - (x * c + y * s);
    double L = -x * s + y * c;
    u = g->sdd * L / U;
    *w = g->pix * g->pix * g->sdd * sqrt(U * U + L * L) / (g->du * U * U);
  }
  *t = u / g->du + 0.5 * (g->nd - 1);
}

/* y = A x (threads over angles: every ray is an independent output) */
void og_forward(const og_geom *g, const double *x, double *y) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < g->na; ++a)
    for (int d = 0; d < g->nd; ++d)
      y[(size_t)a * g->nd + d] = joseph_ray(g, a, d, x);
}

/*
 * x = A^T y.  Every ray deposits A[r,p] y[r] into the two pixels next to its
 * crossing of each line it steps over.  Row-stepping rays only ever deposit
 * into the row they cross, column-stepping rays into the column: the
 * row-stepping part is summed per image row (rays in (a, d) order) and the
 * column-stepping part per image column (same order), and x is their sum --
 * for any number of threads, which take rows, then columns.
 */
void og_forward_T(const og_geom *g, const double *y, double *x) {
  const size_t n = (size_t)g->nx * g->ny, m = (size_t)g->na * g->nd;
  double *xcol = (double *)calloc(n, sizeof(double));
  og_ray *rays = (og_ray *)malloc(m * sizeof(og_ray));
  for (int a = 0; a < g->na; ++a)
    for (int d = 0; d < g->nd; ++d) rays[(size_t)a * g->nd + d] = ray_get(g, a, d);
  memset(x, 0, sizeof(double) * n);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < g->ny; ++i) {
    double *row = x + (size_t)i * g->nx;
    for (size_t r = 0; r < m; ++r) {
      double lo, f;
      if (ray_axis(&rays[r]) != 0) continue;
      joseph_line(g, &rays[r], i, &lo, &f);
      if (lo < -1.0 || lo > (double)g->nx) continue;
      const int j = (int)lo;
      const double scale = ray_scale(g, &rays[r]), v = y[r];
      if (j >= 0 && j < g->nx) row[j] += (1.0 - f) * scale * v;
      if (j + 1 >= 0 && j + 1 < g->nx) row[j + 1] += f * scale * v;
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < g->nx; ++j)
    for (size_t r = 0; r < m; ++r) {
      double lo, f;
      if (ray_axis(&rays[r]) != 1) continue;
      joseph_line(g, &rays[r], j, &lo, &f);
      if (lo < -1.0 || lo > (double)g->ny) continue;
      const int i = (int)lo;
      const double scale = ray_scale(g, &rays[r]), v = y[r];
      if (i >= 0 && i < g->ny) xcol[(size_t)i * g->nx + j] += (1.0 - f) * scale * v;
      if (i + 1 >= 0 && i + 1 < g->ny) xcol[(size_t)(i + 1) * g->nx + j] += f * scale * v;
    }
  for (size_t p = 0; p < n; ++p) x[p] += xcol[p];
  free(rays);
  free(xcol);
}

/* x = B y (threads over image rows) */
void og_back(const og_geom *g, const double *y, double *x) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < g->ny; ++i)
    for (int j = 0; j < g->nx; ++j) {
      double acc = 0.0;
      for (int a = 0; a < g->na; ++a) {
        double t, w;
        pixel_bin(g, a, i, j, &t, &w);
        double d0 = floor(t), f = t - d0;
        if (d0 < -1.0 || d0 > (double)g->nd) continue;
        int d = (int)d0;
        const double *row = y + (size_t)a * g->nd;
        double v = 0.0;
        if (d >= 0 && d < g->nd) v += (1.0 - f) * row[d];
        if (d + 1 >= 0 && d + 1 < g->nd) v += f * row[d + 1];
        acc += w * v;
      }
      x[(size_t)i * g->nx + j] = acc;
    }
}

/* y = B^T x: every pixel deposits into the two bins next to its projection
 * at every angle (threads over angles; each bin sums its pixels in row-major
 * order) */
void og_back_T(const og_geom *g, const double *x, double *y) {
  memset(y, 0, sizeof(double) * (size_t)g->na * g->nd);
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < g->na; ++a) {
    double *row = y + (size_t)a * g->nd;
    for (int i = 0; i < g->ny; ++i)
      for (int j = 0; j < g->nx; ++j) {
        const double xv = x[(size_t)i * g->nx + j];
        double t, w;
        pixel_bin(g, a, i, j, &t, &w);
        double d0 = floor(t), f = t - d0;
        if (d0 < -1.0 || d0 > (double)g->nd) continue;
        int d = (int)d0;
        if (d >= 0 && d < g->nd) row[d] += w * (1.0 - f) * xv;
        if (d + 1 >= 0 && d + 1 < g->nd) row[d + 1] += w * f * xv;
      }
  }
}

/* threads the parallel loops use (1 without OpenMP) */
int og_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void og_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---- single entries, for sampled checks at sizes where a full pass is slow ---- */

/* (A x)[a, d] */
double og_forward_ray(const og_geom *g, const double *x, int a, int d) {
  return joseph_ray(g, a, d, x);
}

/* (B y)[i, j] */
double og_back_pixel(const og_geom *g, const double *y, int i, int j) {
  double acc = 0.0;
  for (int a = 0; a < g->na; ++a) {
    double t, w;
    pixel_bin(g, a, i, j, &t, &w);
    double d0 = floor(t), f = t - d0;
    if (d0 < -1.0 || d0 > (double)g->nd) continue;
    int d = (int)d0;
    const double *row = y + (size_t)a * g->nd;
    double v = 0.0;
    if (d >= 0 && d < g->nd) v += (1.0 - f) * row[d];
    if (d + 1 >= 0 && d + 1 < g->nd) v += f * row[d + 1];
    acc += w * v;
  }
  return acc;
}

/* (A^T y)[i, j] = sum over all rays of A[r, p] y[r]: each ray's Joseph weight
 * on pixel (i, j) is recomputed from the ray's crossing of row i (or column j). */
double og_forward_T_pixel(const og_geom *g, const double *y, int i, int j) {
  double acc = 0.0;
  for (int a = 0; a < g->na; ++a)
    for (int d = 0; d < g->nd; ++d) {
      const og_ray r = ray_get(g, a, d);
      const int axis = ray_axis(&r);
      double lo, f, wgt = 0.0;
      joseph_line(g, &r, axis ? j : i, &lo, &f);
      const double me = axis ? (double)i : (double)j;     /* position of the pixel on that line */
      if (lo == me) wgt = 1.0 - f;
      else if (lo + 1.0 == me) wgt = f;
      if (wgt != 0.0) acc += wgt * ray_scale(g, &r) * y[(size_t)a * g->nd + d];
    }
  return acc;
}

/* (B^T x)[a, d] = sum over pixels of B[p, (a, d)] x[p]. */
double og_back_T_ray(const og_geom *g, const double *x, int a, int d) {
  double acc = 0.0;
  for (int i = 0; i < g->ny; ++i)
    for (int j = 0; j < g->nx; ++j) {
      double t, w;
      pixel_bin(g, a, i, j, &t, &w);
      double d0 = floor(t), f = t - d0;
      double wgt = 0.0;
      if (d0 == (double)d) wgt = 1.0 - f;
      else if (d0 + 1.0 == (double)d) wgt = f;
      if (wgt != 0.0) acc += w * wgt * x[(size_t)i * g->nx + j];
    }
  return acc;
}

/*
 * FP64 reference projectors -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct loops for the unmatched projector pair of
 * the paper (Sec. 1, Eq. 1: A x ~ b with a forward projector A and a back
 * projector B != A^T) and for the exact transposes A^T and B^T that the
 * AB-/BA-GKB recurrences apply (Algorithms 4 and 5, steps 2 and 8; Sec. 5
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
 * Nothing here is shared with the CUDA path.  Only the test suite, the smoke
 * entry and the benchmark's CPU-baseline leg load this library.
 */
#include <math.h>
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
 * Joseph's method for one ray.  mode 0: return sum_p A[r,p] x[p].
 * mode 1: x[p] += A[r,p] * val for every pixel the ray touches (scatter).
 */
static double joseph_ray(const og_geom *g, int a, int d, const double *xin,
                         double *xout, double val, int mode) {
  double px, py, ex, ey;
  ray_of(g, a, d, &px, &py, &ex, &ey);
  double acc = 0.0;
  if (fabs(ey) >= fabs(ex)) {
    double scale = g->pix / fabs(ey);
    for (int i = 0; i < g->ny; ++i) {
      double xs = px + (yc(g, i) - py) / ey * ex;       /* crossing of row i */
      double jf = xs / g->pix + 0.5 * (g->nx - 1);      /* column coordinate */
      double j0 = floor(jf), f = jf - j0;
      if (j0 < -1.0 || j0 > (double)g->nx) continue;
      int j = (int)j0;
      if (j >= 0 && j < g->nx) {
        if (mode == 0) acc += (1.0 - f) * xin[(size_t)i * g->nx + j];
        else xout[(size_t)i * g->nx + j] += (1.0 - f) * scale * val;
      }
      if (j + 1 >= 0 && j + 1 < g->nx) {
        if (mode == 0) acc += f * xin[(size_t)i * g->nx + j + 1];
        else xout[(size_t)i * g->nx + j + 1] += f * scale * val;
      }
    }
    return acc * scale;
  } else {
    double scale = g->pix / fabs(ex);
    for (int j = 0; j < g->nx; ++j) {
      double ys = py + (xc(g, j) - px) / ex * ey;       /* crossing of column j */
      double fi = 0.5 * (g->ny - 1) - ys / g->pix;      /* row coordinate */
      double i0 = floor(fi), f = fi - i0;
      if (i0 < -1.0 || i0 > (double)g->ny) continue;
      int i = (int)i0;
      if (i >= 0 && i < g->ny) {
        if (mode == 0) acc += (1.0 - f) * xin[(size_t)i * g->nx + j];
        else xout[(size_t)i * g->nx + j] += (1.0 - f) * scale * val;
      }
      if (i + 1 >= 0 && i + 1 < g->ny) {
        if (mode == 0) acc += f * xin[(size_t)(i + 1) * g->nx + j];
        else xout[(size_t)(i + 1) * g->nx + j] += f * scale * val;
      }
    }
    return acc * scale;
  }
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

/* y = A x */
void og_forward(const og_geom *g, const double *x, double *y) {
  for (int a = 0; a < g->na; ++a)
    for (int d = 0; d < g->nd; ++d)
      y[(size_t)a * g->nd + d] = joseph_ray(g, a, d, x, NULL, 0.0, 0);
}

/* x = A^T y  (scatter form of og_forward) */
void og_forward_T(const og_geom *g, const double *y, double *x) {
  memset(x, 0, sizeof(double) * (size_t)g->nx * g->ny);
  for (int a = 0; a < g->na; ++a)
    for (int d = 0; d < g->nd; ++d)
      joseph_ray(g, a, d, NULL, x, y[(size_t)a * g->nd + d], 1);
}

/* x = B y */
void og_back(const og_geom *g, const double *y, double *x) {
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

/* y = B^T x  (scatter form of og_back) */
void og_back_T(const og_geom *g, const double *x, double *y) {
  memset(y, 0, sizeof(double) * (size_t)g->na * g->nd);
  for (int i = 0; i < g->ny; ++i)
    for (int j = 0; j < g->nx; ++j) {
      double xv = x[(size_t)i * g->nx + j];
      for (int a = 0; a < g->na; ++a) {
        double t, w;
        pixel_bin(g, a, i, j, &t, &w);
        double d0 = floor(t), f = t - d0;
        if (d0 < -1.0 || d0 > (double)g->nd) continue;
        int d = (int)d0;
        double *row = y + (size_t)a * g->nd;
        if (d >= 0 && d < g->nd) row[d] += w * (1.0 - f) * xv;
        if (d + 1 >= 0 && d + 1 < g->nd) row[d + 1] += w * f * xv;
      }
    }
}

/* ---- single entries, for sampled checks at sizes where a full pass is slow ---- */

/* (A x)[a, d] */
double og_forward_ray(const og_geom *g, const double *x, int a, int d) {
  return joseph_ray(g, a, d, x, NULL, 0.0, 0);
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
      double px, py, ex, ey, wgt = 0.0;
      ray_of(g, a, d, &px, &py, &ex, &ey);
      if (fabs(ey) >= fabs(ex)) {
        double xs = px + (yc(g, i) - py) / ey * ex;
        double jf = xs / g->pix + 0.5 * (g->nx - 1);
        double j0 = floor(jf), f = jf - j0;
        if (j0 == (double)j) wgt = 1.0 - f;
        else if (j0 + 1.0 == (double)j) wgt = f;
        wgt *= g->pix / fabs(ey);
      } else {
        double ys = py + (xc(g, j) - px) / ex * ey;
        double fi = 0.5 * (g->ny - 1) - ys / g->pix;
        double i0 = floor(fi), f = fi - i0;
        if (i0 == (double)i) wgt = 1.0 - f;
        else if (i0 + 1.0 == (double)i) wgt = f;
        wgt *= g->pix / fabs(ex);
      }
      if (wgt != 0.0) acc += wgt * y[(size_t)a * g->nd + d];
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

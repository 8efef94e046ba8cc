/*
 * Synthetic dose-deposition matrix D for seeded VMAT phantoms.
 *
 * The paper takes D_ij as given: it is precomputed by a separate GPU dose
 * engine (Sec. 2.1) and is an INPUT to the optimisation method, not part of
 * it.  This file stands in for that engine with a plain parallel-ray model so
 * that the oracle and the CUDA path can be fed identical matrices.  It holds
 * none of the method's arithmetic (no cost, price, pricing or master step).
 *
 * Geometry (all lengths in mm, angles in degrees):
 *   voxel (ix,iy,iz) has centre ((ix-(nx-1)/2)h, (iy-(ny-1)/2)h, (iz-(nz-1)/2)h)
 *   and flat index j = (iz*ny + iy)*nx + ix.
 *   The gantry turns about z.  At angle theta the beam travels along
 *   b = (-sin t, cos t, 0) (theta = 0: anterior source, beam towards +y) and
 *   the MLC's lateral axis is u = (cos t, sin t, 0).
 *   Beamlet i = (k*R + r)*C + c has its central ray through
 *   u_c*u + v_r*zhat, u_c = (c-(C-1)/2)*w_col, v_r = (r-(R-1)/2)*w_row.
 *   depth = max(0, p.b - a_in), a_in = where that central ray enters the body;
 *   a ray that misses the body (or leaves the grid's z range) deposits nothing.
 *   D_ij = exp(-mu*depth) * exp(-d^2/(2 sigma^2)), d = distance of the voxel
 *   centre from the central ray, kept only where D_ij >= cutoff and the voxel
 *   centre lies inside the body.
 *
 * Output: beamlet-major CSR (row_ptr[B+1] int64, vox[nnz] int32 ascending
 * within each row, val[nnz] double).  Rows are computed independently, so the
 * result does not depend on the OpenMP thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t nx, ny, nz;
  double h;
  int32_t body_kind; /* 0: the whole grid box, 1: elliptic cylinder along z */
  double body_ax, body_ay;
  int32_t n_angles;
  const double *theta_deg;
  int32_t n_rows, n_cols;
  double w_row, w_col;
  double sigma, mu, cutoff;
  int32_t round_f32; /* store (double)(float)D so FP32 storage is exact */
} ph_spec;

static const double PH_PI = 3.14159265358979323846;

static double coord(int32_t i, int32_t n, double h) { return (i - 0.5 * (n - 1)) * h; }

static int inside_body(const ph_spec *s, double x, double y) {
  if (s->body_kind == 0) return 1;
  double ex = x / s->body_ax, ey = y / s->body_ay;
  return ex * ex + ey * ey <= 1.0;
}

/* Parameter a at which the central ray q(a) = u_c*u + a*b (in the xy plane)
 * enters the body; returns 0 if the ray misses it. */
static int ray_entry(const ph_spec *s, double ct, double st, double uc, double *a_in) {
  double px = uc * ct, py = uc * st; /* point at a = 0 */
  double bx = -st, by = ct;
  if (s->body_kind == 0) {
    double X = 0.5 * s->nx * s->h, Y = 0.5 * s->ny * s->h;
    double lo = -INFINITY, hi = INFINITY;
    double p[2] = {px, py}, b[2] = {bx, by}, E[2] = {X, Y};
    for (int d = 0; d < 2; ++d) {
      if (fabs(b[d]) < 1e-12) {
        if (p[d] < -E[d] || p[d] > E[d]) return 0;
      } else {
        double t0 = (-E[d] - p[d]) / b[d], t1 = (E[d] - p[d]) / b[d];
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
      }
    }
    if (lo > hi) return 0;
    *a_in = lo;
    return 1;
  }
  double iax2 = 1.0 / (s->body_ax * s->body_ax), iay2 = 1.0 / (s->body_ay * s->body_ay);
  double A = bx * bx * iax2 + by * by * iay2;
  double Bq = 2.0 * (px * bx * iax2 + py * by * iay2);
  double Cq = px * px * iax2 + py * py * iay2 - 1.0;
  double disc = Bq * Bq - 4.0 * A * Cq;
  if (disc < 0.0) return 0;
  *a_in = (-Bq - sqrt(disc)) / (2.0 * A);
  return 1;
}

/* Visit every kept (voxel, value) of beamlet i in ascending voxel order.
 * If vox/val are NULL only counts.  Returns the number of entries. */
static int64_t beamlet_row(const ph_spec *s, int64_t i, int32_t *vox, double *val) {
  const int32_t RC = s->n_rows * s->n_cols;
  const int32_t k = (int32_t)(i / RC);
  const int32_t r = (int32_t)((i % RC) / s->n_cols);
  const int32_t c = (int32_t)(i % s->n_cols);
  const double th = s->theta_deg[k] * PH_PI / 180.0;
  const double ct = cos(th), st = sin(th);
  const double uc = (c - 0.5 * (s->n_cols - 1)) * s->w_col;
  const double vr = (r - 0.5 * (s->n_rows - 1)) * s->w_row;
  const double zhalf = 0.5 * s->nz * s->h;
  if (vr < -zhalf || vr > zhalf) return 0;
  double a_in;
  if (!ray_entry(s, ct, st, uc, &a_in)) return 0;

  const double dmax = s->sigma * sqrt(2.0 * log(1.0 / s->cutoff));
  const double inv2s2 = 1.0 / (2.0 * s->sigma * s->sigma);
  int64_t n = 0;
  for (int32_t iz = 0; iz < s->nz; ++iz) {
    const double pz = coord(iz, s->nz, s->h);
    const double dz = pz - vr;
    if (fabs(dz) > dmax) continue;
    const double ell = sqrt(dmax * dmax - dz * dz);
    for (int32_t iy = 0; iy < s->ny; ++iy) {
      const double py = coord(iy, s->ny, s->h);
      int32_t ix0 = 0, ix1 = s->nx - 1;
      /* x*ct + py*st must lie in [uc-ell, uc+ell] */
      if (fabs(ct) > 1e-12) {
        double x0 = (uc - ell - py * st) / ct, x1 = (uc + ell - py * st) / ct;
        if (x0 > x1) { double t = x0; x0 = x1; x1 = t; }
        double f0 = x0 / s->h + 0.5 * (s->nx - 1), f1 = x1 / s->h + 0.5 * (s->nx - 1);
        if (f1 < 0.0 || f0 > s->nx - 1) continue;
        int32_t a = (int32_t)ceil(f0), b = (int32_t)floor(f1);
        ix0 = a > 0 ? a - 1 : 0; /* one voxel of slack; exact test below */
        ix1 = b < s->nx - 1 ? b + 1 : s->nx - 1;
      } else {
        double lat = py * st - uc;
        if (fabs(lat) > ell) continue;
      }
      for (int32_t ix = ix0; ix <= ix1; ++ix) {
        const double px = coord(ix, s->nx, s->h);
        if (!inside_body(s, px, py)) continue;
        const double lat = px * ct + py * st - uc;
        const double d2 = lat * lat + dz * dz;
        if (d2 > dmax * dmax) continue;
        double depth = (-px * st + py * ct) - a_in;
        if (depth < 0.0) depth = 0.0;
        double D = exp(-s->mu * depth - d2 * inv2s2);
        if (!(D >= s->cutoff)) continue;
        if (vox) {
          vox[n] = (iz * s->ny + iy) * s->nx + ix;
          val[n] = s->round_f32 ? (double)(float)D : D;
        }
        ++n;
      }
    }
  }
  return n;
}

/* Pass 1: per-beamlet entry counts; returns the total nnz. */
int64_t ph_count(const ph_spec *s, int64_t *row_nnz) {
  const int64_t B = (int64_t)s->n_angles * s->n_rows * s->n_cols;
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int64_t i = 0; i < B; ++i) {
    row_nnz[i] = beamlet_row(s, i, NULL, NULL);
    total += row_nnz[i];
  }
  return total;
}

/* Pass 2: fill vox/val at the offsets row_ptr (from pass 1's counts). */
int ph_fill(const ph_spec *s, const int64_t *row_ptr, int32_t *vox, double *val) {
  const int64_t B = (int64_t)s->n_angles * s->n_rows * s->n_cols;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t i = 0; i < B; ++i) {
    int64_t n = beamlet_row(s, i, vox + row_ptr[i], val + row_ptr[i]);
    if (n != row_ptr[i + 1] - row_ptr[i]) bad = 1;
  }
  return bad ? -1 : 0;
}

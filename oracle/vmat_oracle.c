/*
 * FP64 CPU oracle of the column-generation VMAT optimiser
 * (Men, Romeijn, Jia, Jiang, "Ultra-fast treatment plan optimization for
 * volumetric modulated arc therapy").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * Notation (Sec. 2.1): N beams sorted by angle theta_k (degrees), each with an
 * MLC of R leaf rows x C beamlet columns; beamlet i = (k*R + r)*C + c; voxel
 * set V; dose z_j = sum_k y_k sum_{i in A_k} D_ij; an aperture A_k is one open
 * interval [l, r) of columns in every leaf row of beam k.
 *
 * Precision: everything is double except the *_f32 pricing routines, which
 * take the pricing decisions in single precision so that a single-precision
 * kernel can be compared with them decision for decision.  Sums run in a
 * fixed, stated order.  OpenMP is used only where every output element is
 * computed by one thread in a fixed order (row-wise or column-wise dot
 * products); the result does not depend on the thread count.
 *
 * Readings of points the paper leaves open (same in the CUDA path):
 *   - y_k is held at 0 for beams without an aperture yet (restricted master).
 *   - G may run over a ring (cyclic != 0, extra term between the last and the
 *     first beam with gap theta_1 + 360 - theta_N) or over the path of Eq. 2.
 *   - The leaf-travel limit is an integer s of columns per angle step, applied
 *     to both leaves against the nearest beam with an aperture on each side.
 *   - The most promising aperture is the one of least (most negative) total
 *     price; it is added even if that price is not negative.
 *   - Within a row: least value, then shortest interval, then smallest l;
 *     across beams: least price, then lowest index.
 *   - Master problem: projected gradient with the adaptive Barzilai-Borwein
 *     step (ABBmin for a solve's first iterations, the short step after
 *     them; see vo_master), an exact line search on [0,1] and the natural
 *     KKT residual.
 *   - Dose-volume histograms (the evaluation behind Fig. 2): bins of width
 *     dose_max / n_bins from 0; the last bin also holds doses at or above
 *     dose_max, the first one doses below 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Eq. 1: one-sided quadratic voxel cost and its derivative                   */
/* ------------------------------------------------------------------------ */
double vo_F(double z, double T, double a, double b) {
  double under = T - z > 0.0 ? T - z : 0.0;
  double over = z - T > 0.0 ? z - T : 0.0;
  return a * under * under + b * over * over;
}

double vo_dF(double z, double T, double a, double b) {
  if (z < T) return -2.0 * a * (T - z);
  if (z > T) return 2.0 * b * (z - T);
  return 0.0;
}

/* sum_j F(z_j) in voxel order; sid selects (T, alpha, beta) per voxel */
double vo_voxel_cost(int64_t V, const double *z, const uint8_t *sid, const double *T,
                     const double *a, const double *b) {
  double s = 0.0;
  for (int64_t j = 0; j < V; ++j) s += vo_F(z[j], T[sid[j]], a[sid[j]], b[sid[j]]);
  return s;
}

void vo_voxel_dcost(int64_t V, const double *z, const uint8_t *sid, const double *T,
                    const double *a, const double *b, double *fp) {
  for (int64_t j = 0; j < V; ++j) fp[j] = vo_dF(z[j], T[sid[j]], a[sid[j]], b[sid[j]]);
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: dose-rate smoothing G(y) = sum (y_{k+1}-y_k)^2 / (theta_{k+1}-theta_k) */
/* ------------------------------------------------------------------------ */
static double gap(int N, const double *theta, int k) { /* gap between beam k and k+1 */
  return k + 1 < N ? theta[k + 1] - theta[k] : theta[0] + 360.0 - theta[N - 1];
}

double vo_G(int N, const double *theta, const double *y, int cyclic) {
  double s = 0.0;
  int last = cyclic ? N : N - 1;
  for (int k = 0; k < last; ++k) {
    double d = y[(k + 1) % N] - y[k];
    s += d * d / gap(N, theta, k);
  }
  return s;
}

void vo_dG(int N, const double *theta, const double *y, int cyclic, double *out) {
  for (int k = 0; k < N; ++k) out[k] = 0.0;
  int last = cyclic ? N : N - 1;
  for (int k = 0; k < last; ++k) {
    int k1 = (k + 1) % N;
    double t = 2.0 * (y[k1] - y[k]) / gap(N, theta, k);
    out[k1] += t;
    out[k] -= t;
  }
}

/* ------------------------------------------------------------------------ */
/* Dose z = D^T x and price g = D f (Sec. 2.1, Sec. 2.2)                     */
/* ------------------------------------------------------------------------ */
/* z_j = sum_i D_ij x_i: beamlet rows in order, entries in row order */
void vo_dose(int64_t B, int64_t V, const int64_t *row_ptr, const int32_t *vox,
             const double *val, const double *x, double *z) {
  for (int64_t j = 0; j < V; ++j) z[j] = 0.0;
  for (int64_t i = 0; i < B; ++i) {
    double xi = x[i];
    if (xi == 0.0) continue;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) z[vox[e]] += val[e] * xi;
  }
}

/* g_i = sum_j D_ij f_j for every beamlet of a beam with mask[k] != 0 (mask
 * NULL: all beams); other entries of g are left untouched. */
void vo_price(int64_t B, int32_t RC, const int64_t *row_ptr, const int32_t *vox,
              const double *val, const double *f, const uint8_t *mask, double *g) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < B; ++i) {
    if (mask && !mask[i / RC]) continue;
    double s = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * f[vox[e]];
    g[i] = s;
  }
}

/* fluence of apertures: x_i = y_k if column c of row r is open in beam k */
void vo_aperture_fluence(int N, int R, int C, const int16_t *l, const int16_t *r,
                         const double *y, double *x) {
  for (int k = 0; k < N; ++k)
    for (int rr = 0; rr < R; ++rr)
      for (int c = 0; c < C; ++c) {
        int64_t i = ((int64_t)k * R + rr) * C + c;
        x[i] = (c >= l[k * R + rr] && c < r[k * R + rr]) ? y[k] : 0.0;
      }
}

/* (A^T g)_k = sum over open beamlets of beam k of g_i (rows, then columns) */
void vo_aperture_adjoint(int N, int R, int C, const int16_t *l, const int16_t *r,
                         const double *g, double *out) {
  for (int k = 0; k < N; ++k) {
    double s = 0.0;
    for (int rr = 0; rr < R; ++rr)
      for (int c = l[k * R + rr]; c < r[k * R + rr]; ++c) s += g[((int64_t)k * R + rr) * C + c];
    out[k] = s;
  }
}

/* one column of the aperture-dose matrix: col_j = sum_{i in A_k} D_ij,
 * open beamlets in (row, column) order */
void vo_aperture_dose(int64_t V, int R, int C, const int64_t *row_ptr, const int32_t *vox,
                      const double *val, int k, const int16_t *l, const int16_t *r,
                      double *col) {
  for (int64_t j = 0; j < V; ++j) col[j] = 0.0;
  for (int rr = 0; rr < R; ++rr)
    for (int c = l[rr]; c < r[rr]; ++c) {
      int64_t i = ((int64_t)k * R + rr) * C + c;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) col[vox[e]] += val[e];
    }
}

/* ------------------------------------------------------------------------ */
/* Pricing subproblem (Sec. 2.2)                                              */
/* ------------------------------------------------------------------------ */
/* Leaf-position limits of beam k from the nearest beams with an aperture on
 * each side, d steps away: a leaf may be at most s*d columns from the
 * neighbour's.  Without an occupied neighbour a leaf ranges over [0, C]. */
void vo_leaf_limits(int N, int R, int C, int s, int cyclic, const uint8_t *occ,
                    const int16_t *lleaf, const int16_t *rleaf, int k, int *Llo, int *Lhi,
                    int *Rlo, int *Rhi) {
  int nb[2] = {-1, -1}, dist[2] = {0, 0};
  for (int side = 0; side < 2; ++side) {
    int step = side == 0 ? -1 : 1;
    for (int d = 1; d < N; ++d) {
      int q = k + step * d;
      if (cyclic) q = ((q % N) + N) % N;
      else if (q < 0 || q >= N) break;
      if (occ[q]) { nb[side] = q; dist[side] = d; break; }
    }
  }
  for (int rr = 0; rr < R; ++rr) {
    int llo = 0, lhi = C, rlo = 0, rhi = C;
    for (int side = 0; side < 2; ++side) {
      if (nb[side] < 0) continue;
      int m = s * dist[side];
      int ln = lleaf[nb[side] * R + rr], rn = rleaf[nb[side] * R + rr];
      if (ln - m > llo) llo = ln - m;
      if (ln + m < lhi) lhi = ln + m;
      if (rn - m > rlo) rlo = rn - m;
      if (rn + m < rhi) rhi = rn + m;
    }
    Llo[rr] = llo; Lhi[rr] = lhi; Rlo[rr] = rlo; Rhi[rr] = rhi;
  }
}

/* One left-to-right pass over a leaf row (prefix sums P[0]=0,
 * P[c+1]=P[c]+g[c]): open interval [l, r) has value P[r]-P[l].  For each r
 * the best l in [Llo, min(r, Lhi)] is the one of largest P[l] (ties: largest
 * l); over r keep the least value, then the shortest interval, then the
 * smallest l.  Returns 0, or -1 if no feasible (l, r) exists. */
int vo_row_scan(int C, const double *g, int Llo, int Lhi, int Rlo, int Rhi, double *value,
                int *lout, int *rout) {
  double P = 0.0, Pbest = 0.0;
  int lbest = -1, found = 0;
  double bv = 0.0;
  int bl = 0, br = 0;
  for (int c = 0; c <= C; ++c) {
    if (c > 0) P = P + g[c - 1];
    if (c >= Llo && c <= Lhi && (lbest < 0 || P >= Pbest)) { Pbest = P; lbest = c; }
    if (c >= Rlo && c <= Rhi && lbest >= 0) {
      double v = P - Pbest;
      int len = c - lbest;
      if (!found || v < bv || (v == bv && len < br - bl)) { bv = v; bl = lbest; br = c; found = 1; }
    }
  }
  if (!found) return -1;
  *value = bv; *lout = bl; *rout = br;
  return 0;
}

/* Same pass with P and the values formed in single precision. */
int vo_row_scan_f32(int C, const float *g, int Llo, int Lhi, int Rlo, int Rhi, float *value,
                    int *lout, int *rout) {
  volatile float P = 0.0f; /* volatile: keep every partial sum in single precision */
  float Pbest = 0.0f;
  int lbest = -1, found = 0;
  float bv = 0.0f;
  int bl = 0, br = 0;
  for (int c = 0; c <= C; ++c) {
    if (c > 0) P = P + g[c - 1];
    float Pc = P;
    if (c >= Llo && c <= Lhi && (lbest < 0 || Pc >= Pbest)) { Pbest = Pc; lbest = c; }
    if (c >= Rlo && c <= Rhi && lbest >= 0) {
      volatile float v = Pc - Pbest;
      int len = c - lbest;
      if (!found || v < bv || (v == bv && len < br - bl)) { bv = v; bl = lbest; br = c; found = 1; }
    }
  }
  if (!found) return -1;
  *value = bv; *lout = bl; *rout = br;
  return 0;
}

/* Least feasible value strictly above `best` over all (l, r) of the row, by
 * enumeration (used only to report how close a row decision was). */
static double row_runner_up(int C, const double *g, int Llo, int Lhi, int Rlo, int Rhi,
                            double best) {
  double out = INFINITY;
  for (int l = Llo; l <= Lhi; ++l)
    for (int r = l > Rlo ? l : Rlo; r <= Rhi; ++r) {
      double v = 0.0;
      for (int c = l; c < r; ++c) v += g[c];
      if (v > best && v < out) out = v;
    }
  return out;
}

/* Pricing over all beams without an aperture.  Aperture price p_k = sum of
 * the row values in row order (double).  Chosen beam: least p_k, ties to the
 * lowest k.  f32 != 0 runs the row scans in single precision on (float)g.
 * Outputs: k*, its leaves l/r [R], p*, the second-least price p2 (INFINITY
 * if only one candidate), and the least row margin (runner-up value minus
 * chosen value over the rows of k*, FP64 enumeration; NULL to skip).
 * offset [N] (NULL: none) is added to each beam's price after the row sum:
 * the column generation passes gamma * dG/dy_k of Eq. 2 at the current y for
 * the exact reduced cost of a new column (see vo_colgen).
 * res [2] (NULL to skip): the resolution of the decision when the row scans
 * run in single precision.  A row value P[r] - P[l] is a difference of
 * prefix sums, so one unit in the last place of the row's largest prefix sum
 * |P| (2^-23 of it) is the least change a one-ulp change of a single price
 * can make to it.  res[0] = 2^-23 times the sum over the rows of the chosen
 * beam and of the runner-up beam of their largest |P| (an absolute price);
 * res[1] = the least, over the rows of the chosen beam, of the row's margin
 * (runner-up value minus chosen value, FP64) over 2^-22 times its largest |P|.
 * Returns 0, -1 if no beam is free, -2 if some free beam has an infeasible row. */
/* sum over the rows of beam k of the largest |prefix sum| of the row */
static double beam_prefix_scale(int R, int C, const double *gk) {
  double sum = 0.0;
  for (int rr = 0; rr < R; ++rr) {
    double P = 0.0, mx = 0.0;
    for (int c = 0; c < C; ++c) {
      P += gk[(int64_t)rr * C + c];
      if (fabs(P) > mx) mx = fabs(P);
    }
    sum += mx;
  }
  return sum;
}

int vo_pricing(int N, int R, int C, int s, int cyclic, const uint8_t *occ, const int16_t *lleaf,
               const int16_t *rleaf, const double *g, int f32, int *kstar, int16_t *lout,
               int16_t *rout, double *pstar, double *p2, double *row_margin,
               const double *offset, double *res) {
  int *Llo = malloc(sizeof(int) * R * 4);
  int *Lhi = Llo + R, *Rlo = Llo + 2 * R, *Rhi = Llo + 3 * R;
  float *gf = malloc(sizeof(float) * C);
  int best = -1, ksecond = -1, status = 0;
  double bp = 0.0, second = INFINITY;
  for (int k = 0; k < N; ++k) {
    if (occ[k]) continue;
    vo_leaf_limits(N, R, C, s, cyclic, occ, lleaf, rleaf, k, Llo, Lhi, Rlo, Rhi);
    double p = 0.0;
    for (int rr = 0; rr < R; ++rr) {
      const double *grow = g + ((int64_t)k * R + rr) * C;
      int l, r, rc;
      double v;
      if (f32) {
        float vf;
        for (int c = 0; c < C; ++c) gf[c] = (float)grow[c];
        rc = vo_row_scan_f32(C, gf, Llo[rr], Lhi[rr], Rlo[rr], Rhi[rr], &vf, &l, &r);
        v = (double)vf;
      } else {
        rc = vo_row_scan(C, grow, Llo[rr], Lhi[rr], Rlo[rr], Rhi[rr], &v, &l, &r);
      }
      if (rc != 0) { status = -2; goto done; }
      p += v;
    }
    if (offset) p += offset[k];
    if (best < 0 || p < bp) {
      if (best >= 0) { second = bp; ksecond = best; }
      best = k; bp = p;
    } else if (p < second) {
      second = p;
      ksecond = k;
    }
  }
  if (best < 0) { status = -1; goto done; }
  vo_leaf_limits(N, R, C, s, cyclic, occ, lleaf, rleaf, best, Llo, Lhi, Rlo, Rhi);
  double margin = INFINITY, row_res = INFINITY;
  for (int rr = 0; rr < R; ++rr) {
    const double *grow = g + ((int64_t)best * R + rr) * C;
    int l, r;
    double v;
    if (f32) {
      float vf;
      for (int c = 0; c < C; ++c) gf[c] = (float)grow[c];
      vo_row_scan_f32(C, gf, Llo[rr], Lhi[rr], Rlo[rr], Rhi[rr], &vf, &l, &r);
      v = (double)vf;
    } else {
      vo_row_scan(C, grow, Llo[rr], Lhi[rr], Rlo[rr], Rhi[rr], &v, &l, &r);
    }
    lout[rr] = (int16_t)l; rout[rr] = (int16_t)r;
    if (row_margin || res) {
      double vx = 0.0; /* chosen interval's value in FP64 */
      for (int c = l; c < r; ++c) vx += grow[c];
      double ru = row_runner_up(C, grow, Llo[rr], Lhi[rr], Rlo[rr], Rhi[rr], vx);
      if (ru - vx < margin) margin = ru - vx;
      double unit = 0x1p-22 * beam_prefix_scale(1, C, grow);
      double q = unit > 0.0 ? (ru - vx) / unit : INFINITY;
      if (q < row_res) row_res = q;
    }
  }
  *kstar = best; *pstar = bp; *p2 = second;
  if (row_margin) *row_margin = margin;
  if (res) {
    double sc = beam_prefix_scale(R, C, g + (int64_t)best * R * C);
    if (ksecond >= 0) sc += beam_prefix_scale(R, C, g + (int64_t)ksecond * R * C);
    res[0] = 0x1p-23 * sc;
    res[1] = row_res;
  }
done:
  free(Llo);
  free(gf);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Master problem (Eq. 3 with the apertures fixed): projected gradient        */
/* ------------------------------------------------------------------------ */
typedef struct {
  double t;
  int64_t j;
} brk;

static int brk_cmp(const void *a, const void *b) {
  double x = ((const brk *)a)->t, y = ((const brk *)b)->t;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Exact minimiser over t in [0,1] of
 *   phi(t) = sum_j F(z_j + t w_j) + gamma*G(y + t d).
 * phi' is continuous, nondecreasing and linear between the voxel breakpoints
 * t_j = (T_j - z_j)/w_j; walk them in order until phi' changes sign. */
double vo_line_search(int64_t V, const double *z, const double *w, const uint8_t *sid,
                      const double *T, const double *al, const double *be, double gdot,
                      double Gd, double gamma) {
  /* phi'(t) = A + B t on the current piece */
  double A = gamma * gdot, Bc = 2.0 * gamma * Gd;
  brk *bk = malloc(sizeof(brk) * (V > 0 ? V : 1));
  int64_t nb = 0;
  for (int64_t j = 0; j < V; ++j) {
    double wj = w[j];
    if (wj == 0.0) continue;
    double e0 = z[j] - T[sid[j]];
    int over = e0 > 0.0 || (e0 == 0.0 && wj > 0.0);
    double c = over ? be[sid[j]] : al[sid[j]];
    A += 2.0 * c * wj * e0;
    Bc += 2.0 * c * wj * wj;
    double tj = -e0 / wj;
    if (tj > 0.0 && tj < 1.0) { bk[nb].t = tj; bk[nb].j = j; ++nb; }
  }
  qsort(bk, nb, sizeof(brk), brk_cmp);
  double lo = 0.0, t = 1.0;
  int done = 0;
  for (int64_t q = 0; q <= nb && !done; ++q) {
    double hi = q < nb ? bk[q].t : 1.0;
    if (A + Bc * hi >= 0.0) {
      double root = Bc > 0.0 ? -A / Bc : lo;
      t = root < lo ? lo : (root > hi ? hi : root);
      done = 1;
      break;
    }
    if (q == nb) break;
    /* voxel j crosses its threshold at hi: swap its side */
    int64_t j = bk[q].j;
    double wj = w[j], e0 = z[j] - T[sid[j]];
    double cold, cnew;
    if (wj > 0.0) { cold = al[sid[j]]; cnew = be[sid[j]]; }
    else { cold = be[sid[j]]; cnew = al[sid[j]]; }
    A += 2.0 * (cnew - cold) * wj * e0;
    Bc += 2.0 * (cnew - cold) * wj * wj;
    lo = hi;
  }
  if (!done) t = 1.0;
  free(bk);
  return t;
}

/* Gradient of f(y) = sum_j F((My)_j) + gamma*G(y) on the occupied beams.
 * M holds ncol columns of length V; column q belongs to beam col_beam[q]. */
static void master_grad(int64_t V, int ncol, const double *M, const int32_t *col_beam, int N,
                        const double *theta, int cyclic, double gamma, const double *fp,
                        const double *y, double *grad) {
  vo_dG(N, theta, y, cyclic, grad);
  for (int k = 0; k < N; ++k) grad[k] *= gamma;
  double *dots = malloc(sizeof(double) * (ncol > 0 ? ncol : 1));
#pragma omp parallel for schedule(static)
  for (int q = 0; q < ncol; ++q) {
    const double *m = M + (int64_t)q * V;
    double s = 0.0;
    for (int64_t j = 0; j < V; ++j) s += m[j] * fp[j];
    dots[q] = s;
  }
  for (int q = 0; q < ncol; ++q) grad[col_beam[q]] += dots[q];
  free(dots);
}

/* v = M u restricted to columns: v_j = sum_q M[q][j] * u[col_beam[q]] */
static void master_apply(int64_t V, int ncol, const double *M, const int32_t *col_beam,
                         const double *u, double *v) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < V; ++j) {
    double s = 0.0;
    for (int q = 0; q < ncol; ++q) s += M[(int64_t)q * V + j] * u[col_beam[q]];
    v[j] = s;
  }
}

/* Natural KKT residual of min f(y), y_k >= 0 (k occupied), y_k = 0 otherwise:
 * rho = max over occupied k of |min(y_k, grad_k)|. */
static double kkt_residual(int ncol, const int32_t *col_beam, const double *y, const double *g) {
  double r = 0.0;
  for (int q = 0; q < ncol; ++q) {
    int k = col_beam[q];
    double m = y[k] < g[k] ? y[k] : g[k];
    if (fabs(m) > r) r = fabs(m);
  }
  return r;
}

/* Step rule of the gradient projection: adaptive Barzilai-Borwein (ABBmin,
 * Frassoldati, Zanni and Zanghirati 2008) with a memory of ABB_M short steps
 * and switch ratio ABB_TAU for the first ABB_ITERS iterations of a solve, the
 * short step alone after them. */
#define ABB_M 3
#define ABB_TAU 0.5
#define ABB_ITERS 300

/* Projected gradient for the master problem.  y [N] is the warm start on
 * entry (zero at beams without a column) and the solution on exit; z [V]
 * receives M y.  Step from the previous move dy and gradient change dg (over
 * beams with a column): the short Barzilai-Borwein step BB2 = dy.dg / dg.dg
 * (1e12 unless both are positive) and the long one BB1 = dy.dy / dy.dg
 * (1e12 unless dy.dg > 0); where BB2 < ABB_TAU * BB1 the step is the least
 * BB2 of this and the previous ABB_M - 1 iterations, else BB1 (from
 * iteration ABB_ITERS on: BB2); clamped to
 * [1e-12, 1e12]; the first step is max(|y|_inf, 1)/|g|_inf; direction
 * d = P+(y - s g) - y; exact line search on [0,1].  Stops when
 * rho <= eps * max(rho_start, rho_ref, 1e-300) or after max_iter
 * iterations; rho_ref is a caller-given scale (column generation passes the
 * residual at the start of the plan's first master problem, so that a
 * column that brings no improvement does not demand an unreachable
 * absolute accuracy).
 * Returns 0 on convergence, 1 on hitting max_iter, 2 if the line search
 * returns t = 0 before convergence.  out[0..3] = cost, rho, rho_start, iters. */
int vo_master(int64_t V, int ncol, const double *M, const int32_t *col_beam, int N,
              const double *theta, int cyclic, double gamma, const uint8_t *sid,
              const double *T, const double *al, const double *be, double eps,
              double rho_ref, int max_iter, double *y, double *z, double *out) {
  double *fp = malloc(sizeof(double) * V);
  double *w = malloc(sizeof(double) * V);
  double *g = malloc(sizeof(double) * N), *gold = malloc(sizeof(double) * N);
  double *d = calloc(N, sizeof(double)), *dG = malloc(sizeof(double) * N);
  master_apply(V, ncol, M, col_beam, y, z);
  vo_voxel_dcost(V, z, sid, T, al, be, fp);
  master_grad(V, ncol, M, col_beam, N, theta, cyclic, gamma, fp, y, g);
  double rho = kkt_residual(ncol, col_beam, y, g);
  double rho0 = rho, scale = rho0 > rho_ref ? rho0 : rho_ref;
  double tol = eps * (scale > 1e-300 ? scale : 1e-300);
  int it = 0, status = 1;
  double dgg = 0.0, dyg = 0.0, dyy = 0.0;
  double bb2_hist[ABB_M - 1]; /* previous short steps, newest first */
  for (int q = 0; q < ABB_M - 1; ++q) bb2_hist[q] = INFINITY;
  for (it = 0; it < max_iter; ++it) {
    if (rho <= tol) { status = 0; break; }
    double step;
    if (it == 0) {
      double ym = 0.0, gm = 0.0;
      for (int q = 0; q < ncol; ++q) {
        int k = col_beam[q];
        if (fabs(y[k]) > ym) ym = fabs(y[k]);
        if (fabs(g[k]) > gm) gm = fabs(g[k]);
      }
      step = (ym > 1.0 ? ym : 1.0) / (gm > 1e-300 ? gm : 1e-300);
    } else {
      double bb2 = (dyg > 0.0 && dgg > 0.0) ? dyg / dgg : 1e12;
      double bb1 = dyg > 0.0 ? dyy / dyg : 1e12;
      double hmin = bb2;
      for (int q = 0; q < ABB_M - 1; ++q)
        if (bb2_hist[q] < hmin) hmin = bb2_hist[q];
      for (int q = ABB_M - 2; q > 0; --q) bb2_hist[q] = bb2_hist[q - 1];
      bb2_hist[0] = bb2;
      step = it >= ABB_ITERS ? bb2 : (bb2 < ABB_TAU * bb1 ? hmin : bb1);
    }
    if (step < 1e-12) step = 1e-12;
    if (step > 1e12) step = 1e12;
    for (int k = 0; k < N; ++k) d[k] = 0.0;
    for (int q = 0; q < ncol; ++q) {
      int k = col_beam[q];
      double p = y[k] - step * g[k];
      d[k] = (p > 0.0 ? p : 0.0) - y[k];
    }
    master_apply(V, ncol, M, col_beam, d, w);
    vo_dG(N, theta, y, cyclic, dG);
    double gdot = 0.0;
    for (int k = 0; k < N; ++k) gdot += dG[k] * d[k];
    double Gd = vo_G(N, theta, d, cyclic);
    double t = vo_line_search(V, z, w, sid, T, al, be, gdot, Gd, gamma);
    if (t <= 0.0) { status = 2; break; }
    for (int k = 0; k < N; ++k) y[k] += t * d[k];
    for (int64_t j = 0; j < V; ++j) z[j] += t * w[j];
    memcpy(gold, g, sizeof(double) * N);
    vo_voxel_dcost(V, z, sid, T, al, be, fp);
    master_grad(V, ncol, M, col_beam, N, theta, cyclic, gamma, fp, y, g);
    dgg = 0.0; dyg = 0.0; dyy = 0.0;
    for (int q = 0; q < ncol; ++q) {
      int k = col_beam[q];
      double dy = t * d[k], dg = g[k] - gold[k];
      dgg += dg * dg;
      dyg += dy * dg;
      dyy += dy * dy;
    }
    rho = kkt_residual(ncol, col_beam, y, g);
  }
  if (status == 1 && rho <= tol) status = 0;
  out[0] = vo_voxel_cost(V, z, sid, T, al, be) + gamma * vo_G(N, theta, y, cyclic);
  out[1] = rho;
  out[2] = rho0;
  out[3] = (double)it;
  free(fp); free(w); free(g); free(gold); free(d); free(dG);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Column generation (Sec. 2.2, Fig. 1)                                       */
/* ------------------------------------------------------------------------ */
/* Runs n_iter iterations from an empty plan: prices (Sec. 2.2) from
 * F'(z), pricing over beams without an aperture, add the column, re-solve the
 * master.  If forced_k is non-NULL iteration t takes beam forced_k[t] with
 * leaves forced_l/forced_r [n_iter*R] instead of the pricing result (replay).
 * Per-iteration records (arrays of n_iter): beam, p*, angle margin
 * (p2-p*)/max(|p*|,1e-300), least row margin / max(|p*|,1e-300), the
 * single-precision resolution of the beam decision / max(|p*|,1e-300) and
 * the least row margin in units of its row's resolution (see vo_pricing;
 * either record may be NULL), cost, rho, master iterations, master status.  The master problems stop at
 * rho <= eps * max(rho_start, rho_plan), rho_plan = the residual at the start
 * of the first one.  Final y [N], z [V], leaves
 * lleaf/rleaf [N*R] (rows of beams without an aperture are 0).
 * price_smoothing != 0 prices a beam by the exact reduced cost of its new
 * column: the derivative of Eq. 3 along it is the summed beamlet price of
 * the aperture plus gamma * dG/dy_k at the current y (y_k = 0 for a beam
 * without an aperture, so the term is -2 gamma times the neighbours'
 * intensities over their gaps, never positive); otherwise the aperture price
 * is the beamlet sum alone, as the paper states it.
 * Returns 0, or a negative pricing status. */
int vo_colgen(int64_t V, int N, int R, int C, const int64_t *row_ptr, const int32_t *vox,
              const double *val, const uint8_t *sid, const double *T, const double *al,
              const double *be, const double *theta, double gamma, int cyclic, int s,
              int n_iter, double eps, int max_iter, const int32_t *forced_k,
              const int16_t *forced_l, const int16_t *forced_r, int f32_pricing,
              int price_smoothing, int32_t *rec_k, double *rec_p, double *rec_margin, double *rec_row_margin,
              double *rec_res, double *rec_row_res,
              double *rec_cost, double *rec_rho, int32_t *rec_iters, int32_t *rec_status,
              double *y, double *z, int16_t *lleaf, int16_t *rleaf) {
  const int64_t B = (int64_t)N * R * C;
  double *M = malloc(sizeof(double) * V * (n_iter > 0 ? n_iter : 1));
  int32_t *col_beam = malloc(sizeof(int32_t) * (n_iter > 0 ? n_iter : 1));
  uint8_t *occ = calloc(N, 1), *mask = malloc(N);
  double *fp = malloc(sizeof(double) * V), *g = calloc(B, sizeof(double));
  int16_t *lk = malloc(sizeof(int16_t) * R), *rk = malloc(sizeof(int16_t) * R);
  double *off = malloc(sizeof(double) * N);
  int status = 0;
  double rho_plan = 0.0;
  for (int k = 0; k < N; ++k) y[k] = 0.0;
  for (int64_t j = 0; j < V; ++j) z[j] = 0.0;
  memset(lleaf, 0, sizeof(int16_t) * N * R);
  memset(rleaf, 0, sizeof(int16_t) * N * R);
  for (int t = 0; t < n_iter; ++t) {
    vo_voxel_dcost(V, z, sid, T, al, be, fp);
    for (int k = 0; k < N; ++k) mask[k] = !occ[k];
    vo_price(B, R * C, row_ptr, vox, val, fp, mask, g);
    int k;
    double p, p2, rm;
    if (price_smoothing) {
      vo_dG(N, theta, y, cyclic, off);
      for (int q = 0; q < N; ++q) off[q] *= gamma;
    }
    double res[2];
    int rc = vo_pricing(N, R, C, s, cyclic, occ, lleaf, rleaf, g, f32_pricing, &k, lk, rk, &p,
                        &p2, &rm, price_smoothing ? off : NULL, res);
    if (rc != 0) { status = rc; break; }
    double scale = fabs(p) > 1e-300 ? fabs(p) : 1e-300;
    rec_p[t] = p;
    rec_margin[t] = (p2 - p) / scale;
    rec_row_margin[t] = rm / scale;
    if (rec_res) rec_res[t] = res[0] / scale;
    if (rec_row_res) rec_row_res[t] = res[1];
    if (forced_k) {
      k = forced_k[t];
      memcpy(lk, forced_l + (int64_t)t * R, sizeof(int16_t) * R);
      memcpy(rk, forced_r + (int64_t)t * R, sizeof(int16_t) * R);
    }
    rec_k[t] = k;
    vo_aperture_dose(V, R, C, row_ptr, vox, val, k, lk, rk, M + (int64_t)t * V);
    col_beam[t] = k;
    occ[k] = 1;
    memcpy(lleaf + k * R, lk, sizeof(int16_t) * R);
    memcpy(rleaf + k * R, rk, sizeof(int16_t) * R);
    y[k] = 0.0;
    double out[4];
    rec_status[t] = vo_master(V, t + 1, M, col_beam, N, theta, cyclic, gamma, sid, T, al, be,
                              eps, rho_plan, max_iter, y, z, out);
    if (t == 0) rho_plan = out[2];
    rec_cost[t] = out[0];
    rec_rho[t] = out[1];
    rec_iters[t] = (int32_t)out[3];
  }
  free(M); free(col_beam); free(occ); free(mask); free(fp); free(g); free(lk); free(rk);
  free(off);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Dose-volume histograms (plan evaluation, Fig. 2)                           */
/* ------------------------------------------------------------------------ */
/* counts[s*n_bins + b] = number of voxels j of structure s = sid[j] whose
 * dose lies in bin b, i.e. b*w <= z_j < (b+1)*w with w = dose_max/n_bins;
 * z_j >= dose_max goes to the last bin and z_j < 0 to the first.  The bin is
 * found by comparing z_j with the edges b*dose_max/n_bins (each edge one
 * FP64 product and quotient), scanning up from bin 0: plain and slow, and
 * independent of how a kernel rounds z_j * n_bins / dose_max. */
void vo_dvh(int64_t V, const double *z, const uint8_t *sid, int n_struct, double dose_max,
            int n_bins, int64_t *counts) {
  for (int64_t q = 0; q < (int64_t)n_struct * n_bins; ++q) counts[q] = 0;
  for (int64_t j = 0; j < V; ++j) {
    int b = 0;
    while (b + 1 < n_bins && z[j] >= (double)(b + 1) * dose_max / (double)n_bins) ++b;
    counts[(int64_t)sid[j] * n_bins + b] += 1;
  }
}

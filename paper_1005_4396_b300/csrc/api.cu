// Public entry points of libvmat (see include/vmat.h) and the column-generation
// loop of Sec. 2.2 (Fig. 1): prices -> pricing -> add column -> master problem,
// enqueued entirely on the context's stream; the host reads the records once.
#include <math.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "vmat_internal.cuh"

vmat_status vmat_launch_pricing_rec(vmat_ctx *ctx, const float *g, int32_t *rec_k, double *rec_p,
                                    double *rec_p2);
vmat_status vmat_launch_force(vmat_ctx *ctx, const int32_t *fk, const int16_t *fl,
                              const int16_t *fr, int t);

static vmat_status sync_status(vmat_ctx *ctx) {
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int ds = 0;
  VMAT_CUDA(ctx, cudaMemcpy(&ds, ctx->dstatus, 4, cudaMemcpyDeviceToHost));
  if (ds == VMAT_ETIMEOUT) return vmat_fail(ctx, VMAT_ETIMEOUT, "a bounded device wait ran out");
  if (ds != 0) return vmat_fail(ctx, (vmat_status)ds, "device reported status %d", ds);
  return VMAT_OK;
}

extern "C" vmat_status vmat_dose(vmat_ctx *ctx, const float *x_dev, float *z_dev, float *fprime_dev,
                                 double *cost_host) {
  if (!ctx || !x_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "x is NULL") : VMAT_EINVAL;
  double *cdev = cost_host ? ctx->red + ctx->red_len - 1 : nullptr;
  vmat_status s = vmat_launch_dose(ctx, x_dev, z_dev, fprime_dev, cdev);
  if (s != VMAT_OK) return s;
  if (cost_host) {
    double c = 0.0;
    VMAT_CUDA(ctx, cudaMemcpyAsync(&c, cdev, 8, cudaMemcpyDeviceToHost, ctx->stream));
    VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *cost_host = c + ctx->inactive_cost;
  }
  return sync_status(ctx);
}

extern "C" vmat_status vmat_price(vmat_ctx *ctx, const float *f_dev, const uint8_t *angle_mask_dev,
                                  float *g_dev) {
  if (!ctx || !f_dev || !g_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = vmat_gather_active(ctx, f_dev, ctx->fgather);
  if (s != VMAT_OK) return s;
  s = vmat_launch_price(ctx, ctx->fgather, angle_mask_dev, angle_mask_dev ? 1 : 0, g_dev);
  if (s != VMAT_OK) return s;
  return sync_status(ctx);
}

extern "C" vmat_status vmat_pricing_select(vmat_ctx *ctx, const float *g_dev, vmat_column *out) {
  if (!ctx || !g_dev || !out || !out->l || !out->r)
    return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = vmat_launch_pricing(ctx, g_dev);
  if (s != VMAT_OK) return s;
  SelRec r;
  VMAT_CUDA(ctx, cudaMemcpyAsync(&r, ctx->sel, sizeof r, cudaMemcpyDeviceToHost, ctx->stream));
  VMAT_CUDA(ctx, cudaMemcpyAsync(out->l, ctx->sel_l, ctx->R * 2, cudaMemcpyDeviceToHost, ctx->stream));
  VMAT_CUDA(ctx, cudaMemcpyAsync(out->r, ctx->sel_r, ctx->R * 2, cudaMemcpyDeviceToHost, ctx->stream));
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out->angle = r.k;
  out->price = r.p;
  out->runner_up = r.p2;
  if (r.status != 0)
    return vmat_fail(ctx, VMAT_ESTATE, r.k < 0 ? "no free beam" : "a free beam has a leaf row with no feasible interval");
  return VMAT_OK;
}

extern "C" vmat_status vmat_add_column(vmat_ctx *ctx, const vmat_column *col) {
  if (!ctx || !col || !col->l || !col->r)
    return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  if (col->angle < 0 || col->angle >= ctx->N) return vmat_fail(ctx, VMAT_EINVAL, "angle out of range");
  if (ctx->n_slots >= ctx->N) return vmat_fail(ctx, VMAT_ESTATE, "every beam has an aperture");
  for (int r = 0; r < ctx->R; ++r)
    if (col->l[r] < 0 || col->l[r] > col->r[r] || col->r[r] > ctx->C)
      return vmat_fail(ctx, VMAT_EINVAL, "row %d: leaves must satisfy 0 <= l <= r <= C", r);
  uint8_t occ = 0;
  VMAT_CUDA(ctx, cudaMemcpy(&occ, ctx->occ + col->angle, 1, cudaMemcpyDeviceToHost));
  if (occ) return vmat_fail(ctx, VMAT_EINVAL, "beam %d already has an aperture", col->angle);
  SelRec r = {col->angle, 0, col->price, col->runner_up};
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->sel, &r, sizeof r, cudaMemcpyHostToDevice, ctx->stream));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->sel_l, col->l, ctx->R * 2, cudaMemcpyHostToDevice, ctx->stream));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->sel_r, col->r, ctx->R * 2, cudaMemcpyHostToDevice, ctx->stream));
  vmat_status s = vmat_launch_add_column(ctx, ctx->n_slots);
  if (s != VMAT_OK) return s;
  s = sync_status(ctx);
  if (s != VMAT_OK) return s;
  ctx->n_slots += 1;
  return VMAT_OK;
}

extern "C" vmat_status vmat_master_step(vmat_ctx *ctx, int32_t max_iters, double kkt_tol,
                                        double rho_ref, double *y_host, double *cost, double *kkt,
                                        int32_t *iters) {
  if (!ctx) return VMAT_EINVAL;
  if (max_iters < 0 || !(kkt_tol >= 0.0) || !(rho_ref >= 0.0))
    return vmat_fail(ctx, VMAT_EINVAL, "max_iters >= 0, kkt_tol >= 0, rho_ref >= 0 required");
  if (y_host) {
    std::vector<uint8_t> occ(ctx->N);
    VMAT_CUDA(ctx, cudaMemcpy(occ.data(), ctx->occ, ctx->N, cudaMemcpyDeviceToHost));
    for (int k = 0; k < ctx->N; ++k)
      if (!(y_host[k] >= 0.0) || !isfinite(y_host[k]) || (!occ[k] && y_host[k] != 0.0))
        return vmat_fail(ctx, VMAT_EINVAL,
                         "y must be finite, >= 0, and 0 at beams without an aperture (k=%d)", k);
    VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->y, y_host, ctx->N * 8, cudaMemcpyHostToDevice, ctx->stream));
  }
  vmat_status s = vmat_launch_master(ctx, max_iters, kkt_tol, rho_ref, 0, nullptr, nullptr,
                                     nullptr, nullptr);
  if (s != VMAT_OK) return s;
  MasterOut o;
  VMAT_CUDA(ctx, cudaMemcpyAsync(&o, ctx->mout, sizeof o, cudaMemcpyDeviceToHost, ctx->stream));
  if (y_host)
    VMAT_CUDA(ctx, cudaMemcpyAsync(y_host, ctx->y, ctx->N * 8, cudaMemcpyDeviceToHost, ctx->stream));
  s = sync_status(ctx);
  if (s != VMAT_OK) return s;
  if (cost) *cost = o.cost_active + ctx->inactive_cost + ctx->gamma * o.smooth;
  if (kkt) *kkt = o.rho;
  if (iters) *iters = o.iters;
  if (o.status == VMAT_ETIMEOUT) return vmat_fail(ctx, VMAT_ETIMEOUT, "master: bounded wait ran out");
  if (o.status != VMAT_OK)
    return vmat_fail(ctx, VMAT_ENOTCONV, "master: rho %.3e after %d iterations", o.rho, o.iters);
  return VMAT_OK;
}

// Largest dose-rate variation over neighbouring beams with an aperture or
// without (y = 0 there), |y_k' - y_k| / gap(k, k') in intensity units per
// degree, minus the limit: <= 0 when the plan meets it.
static double rate_violation(const vmat_ctx *ctx, const std::vector<double> &y, double max_rate) {
  const int N = ctx->N;
  double worst = -INFINITY;
  for (int k = 0; k + 1 < N || (ctx->cyclic && N > 1 && k < N); ++k) {
    const int kp = k + 1 < N ? k + 1 : 0;
    if (kp == k) break;
    const double gap = kp > k ? ctx->theta_h[kp] - ctx->theta_h[k]
                              : ctx->theta_h[0] + 360.0 - ctx->theta_h[N - 1];
    worst = fmax(worst, fabs(y[kp] - y[k]) / gap - max_rate);
  }
  return N > 1 ? worst : -max_rate;
}

extern "C" vmat_status vmat_dose_rate_feasibility(vmat_ctx *ctx, double max_rate, double gamma_factor,
                                                  int32_t max_rounds, int32_t master_max_iters,
                                                  double kkt_tol, double *y_host, double *gamma_out,
                                                  int32_t *rounds_out, double *violation_out,
                                                  double *cost_out) {
  if (!ctx) return VMAT_EINVAL;
  if (!(max_rate >= 0.0) || !isfinite(max_rate) || !(gamma_factor > 1.0) || !isfinite(gamma_factor) ||
      max_rounds < 0 || master_max_iters < 0 || !(kkt_tol >= 0.0))
    return vmat_fail(ctx, VMAT_EINVAL,
                     "max_rate >= 0, gamma_factor > 1, max_rounds >= 0, master_max_iters >= 0 and "
                     "kkt_tol >= 0 required");
  const int N = ctx->N;
  std::vector<double> y(N);
  VMAT_CUDA(ctx, cudaMemcpyAsync(y.data(), ctx->y, N * 8, cudaMemcpyDeviceToHost, ctx->stream));
  vmat_status s = sync_status(ctx);
  if (s != VMAT_OK) return s;
  const double gamma0 = ctx->gamma;
  double v = rate_violation(ctx, y, max_rate);
  int rounds = 0;
  MasterOut o = {};
  // the cost at the current plan (a master launch of no iterations), then one
  // master solve per round with gamma raised, warm-started from the last y
  for (;;) {
    const bool more = v > 0.0 && rounds < max_rounds;
    if (more) {
      ctx->gamma *= gamma_factor;
      ++rounds;
    }
    s = vmat_launch_master(ctx, more ? master_max_iters : 0, kkt_tol, 0.0, 0, nullptr, nullptr,
                           nullptr, nullptr);
    if (s == VMAT_OK) {
      VMAT_CUDA(ctx, cudaMemcpyAsync(&o, ctx->mout, sizeof o, cudaMemcpyDeviceToHost, ctx->stream));
      VMAT_CUDA(ctx, cudaMemcpyAsync(y.data(), ctx->y, N * 8, cudaMemcpyDeviceToHost, ctx->stream));
      s = sync_status(ctx);
    }
    if (s == VMAT_OK && o.status == VMAT_ETIMEOUT)
      s = vmat_fail(ctx, VMAT_ETIMEOUT, "master: bounded wait ran out");
    if (s != VMAT_OK) {
      ctx->gamma = gamma0;
      return s;
    }
    v = rate_violation(ctx, y, max_rate);
    if (!more) break;
  }
  if (y_host) std::copy(y.begin(), y.end(), y_host);
  if (gamma_out) *gamma_out = ctx->gamma;
  if (rounds_out) *rounds_out = rounds;
  if (violation_out) *violation_out = v;
  if (cost_out) *cost_out = o.cost_active + ctx->inactive_cost + ctx->gamma * o.smooth;
  ctx->gamma = gamma0;
  if (v > 0.0)
    return vmat_fail(ctx, VMAT_ENOTCONV, "dose-rate limit still exceeded by %.3e after %d rounds", v,
                     rounds);
  return VMAT_OK;
}

__global__ void k_scatter_active(const float *__restrict__ act_val, const int32_t *__restrict__ act,
                                 int32_t Va, float *__restrict__ full) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < Va) full[act[a]] = act_val[a];
}

extern "C" vmat_status vmat_plan_dose(vmat_ctx *ctx, float *z_dev) {
  if (!ctx || !z_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "z is NULL") : VMAT_EINVAL;
  VMAT_CUDA(ctx, cudaMemsetAsync(z_dev, 0, (size_t)ctx->V * 4, ctx->stream));
  if (ctx->Va > 0)
    k_scatter_active<<<(ctx->Va + 255) / 256, 256, 0, ctx->stream>>>(ctx->zact, ctx->act_vox,
                                                                     ctx->Va, z_dev);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  return sync_status(ctx);
}

// ---------------------------------------------------------------- column generation
vmat_status vmat_enqueue_colgen(vmat_ctx *ctx, int n, int master_max_iters, double kkt_tol,
                                const Records &rec, bool fresh) {
  for (int t = 0; t < n; ++t) {
    vmat_status s = vmat_launch_price(ctx, ctx->fpact, ctx->occ, 2, ctx->g, ctx->master_xp ? ctx->fplo : nullptr);
    if (s != VMAT_OK) return s;
    s = vmat_launch_pricing_rec(ctx, ctx->g, rec.k + t, rec.p + t, rec.p2 + t);
    if (s != VMAT_OK) return s;
    s = vmat_launch_add_column(ctx, ctx->n_slots, rec.tiles + t);
    if (s != VMAT_OK) return s;
    ctx->n_slots += 1;
    s = vmat_launch_master(ctx, master_max_iters, kkt_tol, 0.0, fresh && t == 0 ? 1 : 0,
                           rec.cost + t, rec.rho + t, rec.iters + t, rec.status + t);
    if (s != VMAT_OK) return s;
  }
  return VMAT_OK;
}

extern "C" vmat_status vmat_colgen_run(vmat_ctx *ctx, const vmat_colgen_opts *o,
                                       vmat_colgen_result *res) {
  if (!ctx || !o) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  const int n = o->n_iters, N = ctx->N, R = ctx->R;
  if (n < 0 || n > N - ctx->n_slots)
    return vmat_fail(ctx, VMAT_EINVAL, "n_iters must be in [0, free beams = %d]", N - ctx->n_slots);
  if (o->master_max_iters < 0 || !(o->kkt_tol >= 0.0))
    return vmat_fail(ctx, VMAT_EINVAL, "master_max_iters >= 0 and kkt_tol >= 0 required");
  if (o->forced_angle) {
    if (!o->forced_l || !o->forced_r) return vmat_fail(ctx, VMAT_EINVAL, "forced leaves missing");
    std::vector<uint8_t> used(N, 0);
    std::vector<uint8_t> occ(N);
    VMAT_CUDA(ctx, cudaMemcpy(occ.data(), ctx->occ, N, cudaMemcpyDeviceToHost));
    for (int t = 0; t < n; ++t) {
      int k = o->forced_angle[t];
      if (k < 0 || k >= N || used[k] || occ[k])
        return vmat_fail(ctx, VMAT_EINVAL, "forced beam %d invalid or repeated", k);
      used[k] = 1;
      for (int r = 0; r < R; ++r) {
        int l = o->forced_l[(int64_t)t * R + r], rr = o->forced_r[(int64_t)t * R + r];
        if (l < 0 || l > rr || rr > ctx->C) return vmat_fail(ctx, VMAT_EINVAL, "forced leaves invalid");
      }
    }
  }
  cudaStream_t st = ctx->stream;
  // device records (one block) and forced plan
  size_t nn = n > 0 ? n : 1;
  const bool want_priced = res && (res->priced_l || res->priced_r);
  size_t bytes = nn * (4 * 4 + 4 * 8) + 64 + (o->forced_angle ? nn * (4 + 4 * (size_t)R) + 64 : 0) +
                 (want_priced ? nn * 4 * (size_t)R + 64 : 0);
  char *blk = nullptr;
  VMAT_CUDA(ctx, cudaMallocAsync((void **)&blk, bytes, st));
  Records rec;
  rec.p = (double *)blk;
  rec.p2 = rec.p + nn;
  rec.cost = rec.p2 + nn;
  rec.rho = rec.cost + nn;
  rec.k = (int32_t *)(rec.rho + nn);
  rec.iters = rec.k + nn;
  rec.status = rec.iters + nn;
  rec.tiles = rec.status + nn;
  int32_t *fk = nullptr;
  int16_t *fl = nullptr, *fr = nullptr;
  int16_t *pl = nullptr, *pr = nullptr;  // leaves of the pricing result at every iteration
  char *tail = (char *)(rec.tiles + nn);
  if (want_priced) {
    pl = (int16_t *)(((uintptr_t)tail + 15) & ~(uintptr_t)15);
    pr = pl + nn * R;
    tail = (char *)(pr + nn * R);
  }
  if (o->forced_angle) {
    fk = (int32_t *)(((uintptr_t)tail + 15) & ~(uintptr_t)15);
    fl = (int16_t *)(fk + nn);
    fr = fl + nn * R;
    cudaMemcpyAsync(fk, o->forced_angle, n * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(fl, o->forced_l, (size_t)n * R * 2, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(fr, o->forced_r, (size_t)n * R * 2, cudaMemcpyHostToDevice, st);
  }
  vmat_status s = VMAT_OK;
  const bool fresh = ctx->n_slots == 0;
  // optional phase timing: 5 events per iteration bracket its 4 phases
  const bool prof = ctx->profiling && res && res->phase_ms && n > 0;
  std::vector<cudaEvent_t> ev;
  if (prof) {
    ev.resize((size_t)n * 5);
    for (auto &e : ev) VMAT_CUDA(ctx, cudaEventCreate(&e));
  }
  auto mark = [&](int t, int q) {
    if (prof) cudaEventRecord(ev[(size_t)t * 5 + q], st);
  };
  for (int t = 0; t < n && s == VMAT_OK; ++t) {
    mark(t, 0);
    // prices of the free beams from F'(z) of the current plan dose
    s = vmat_launch_price(ctx, ctx->fpact, ctx->occ, 2, ctx->g, ctx->master_xp ? ctx->fplo : nullptr);
    if (s != VMAT_OK) break;
    mark(t, 1);
    s = vmat_launch_pricing_rec(ctx, ctx->g, rec.k + t, rec.p + t, rec.p2 + t);
    if (s != VMAT_OK) break;
    if (pl) {  // the pricing's own leaves, before a forced aperture replaces them
      cudaMemcpyAsync(pl + (size_t)t * R, ctx->sel_l, (size_t)R * 2, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(pr + (size_t)t * R, ctx->sel_r, (size_t)R * 2, cudaMemcpyDeviceToDevice, st);
    }
    if (fk) {
      s = vmat_launch_force(ctx, fk, fl, fr, t);
      if (s != VMAT_OK) break;
    }
    mark(t, 2);
    s = vmat_launch_add_column(ctx, ctx->n_slots, rec.tiles + t);
    if (s != VMAT_OK) break;
    ctx->n_slots += 1;
    mark(t, 3);
    s = vmat_launch_master(ctx, o->master_max_iters, o->kkt_tol, 0.0, fresh && t == 0 ? 1 : 0,
                           rec.cost + t, rec.rho + t, rec.iters + t, rec.status + t);
    mark(t, 4);
  }
  // rec.k holds the pricing's choice; with forcing, the beam added is the forced one
  std::vector<int32_t> hk(nn), hit(nn), hst(nn), htl(nn);
  std::vector<double> hp(nn), hp2(nn), hc(nn), hr(nn);
  if (n > 0) {
    cudaMemcpyAsync(hk.data(), rec.k, n * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hit.data(), rec.iters, n * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hst.data(), rec.status, n * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(htl.data(), rec.tiles, n * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hp.data(), rec.p, n * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hp2.data(), rec.p2, n * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hc.data(), rec.cost, n * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hr.data(), rec.rho, n * 8, cudaMemcpyDeviceToHost, st);
  }
  if (n > 0 && pl) {
    if (res->priced_l) cudaMemcpyAsync(res->priced_l, pl, (size_t)n * R * 2, cudaMemcpyDeviceToHost, st);
    if (res->priced_r) cudaMemcpyAsync(res->priced_r, pr, (size_t)n * R * 2, cudaMemcpyDeviceToHost, st);
  }
  if (res && res->l) cudaMemcpyAsync(res->l, ctx->lleaf, (size_t)N * R * 2, cudaMemcpyDeviceToHost, st);
  if (res && res->r) cudaMemcpyAsync(res->r, ctx->rleaf, (size_t)N * R * 2, cudaMemcpyDeviceToHost, st);
  if (res && res->y) cudaMemcpyAsync(res->y, ctx->y, (size_t)N * 8, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(blk, st);
  vmat_status s2 = sync_status(ctx);
  if (prof) {
    if (s == VMAT_OK && s2 == VMAT_OK)
      for (int t = 0; t < n; ++t)
        for (int q = 0; q < 4; ++q) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, ev[(size_t)t * 5 + q], ev[(size_t)t * 5 + q + 1]);
          res->phase_ms[(size_t)t * 4 + q] = ms;
        }
    for (auto &e : ev) cudaEventDestroy(e);
  }
  if (s != VMAT_OK) return s;
  if (s2 != VMAT_OK) return s2;
  if (res) {
    for (int t = 0; t < n; ++t) {
      if (res->angle_order) res->angle_order[t] = o->forced_angle ? o->forced_angle[t] : hk[t];
      if (res->priced_angle) res->priced_angle[t] = hk[t];
      if (res->price) res->price[t] = hp[t];
      if (res->runner_up) res->runner_up[t] = hp2[t];
      if (res->cost) res->cost[t] = hc[t];
      if (res->kkt) res->kkt[t] = hr[t];
      if (res->master_iters) res->master_iters[t] = hit[t];
      if (res->col_subtiles) res->col_subtiles[t] = htl[t];
    }
  }
  for (int t = 0; t < n; ++t) {
    if (hst[t] == VMAT_ETIMEOUT) return vmat_fail(ctx, VMAT_ETIMEOUT, "iteration %d: bounded wait ran out", t);
    if (hst[t] != VMAT_OK)
      return vmat_fail(ctx, VMAT_ENOTCONV, "iteration %d: master problem did not converge (rho %.3e)", t, hr[t]);
  }
  return VMAT_OK;
}

extern "C" vmat_status vmat_dose_batch32(vmat_ctx *ctx, const float *X_dev, float *Z_dev,
                                         float *fprime_dev, double *cost_host) {
  if (!ctx || !X_dev || !Z_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  double *cdev = cost_host ? ctx->red + ctx->red_len - 32 : nullptr;
  vmat_status s = vmat_launch_dose_batch32(ctx, X_dev, Z_dev, fprime_dev, cdev);
  if (s != VMAT_OK) return s;
  if (cost_host) {
    VMAT_CUDA(ctx, cudaMemcpyAsync(cost_host, cdev, 32 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < 32; ++b) cost_host[b] += ctx->inactive_cost;
  }
  return sync_status(ctx);
}

extern "C" vmat_status vmat_price_batch32(vmat_ctx *ctx, const float *Fp_dev, const float *w_dev,
                                          float *G_dev) {
  if (!ctx || !Fp_dev || !G_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = vmat_launch_price_batch32(ctx, Fp_dev, w_dev, G_dev);
  if (s != VMAT_OK) return s;
  return sync_status(ctx);
}

extern "C" vmat_status vmat_set_profiling(vmat_ctx *ctx, int32_t on) {
  if (!ctx) return VMAT_EINVAL;
  ctx->profiling = on ? 1 : 0;
  return VMAT_OK;
}

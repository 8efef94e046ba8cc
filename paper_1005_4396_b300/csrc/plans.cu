// Many independent plans at once.
//
// Planning throughput for a clinic runs many plans; a single plan's master
// kernel leaves the GPU latency-bound (grid-wide reductions every iteration),
// and a small plan runs about as fast on a third of the SMs as on all of them.
// A batch gives every plan a CTA budget for its persistent master kernel:
// SMs / share, raised where fewer CTAs would need more than 16 voxels per
// thread.  The budgets are SM "tokens": a list schedule (largest estimated
// work first, each plan on the tokens that free up earliest) decides which
// plans run side by side, and each plan starts after the plans that held its
// tokens before it.  Whatever the actual run times, plans that overlap hold
// disjoint tokens, so their cooperative kernels are co-resident.  The whole
// run (reset + every column-generation iteration of every plan) is captured
// once into a CUDA graph with those dependencies and replayed with a single
// launch.  The share is chosen by an autotuner that times short trial runs.
#include <algorithm>
#include <string>
#include <vector>

#include "vmat_internal.cuh"

struct vmat_batch {
  std::vector<vmat_ctx *> plans;
  std::vector<cudaStream_t> orig;  // each plan's stream before the batch took it
  std::vector<cudaStream_t> plan_st;  // one capture stream per plan
  cudaStream_t user = nullptr;    // caller's stream: the batch starts after its prior work
  cudaStream_t origin = nullptr;  // the batch's own stream (capturable; the legacy stream is not)
  int share = 0;                      // configured SM share (0: not configured)
  std::vector<int> order;             // capture order (list-schedule order)
  std::vector<std::vector<int>> deps; // plans whose SM tokens each plan takes over
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int g_iters = -2, g_trial = -2;
  double g_kkt = -1.0;
  std::vector<double> g_sig;  // per-plan settings the graph was captured with
  std::vector<Records> rec;
  char *rec_block = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_start = nullptr, ev_stop = nullptr;
  std::vector<cudaEvent_t> ev_end, ev_dep;
  std::string err;
};

static vmat_status bfail(vmat_batch *b, vmat_status st, const std::string &msg) {
  b->err = msg;
  return st;
}

#define BCUDA(b, call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                    \
  } while (0)

static void drop_graph(vmat_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->g_iters = -2;
}

extern "C" const char *vmat_batch_last_error(const vmat_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" vmat_status vmat_batch_create(vmat_ctx *const *plans, int32_t n, void *cuda_stream,
                                         vmat_batch **out) {
  if (!out) return VMAT_EINVAL;
  *out = nullptr;
  if (!plans || n <= 0) return vmat_fail(nullptr, VMAT_EINVAL, "vmat_batch_create: no plans");
  for (int p = 0; p < n; ++p) {
    if (!plans[p]) return vmat_fail(nullptr, VMAT_EINVAL, "vmat_batch_create: plan %d is NULL", p);
    if (plans[p]->device != plans[0]->device)
      return vmat_fail(nullptr, VMAT_EINVAL, "vmat_batch_create: plans on different devices");
    for (int q = 0; q < p; ++q)
      if (plans[q] == plans[p]) return vmat_fail(nullptr, VMAT_EINVAL, "vmat_batch_create: plan %d repeated", p);
  }
  vmat_batch *b = new vmat_batch();
  b->plans.assign(plans, plans + n);
  for (vmat_ctx *c : b->plans) b->orig.push_back(c->stream);
  b->user = (cudaStream_t)cuda_stream;
  b->ev_end.resize(n, nullptr);
  b->ev_dep.resize(n, nullptr);
  b->plan_st.resize(n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&b->ev_fork) == cudaSuccess && cudaEventCreate(&b->ev_start) == cudaSuccess &&
            cudaEventCreate(&b->ev_stop) == cudaSuccess;
  for (int p = 0; ok && p < n; ++p)
    ok = cudaEventCreate(&b->ev_end[p]) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_dep[p], cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->plan_st[p], cudaStreamNonBlocking) == cudaSuccess;
  // device records: one block, per plan n_angles entries of each field
  size_t total = 0;
  for (vmat_ctx *c : b->plans) total += (size_t)c->N * (4 * 4 + 4 * 8) + 64;
  ok = ok && cudaMalloc((void **)&b->rec_block, total) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    vmat_batch_destroy(b);
    return vmat_fail(nullptr, VMAT_ENOMEM, "vmat_batch_create: allocation failed");
  }
  char *q = b->rec_block;
  for (vmat_ctx *c : b->plans) {
    const size_t nn = c->N;
    Records r;
    r.p = (double *)q;
    r.p2 = r.p + nn;
    r.cost = r.p2 + nn;
    r.rho = r.cost + nn;
    r.k = (int32_t *)(r.rho + nn);
    r.iters = r.k + nn;
    r.status = r.iters + nn;
    r.tiles = r.status + nn;
    b->rec.push_back(r);
    q += nn * (4 * 4 + 4 * 8) + 64;
  }
  *out = b;
  return VMAT_OK;
}

extern "C" void vmat_batch_destroy(vmat_batch *b) {
  if (!b) return;
  for (cudaStream_t s : b->plan_st)
    if (s) cudaStreamSynchronize(s);
  drop_graph(b);
  for (size_t p = 0; p < b->plans.size(); ++p) b->plans[p]->stream = b->orig[p];
  for (cudaStream_t s : b->plan_st)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_end)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_dep)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->ev_stop) cudaEventDestroy(b->ev_stop);
  if (b->rec_block) cudaFree(b->rec_block);
  if (b->origin) {
    cudaStreamSynchronize(b->origin);
    cudaStreamDestroy(b->origin);
  }
  delete b;
}

// List schedule of plans on SM tokens (host only): plans in order of
// decreasing estimated work (stable), each on the budget[p] tokens that free
// up earliest in the simulated schedule (ties: lowest token), starting after
// the last holders of those tokens, which become its dependencies.
extern "C" vmat_status vmat_list_schedule(int32_t n, const int32_t *budget, const double *est,
                                          int32_t sms, int32_t *order, int32_t *ndep,
                                          int32_t *deps, uint8_t *tokens) {
  if (n <= 0 || sms <= 0 || !budget || !est || !order || !ndep || !deps) return VMAT_EINVAL;
  for (int p = 0; p < n; ++p)
    if (budget[p] < 1 || budget[p] > sms || !(est[p] >= 0.0)) return VMAT_EINVAL;
  std::vector<int> ord(n);
  for (int p = 0; p < n; ++p) ord[p] = p;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return est[x] > est[y]; });
  std::vector<double> free_at(sms, 0.0);
  std::vector<int> holder(sms, -1), tok(sms);
  if (tokens) std::fill(tokens, tokens + (size_t)n * sms, (uint8_t)0);
  for (int i = 0; i < n; ++i) {
    const int p = ord[i];
    order[i] = p;
    for (int t = 0; t < sms; ++t) tok[t] = t;
    std::stable_sort(tok.begin(), tok.end(), [&](int x, int y) { return free_at[x] < free_at[y]; });
    double start = 0.0;
    for (int j = 0; j < budget[p]; ++j) start = std::max(start, free_at[tok[j]]);
    int nd = 0;
    for (int j = 0; j < budget[p]; ++j) {
      const int t = tok[j];
      const int h = holder[t];
      if (h >= 0 && std::find(deps + (size_t)p * n, deps + (size_t)p * n + nd, h) == deps + (size_t)p * n + nd)
        deps[(size_t)p * n + nd++] = h;
      holder[t] = p;
      free_at[t] = start + est[p];
      if (tokens) tokens[(size_t)p * sms + t] = 1;
    }
    ndep[p] = nd;
  }
  return VMAT_OK;
}

// Budgets and list schedule for an SM share: plan p gets
// b_p = max(SMs / share, CTAs for <= 16 voxels per thread at 512 threads)
// tokens; plans are placed largest estimated work (active voxels x beams per
// token) first, each on the b_p tokens that free up earliest (ties: lowest
// token), after the last holders of those tokens.
extern "C" vmat_status vmat_batch_configure(vmat_batch *b, int32_t share) {
  if (!b) return VMAT_EINVAL;
  const int n = (int)b->plans.size();
  const int sms = b->plans[0]->num_sms;
  if (share < 1 || share > sms) return bfail(b, VMAT_EINVAL, "share must be in [1, SMs]");
  for (size_t p = 0; p < b->plans.size(); ++p) BCUDA(b, cudaStreamSynchronize(b->plans[p]->stream));
  drop_graph(b);
  std::vector<int32_t> bud(n);
  std::vector<double> est(n);
  for (int p = 0; p < n; ++p) {
    vmat_ctx *c = b->plans[p];
    const int64_t need = (c->Va + 16 * 512 - 1) / (16 * 512);
    bud[p] = (int)std::min<int64_t>(sms, std::max<int64_t>(sms / share, need));
    vmat_status s = vmat_reset(c);
    if (s == VMAT_OK) s = vmat_set_master_budget(c, bud[p]);
    if (s != VMAT_OK) return bfail(b, s, std::string("plan reconfiguration: ") + c->err);
    est[p] = (double)c->Va * c->N / bud[p];
  }
  std::vector<int32_t> order(n), ndep(n), deps((size_t)n * n);
  vmat_status ls = vmat_list_schedule(n, bud.data(), est.data(), sms, order.data(), ndep.data(),
                                      deps.data(), nullptr);
  if (ls != VMAT_OK) return bfail(b, ls, "list schedule");
  b->deps.assign(n, {});
  for (int p = 0; p < n; ++p) b->deps[p].assign(deps.begin() + (size_t)p * n, deps.begin() + (size_t)p * n + ndep[p]);
  b->order.assign(order.begin(), order.end());
  for (int p = 0; p < n; ++p) b->plans[p]->stream = b->plan_st[p];
  b->share = share;
  return VMAT_OK;
}

// Capture every plan (reset + iterations) into one graph: each plan on its
// own stream, after the fork and after the plans whose tokens it takes over.
// Settings of each plan that its captured launches bake in as arguments.
static std::vector<double> plan_settings(const vmat_batch *b) {
  std::vector<double> v;
  for (const vmat_ctx *c : b->plans) {
    v.push_back(c->gamma);
    v.push_back(c->master_method);
    v.push_back(c->master_xp);
    v.push_back(c->price_smoothing);
    v.push_back(c->price_path);
  }
  return v;
}

static vmat_status build_graph(vmat_batch *b, int trial, int master_max_iters, double kkt) {
  drop_graph(b);
  cudaStream_t o = b->origin;
  BCUDA(b, cudaStreamBeginCapture(o, cudaStreamCaptureModeRelaxed));
  vmat_status st = VMAT_OK;
  cudaError_t ce = cudaEventRecord(b->ev_fork, o);
  for (size_t i = 0; i < b->order.size() && ce == cudaSuccess && st == VMAT_OK; ++i) {
    const int p = b->order[i];
    vmat_ctx *c = b->plans[p];
    ce = cudaStreamWaitEvent(c->stream, b->ev_fork, 0);
    for (size_t q = 0; q < b->deps[p].size() && ce == cudaSuccess; ++q)
      ce = cudaStreamWaitEvent(c->stream, b->ev_dep[b->deps[p][q]], 0);
    if (ce != cudaSuccess) break;
    st = vmat_enqueue_reset(c);
    const int n = trial > 0 ? std::min(trial, c->N) : c->N;
    if (st == VMAT_OK) st = vmat_enqueue_colgen(c, n, master_max_iters, kkt, b->rec[p], true);
    if (st != VMAT_OK) {
      b->err = std::string("capture of plan ") + std::to_string(p) + ": " + c->err;
      break;
    }
    ce = cudaEventRecordWithFlags(b->ev_end[p], c->stream, cudaEventRecordExternal);
    if (ce == cudaSuccess) ce = cudaEventRecord(b->ev_dep[p], c->stream);
  }
  for (size_t p = 0; p < b->plans.size() && ce == cudaSuccess && st == VMAT_OK; ++p)
    ce = cudaStreamWaitEvent(o, b->ev_dep[p], 0);  // join every plan stream
  cudaGraph_t g = nullptr;
  cudaError_t ec = cudaStreamEndCapture(o, &g);
  if (st != VMAT_OK || ce != cudaSuccess || ec != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st != VMAT_OK) return bfail(b, st, b->err);
    return bfail(b, VMAT_ECUDA, std::string("graph capture: ") +
                                    cudaGetErrorString(ce != cudaSuccess ? ce : ec));
  }
  b->graph = g;
  BCUDA(b, cudaGraphInstantiate(&b->exec, g, 0));
  b->g_iters = master_max_iters;
  b->g_kkt = kkt;
  b->g_trial = trial;
  b->g_sig = plan_settings(b);
  return VMAT_OK;
}

static vmat_status launch_graph(vmat_batch *b, double *total_ms) {
  BCUDA(b, cudaEventRecord(b->ev_fork, b->user));  // after the caller's prior work
  BCUDA(b, cudaStreamWaitEvent(b->origin, b->ev_fork, 0));
  BCUDA(b, cudaEventRecord(b->ev_start, b->origin));
  BCUDA(b, cudaGraphLaunch(b->exec, b->origin));
  BCUDA(b, cudaEventRecord(b->ev_stop, b->origin));
  BCUDA(b, cudaStreamSynchronize(b->origin));
  if (total_ms) {
    float ms = 0.f;
    BCUDA(b, cudaEventElapsedTime(&ms, b->ev_start, b->ev_stop));
    *total_ms = ms;
  }
  for (size_t p = 0; p < b->plans.size(); ++p) {
    int ds = 0;
    BCUDA(b, cudaMemcpy(&ds, b->plans[p]->dstatus, 4, cudaMemcpyDeviceToHost));
    if (ds != 0)
      return bfail(b, (vmat_status)ds, "plan " + std::to_string(p) + ": device status " + std::to_string(ds));
  }
  return VMAT_OK;
}

extern "C" vmat_status vmat_batch_tune(vmat_batch *b, int32_t trial_iters, int32_t master_max_iters,
                                       double kkt_tol, int32_t *share_out, double *ms_out) {
  if (!b || trial_iters <= 0) return b ? bfail(b, VMAT_EINVAL, "trial_iters must be > 0") : VMAT_EINVAL;
  const int cand[4] = {1, 2, 3, 4};
  int best = -1;
  double best_ms = 0.0;
  for (int q = 0; q < 4; ++q) {
    if (ms_out) ms_out[q] = -1.0;
    const int share = cand[q];
    if (share > (int)b->plans.size() || share > b->plans[0]->num_sms) continue;
    if (vmat_batch_configure(b, share) != VMAT_OK) continue;
    vmat_status s = build_graph(b, trial_iters, master_max_iters, kkt_tol);
    double ms = 0.0;
    if (s == VMAT_OK) s = launch_graph(b, nullptr);  // first replay: warm-up
    if (s == VMAT_OK) s = launch_graph(b, &ms);
    if (s != VMAT_OK) return s;
    if (ms_out) ms_out[q] = ms;
    if (best < 0 || ms < best_ms) {
      best = share;
      best_ms = ms;
    }
  }
  if (best < 0) return bfail(b, VMAT_EINVAL, "no SM share fits every plan");
  vmat_status s = vmat_batch_configure(b, best);
  if (s != VMAT_OK) return s;
  if (share_out) *share_out = best;
  return VMAT_OK;
}

extern "C" vmat_status vmat_batch_colgen_run(vmat_batch *b, int32_t master_max_iters, double kkt_tol,
                                             vmat_colgen_result *res, double *plan_ms,
                                             double *total_ms) {
  if (!b) return VMAT_EINVAL;
  if (master_max_iters < 0 || !(kkt_tol >= 0.0))
    return bfail(b, VMAT_EINVAL, "master_max_iters >= 0 and kkt_tol >= 0 required");
  if (b->share == 0) {
    vmat_status s = vmat_batch_configure(b, 1);
    if (s != VMAT_OK) return s;
  }
  if (!b->exec || b->g_iters != master_max_iters || b->g_kkt != kkt_tol || b->g_trial != 0 ||
      b->g_sig != plan_settings(b)) {
    vmat_status s = build_graph(b, 0, master_max_iters, kkt_tol);
    if (s != VMAT_OK) return s;
  }
  vmat_status s = launch_graph(b, total_ms);
  if (s != VMAT_OK) return s;
  vmat_status worst = VMAT_OK;
  for (size_t p = 0; p < b->plans.size(); ++p) {
    vmat_ctx *c = b->plans[p];
    const Records &r = b->rec[p];
    const int n = c->N, N = c->N, R = c->R;
    if (plan_ms) {
      float ms = 0.f;
      BCUDA(b, cudaEventElapsedTime(&ms, b->ev_start, b->ev_end[p]));
      plan_ms[p] = ms;
    }
    std::vector<int32_t> st(n);
    BCUDA(b, cudaMemcpy(st.data(), r.status, n * 4, cudaMemcpyDeviceToHost));
    for (int t = 0; t < n; ++t)
      if (st[t] != VMAT_OK) worst = st[t] == VMAT_ETIMEOUT ? VMAT_ETIMEOUT : (worst == VMAT_OK ? VMAT_ENOTCONV : worst);
    if (!res) continue;
    vmat_colgen_result &o = res[p];
    if (o.angle_order) BCUDA(b, cudaMemcpy(o.angle_order, r.k, n * 4, cudaMemcpyDeviceToHost));
    if (o.price) BCUDA(b, cudaMemcpy(o.price, r.p, n * 8, cudaMemcpyDeviceToHost));
    if (o.runner_up) BCUDA(b, cudaMemcpy(o.runner_up, r.p2, n * 8, cudaMemcpyDeviceToHost));
    if (o.cost) BCUDA(b, cudaMemcpy(o.cost, r.cost, n * 8, cudaMemcpyDeviceToHost));
    if (o.kkt) BCUDA(b, cudaMemcpy(o.kkt, r.rho, n * 8, cudaMemcpyDeviceToHost));
    if (o.master_iters) BCUDA(b, cudaMemcpy(o.master_iters, r.iters, n * 4, cudaMemcpyDeviceToHost));
    if (o.col_subtiles) BCUDA(b, cudaMemcpy(o.col_subtiles, r.tiles, n * 4, cudaMemcpyDeviceToHost));
    if (o.l) BCUDA(b, cudaMemcpy(o.l, c->lleaf, (size_t)N * R * 2, cudaMemcpyDeviceToHost));
    if (o.r) BCUDA(b, cudaMemcpy(o.r, c->rleaf, (size_t)N * R * 2, cudaMemcpyDeviceToHost));
    if (o.y) BCUDA(b, cudaMemcpy(o.y, c->y, (size_t)N * 8, cudaMemcpyDeviceToHost));
  }
  if (worst != VMAT_OK) return bfail(b, worst, "some master problem did not converge or timed out");
  return VMAT_OK;
}

// Master problem (Sec. 2.2): with the apertures fixed, minimise Eq. 3,
//   f(y) = sum_j F((M y)_j) + gamma * G(y),  y_k >= 0,
// over the beams that have a column, by gradient projection.  M[:, s] is the
// dose of the aperture added s-th (unit intensity), stored slot-major with
// a padded column stride Vpad.
//
// One cooperative launch runs the whole solve.  Each CTA owns a fixed slice
// of voxels; each thread keeps the dose z and the direction image w of its
// voxels in registers for the whole solve.  Per iteration:
//   pass A  reads M once: per-slot partial sums of M^T F'(z)        (HBM/L2)
//           -> grid reduce in a fixed order (deterministic)
//   every CTA then forms the same direction d = P+(y - s g) - y with the
//   second Barzilai-Borwein step s
//   pass B  reads M once: z = M y (refreshed exactly) and w = M d
//   line search: phi'(t) = sum_j w_j F'(z_j + t w_j) + gamma*(dG.d + 2t G(d))
//           is piecewise linear and nondecreasing; bracketing Newton rounds,
//           two trial points per grid reduction, on register-resident z, w.
// Stop: rho = max_k |min(y_k, g_k)| <= tol * max(rho_start, rho_ref).
// Every grid-wide wait is bounded (time and spin count); a wait that runs
// out sets VMAT_ETIMEOUT and all CTAs leave the kernel.
#include <math.h>

#include "vmat_internal.cuh"

#define LS_ROUNDS 12
#define PART_EXTRA 16  // per-CTA partial row: [N slots | 2x4 line search | cost | spare]

struct MasterArgs {
  const float *M;
  int32_t Vpad, nslots, N, cyclic, max_iters, set_rho_plan;
  const int32_t *slot_beam;
  const uint8_t *sid;
  const float *tabf;
  const double *tabd;
  const double *theta;
  double gamma, kkt_tol, rho_ref;
  double *y;            // [N] in/out
  double *rho_plan;     // [1] read (max with rho_ref) and, if set_rho_plan, written
  double *part;         // [grid][N + PART_EXTRA]
  double *gred;         // [N]
  unsigned *bar;        // [2]
  int *dstatus;
  float *z_out, *fp_out;  // [Vpad]
  MasterOut *out;
  double *rec_cost, *rec_rho;
  int32_t *rec_iters, *rec_status;
  double inactive_cost;
  unsigned long long wait_ns;
};

// ---------------------------------------------------------------- grid barrier
// Sense by generation counter.  Returns false if this or another CTA failed
// (timeout or an error raised elsewhere); the caller then leaves the kernel.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *dstatus, unsigned long long wait_ns,
                                          int *s_ok) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    volatile int *vst = dstatus;
    int ok = 1;
    unsigned g0 = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long t0 = vmat_globaltimer();
      unsigned spins = 0;
      while (*vgen == g0) {
        if (*vst != 0) { ok = 0; break; }
        if (++spins > (1u << 26) || ((spins & 63) == 0 && vmat_globaltimer() - t0 > wait_ns)) {
          atomicCAS(dstatus, 0, (int)VMAT_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (*vst != 0) ok = 0;
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV doubles per thread, fixed order; result valid in all threads.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) s_red[q * 32 + warp] = v[q];
  __syncthreads();
  if (warp == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < nw ? s_red[q * 32 + lane] : 0.0;
      s_red[q * 32 + lane] = 0.0;
      x = warp_sum(x);
      if (lane == 0) s_red[8 * 32 + q] = x;
    }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = s_red[8 * 32 + q];
  __syncthreads();
}

// Sum over CTAs of NV partials stored at part[c*stride + off + q], fixed order.
template <int NV>
__device__ __forceinline__ void grid_gather_sum(const double *part, int stride, int off,
                                                double (&v)[NV], double *s_red) {
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __ldcg(part + (size_t)c * stride + off + q);
  block_sum<NV>(v, s_red);
}

// derivative of the smoothing term G (Eq. 2) at beam k
__device__ __forceinline__ double dG_beam(const double *y, const double *theta, int N, int cyclic,
                                          int k) {
  double r = 0.0;
  if (k > 0 || cyclic) {  // pair (k-1, k)
    int km = k > 0 ? k - 1 : N - 1;
    double gap = k > 0 ? theta[k] - theta[km] : theta[0] + 360.0 - theta[N - 1];
    r += 2.0 * (y[k] - y[km]) / gap;
  }
  if (k < N - 1 || cyclic) {  // pair (k, k+1)
    int kp = k < N - 1 ? k + 1 : 0;
    double gap = k < N - 1 ? theta[kp] - theta[k] : theta[0] + 360.0 - theta[N - 1];
    r -= 2.0 * (y[kp] - y[k]) / gap;
  }
  return r;
}

struct LsPoint {
  double t, f, h;
};

// phi'(t) and phi''(t+) of the line search at two trial points, one grid
// reduction for both (partials double-buffered by round parity).
template <int VPT>
__device__ __forceinline__ bool ls_eval2(const MasterArgs &a, const float (&z)[VPT],
                                         const float (&w)[VPT], const uint8_t (&sid)[VPT],
                                         const float *s_tab, double *s_red, int *s_i,
                                         int &parity, int stride, double gdot, double Gd,
                                         double t1, double t2, LsPoint &p1, LsPoint &p2) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const float tf1 = (float)t1, tf2 = (float)t2;
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const float wq = w[q];
    const int id = sid[q];
    const float T = s_tab[id], al = s_tab[256 + id], be = s_tab[512 + id];
    const float e1 = fmaf(tf1, wq, z[q]) - T;
    const float c1 = e1 > 0.f ? be : (e1 < 0.f ? al : (wq > 0.f ? be : al));
    const float e2 = fmaf(tf2, wq, z[q]) - T;
    const float c2 = e2 > 0.f ? be : (e2 < 0.f ? al : (wq > 0.f ? be : al));
    v[0] += (double)(2.f * c1 * e1 * wq);
    v[1] += (double)(2.f * c1 * wq * wq);
    v[2] += (double)(2.f * c2 * e2 * wq);
    v[3] += (double)(2.f * c2 * wq * wq);
  }
  block_sum<4>(v, s_red);
  const int N = a.N, off = N + 4 * parity;
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) a.part[(size_t)blockIdx.x * stride + off + q] = v[q];
  if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) return false;
  grid_gather_sum<4>(a.part, stride, off, v, s_red);
  parity ^= 1;
  const double c0 = a.gamma * gdot, c1 = 2.0 * a.gamma * Gd;
  p1.t = t1; p1.f = v[0] + c0 + c1 * t1; p1.h = v[1] + c1;
  p2.t = t2; p2.f = v[2] + c0 + c1 * t2; p2.h = v[3] + c1;
  return true;
}

template <int VPT>
__global__ void __launch_bounds__(512, 1) k_master(MasterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, ns = a.nslots, tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const int stride = N + PART_EXTRA;
  constexpr int NG = VPT / 4;  // float4 groups per thread

  double *s_y = (double *)smem;   // [N] per beam
  double *s_d = s_y + N;          // [N] per beam
  double *s_g = s_d + N;          // [N] per slot
  double *s_gold = s_g + N;       // [N] per slot
  double *s_dy = s_gold + N;      // [N] per slot
  double *s_red = s_dy + N;       // [9*32]
  double *s_sc = s_red + 9 * 32;  // [16] scalars shared by the CTA
  float *s_yf = (float *)(s_sc + 16);  // [N] per slot
  float *s_df = s_yf + N;              // [N] per slot
  float *s_tab = s_df + N;             // [768]
  float *s_wp = s_tab + 768;           // [nwarp][N]
  int *s_i = (int *)(s_wp + nwarp * N);  // [8] ints: 0 ok, 1 flag, 2 beam scratch
  int *s_beam = s_i + 8;                 // [N] beam of slot

  for (int q = tid; q < 768; q += nthr) s_tab[q] = a.tabf[q];
  for (int k = tid; k < N; k += nthr) {
    s_y[k] = a.y[k];
    s_d[k] = 0.0;
  }
  for (int s = tid; s < ns; s += nthr) {
    s_beam[s] = a.slot_beam[s];
    s_dy[s] = 0.0;
    s_gold[s] = 0.0;
  }
  __syncthreads();
  for (int s = tid; s < ns; s += nthr) s_yf[s] = (float)s_y[s_beam[s]];

  // own voxels: float4 group m covers voxels base + 4*(tid + nthr*m) .. +3
  const size_t base = (size_t)blockIdx.x * nthr * VPT;
  uint8_t my_sid[VPT];
#pragma unroll
  for (int m = 0; m < NG; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) my_sid[4 * m + q] = a.sid[base + 4 * (tid + nthr * m) + q];
  float z[VPT], w[VPT];
  __syncthreads();

  // z = M y
#pragma unroll
  for (int v = 0; v < VPT; ++v) z[v] = 0.f;
  for (int s = 0; s < ns; ++s) {
    const float4 *Ms = (const float4 *)(a.M + (size_t)s * a.Vpad + base);
    const float ys = s_yf[s];
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      float4 q = __ldg(Ms + tid + nthr * m);
      z[4 * m] = fmaf(q.x, ys, z[4 * m]);
      z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]);
      z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]);
      z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]);
    }
  }

  int it = 0, status = VMAT_ENOTCONV;
  double rho = 0.0, rho0 = 0.0, tol = 0.0;
  bool alive = true;
  int ls_parity = 0;

  for (;;) {
    // ---------------- pass A: per-slot partials of M^T F'(z)
    float fp[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      int q = my_sid[v];
      fp[v] = vmat_dF(z[v], s_tab[q], s_tab[256 + q], s_tab[512 + q]);
    }
    for (int s0 = 0; s0 < ns; s0 += 4) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (s0 + u < ns) {
          const float4 *Ms = (const float4 *)(a.M + (size_t)(s0 + u) * a.Vpad + base);
#pragma unroll
          for (int m = 0; m < NG; ++m) {
            float4 q = __ldg(Ms + tid + nthr * m);
            acc[u] = fmaf(q.x, fp[4 * m], acc[u]);
            acc[u] = fmaf(q.y, fp[4 * m + 1], acc[u]);
            acc[u] = fmaf(q.z, fp[4 * m + 2], acc[u]);
            acc[u] = fmaf(q.w, fp[4 * m + 3], acc[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = warp_sumf(acc[u]);
      if (lane == 0)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (s0 + u < ns) s_wp[warp * N + s0 + u] = acc[u];
    }
    __syncthreads();
    for (int s = tid; s < ns; s += nthr) {
      double sum = 0.0;
      for (int q = 0; q < nwarp; ++q) sum += (double)s_wp[q * N + s];
      a.part[(size_t)blockIdx.x * stride + s] = sum;
    }
    if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }
    // distributed fixed-order reduction: CTA b owns slots b, b+G, ...
    for (int s = blockIdx.x; s < ns; s += gridDim.x) {
      double v[1];
      grid_gather_sum<1>(a.part, stride, s, v, s_red);
      if (tid == 0) a.gred[s] = v[0];
    }
    if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }

    // ---------------- gradient, residual, direction (same in every CTA)
    for (int s = tid; s < ns; s += nthr) {
      int k = s_beam[s];
      s_g[s] = __ldcg(a.gred + s) + a.gamma * dG_beam(s_y, a.theta, N, a.cyclic, k);
    }
    __syncthreads();
    if (warp == 0) {
      double r = 0.0, ym = 0.0, gm = 0.0, dyg = 0.0, dgg = 0.0;
      for (int s = lane; s < ns; s += 32) {
        double yk = s_y[s_beam[s]], gk = s_g[s];
        r = fmax(r, fabs(fmin(yk, gk)));
        ym = fmax(ym, fabs(yk));
        gm = fmax(gm, fabs(gk));
        double dg = gk - s_gold[s];
        dyg += s_dy[s] * dg;
        dgg += dg * dg;
      }
      r = warp_max(r);
      ym = warp_max(ym);
      gm = warp_max(gm);
      dyg = warp_sum(dyg);
      dgg = warp_sum(dgg);
      if (lane == 0) {
        s_sc[0] = r;
        double step;
        if (it == 0) step = fmax(ym, 1.0) / fmax(gm, 1e-300);
        else step = (dyg > 0.0 && dgg > 0.0) ? dyg / dgg : 1e12;
        s_sc[1] = fmin(fmax(step, 1e-12), 1e12);
      }
    }
    __syncthreads();
    rho = s_sc[0];
    if (it == 0) {
      rho0 = rho;
      double ref = fmax(a.rho_ref, a.rho_plan ? *a.rho_plan : 0.0);
      tol = a.kkt_tol * fmax(fmax(rho0, ref), 1e-300);
    }
    if (rho <= tol) { status = VMAT_OK; break; }
    if (it >= a.max_iters) { status = VMAT_ENOTCONV; break; }
    const double step = s_sc[1];
    for (int s = tid; s < ns; s += nthr) {
      int k = s_beam[s];
      double yk = s_y[k];
      double p = yk - step * s_g[s];
      double dk = (p > 0.0 ? p : 0.0) - yk;
      s_d[k] = dk;
      s_df[s] = (float)dk;
      s_gold[s] = s_g[s];
    }
    __syncthreads();
    // gdot = dG(y).d over beams with a column; Gd = G(d) over all pairs
    if (warp == 0) {
      double gd = 0.0, Gd = 0.0;
      for (int s = lane; s < ns; s += 32) {
        int k = s_beam[s];
        gd += dG_beam(s_y, a.theta, N, a.cyclic, k) * s_d[k];
      }
      int npair = a.cyclic ? N : N - 1;
      for (int k = lane; k < npair; k += 32) {
        int kp = k + 1 < N ? k + 1 : 0;
        double gap = k + 1 < N ? a.theta[kp] - a.theta[k] : a.theta[0] + 360.0 - a.theta[N - 1];
        double dd = s_d[kp] - s_d[k];
        Gd += dd * dd / gap;
      }
      gd = warp_sum(gd);
      Gd = warp_sum(Gd);
      if (lane == 0) { s_sc[2] = gd; s_sc[3] = Gd; }
    }
    __syncthreads();
    const double gdot = s_sc[2], Gd = s_sc[3];

    // ---------------- pass B: z = M y, w = M d
#pragma unroll
    for (int v = 0; v < VPT; ++v) { z[v] = 0.f; w[v] = 0.f; }
    for (int s = 0; s < ns; ++s) {
      const float4 *Ms = (const float4 *)(a.M + (size_t)s * a.Vpad + base);
      const float ys = s_yf[s], ds = s_df[s];
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        float4 q = __ldg(Ms + tid + nthr * m);
        z[4 * m] = fmaf(q.x, ys, z[4 * m]);       w[4 * m] = fmaf(q.x, ds, w[4 * m]);
        z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]); w[4 * m + 1] = fmaf(q.y, ds, w[4 * m + 1]);
        z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]); w[4 * m + 2] = fmaf(q.z, ds, w[4 * m + 2]);
        z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]); w[4 * m + 3] = fmaf(q.w, ds, w[4 * m + 3]);
      }
    }

    // ---------------- exact line search on [0, 1]
    LsPoint p0, p1;
    if (!ls_eval2<VPT>(a, z, w, my_sid, s_tab, s_red, s_i, ls_parity, stride, gdot, Gd, 0.0, 1.0,
                       p0, p1)) { alive = false; break; }
    double t;
    if (!(p0.f < 0.0)) {
      t = 0.0;  // not a descent direction: stalled
    } else if (p1.f <= 0.0) {
      t = 1.0;
    } else {
      LsPoint lo = p0, hi = p1;
      t = -1.0;
      for (int r = 0; r < LS_ROUNDS; ++r) {
        const double width = hi.t - lo.t;
        const double tS = lo.t - lo.f * width / (hi.f - lo.f);
        double tA = lo.h > 0.0 ? lo.t - lo.f / lo.h : tS;
        double tB = hi.h > 0.0 ? hi.t - hi.f / hi.h : tS;
        // both ends on one linear piece of phi': the secant root is exact
        if ((fabs(tA - tB) <= 1e-9 * tS && fabs(tA - tS) <= 1e-9 * tS) || width <= 1e-9 * hi.t) {
          t = tS;
          break;
        }
        if (!(tA > lo.t && tA < hi.t)) tA = tS;
        if (!(tB > lo.t && tB < hi.t)) tB = 0.5 * (lo.t + hi.t);
        if (fabs(tA - tB) <= 1e-12 * tA) tB = 0.5 * (lo.t + tA);
        LsPoint qA, qB;
        if (!ls_eval2<VPT>(a, z, w, my_sid, s_tab, s_red, s_i, ls_parity, stride, gdot, Gd, tA, tB,
                           qA, qB)) { alive = false; break; }
        if (qA.f == 0.0) { t = qA.t; break; }
        if (qB.f == 0.0) { t = qB.t; break; }
        if (qA.f < 0.0 && qA.t > lo.t) lo = qA;
        if (qA.f > 0.0 && qA.t < hi.t) hi = qA;
        if (qB.f < 0.0 && qB.t > lo.t) lo = qB;
        if (qB.f > 0.0 && qB.t < hi.t) hi = qB;
      }
      if (!alive) break;
      if (t < 0.0) t = lo.t - lo.f * (hi.t - lo.t) / (hi.f - lo.f);
      t = fmin(fmax(t, lo.t), hi.t);
    }
    if (t <= 0.0) { status = VMAT_ENOTCONV; break; }

    // ---------------- update
    for (int s = tid; s < ns; s += nthr) {
      int k = s_beam[s];
      double dk = s_d[k];
      s_dy[s] = t * dk;
    }
    __syncthreads();
    for (int s = tid; s < ns; s += nthr) {
      int k = s_beam[s];
      s_y[k] += s_dy[s];
      s_yf[s] = (float)s_y[k];
    }
    const float tf = (float)t;
#pragma unroll
    for (int v = 0; v < VPT; ++v) z[v] = fmaf(tf, w[v], z[v]);
    ++it;
    __syncthreads();
  }

  if (!alive) {
    if (blockIdx.x == 0 && tid == 0) {
      a.out->status = VMAT_ETIMEOUT;
      if (a.rec_status) *a.rec_status = VMAT_ETIMEOUT;
    }
    return;
  }

  // ---------------- final dose, derivative and cost at the solution
  __syncthreads();
#pragma unroll
  for (int v = 0; v < VPT; ++v) z[v] = 0.f;
  for (int s = 0; s < ns; ++s) {
    const float4 *Ms = (const float4 *)(a.M + (size_t)s * a.Vpad + base);
    const float ys = s_yf[s];
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      float4 q = __ldg(Ms + tid + nthr * m);
      z[4 * m] = fmaf(q.x, ys, z[4 * m]);
      z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]);
      z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]);
      z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]);
    }
  }
  double cst[1] = {0.0};
#pragma unroll
  for (int m = 0; m < NG; ++m) {
    float zo[4], fo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int v = 4 * m + q;
      int id = my_sid[v];
      fo[q] = vmat_dF(z[v], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      zo[q] = z[v];
      cst[0] += vmat_F((double)z[v], a.tabd[id], a.tabd[256 + id], a.tabd[512 + id]);
    }
    size_t off = base + 4 * (tid + (size_t)nthr * m);
    *(float4 *)(a.z_out + off) = make_float4(zo[0], zo[1], zo[2], zo[3]);
    *(float4 *)(a.fp_out + off) = make_float4(fo[0], fo[1], fo[2], fo[3]);
  }
  block_sum<1>(cst, s_red);
  if (tid == 0) a.part[(size_t)blockIdx.x * stride + N + 8] = cst[0];
  if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) {
    if (blockIdx.x == 0 && tid == 0) a.out->status = VMAT_ETIMEOUT;
    return;
  }
  if (blockIdx.x == 0) {
    double v[1];
    grid_gather_sum<1>(a.part, stride, N + 8, v, s_red);
    if (tid == 0) {
      double G = 0.0;
      int npair = a.cyclic ? N : N - 1;
      for (int k = 0; k < npair; ++k) {
        int kp = k + 1 < N ? k + 1 : 0;
        double gap = k + 1 < N ? a.theta[kp] - a.theta[k] : a.theta[0] + 360.0 - a.theta[N - 1];
        double dd = s_y[kp] - s_y[k];
        G += dd * dd / gap;
      }
      a.out->cost_active = v[0];
      a.out->smooth = G;
      a.out->rho = rho;
      a.out->rho0 = rho0;
      a.out->iters = it;
      a.out->status = status;
      if (a.set_rho_plan && a.rho_plan) *a.rho_plan = rho0;
      if (a.rec_cost) *a.rec_cost = v[0] + a.inactive_cost + a.gamma * G;
      if (a.rec_rho) *a.rec_rho = rho;
      if (a.rec_iters) *a.rec_iters = it;
      if (a.rec_status) *a.rec_status = status;
    }
    for (int k = tid; k < N; k += nthr) a.y[k] = s_y[k];
  }
}

// ---------------------------------------------------------------- launch
static size_t master_smem_bytes(int N, int nthr) {
  int nwarp = nthr / 32;
  return (size_t)(5 * N + 9 * 32 + 16) * 8 + (size_t)(2 * N + 768 + nwarp * N) * 4 +
         (size_t)(8 + N) * 4 + 16;
}

template <int VPT>
static cudaError_t master_occupancy(int nthr, size_t smem, int *nb) {
  cudaError_t e = cudaFuncSetAttribute(k_master<VPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_master<VPT>, nthr, smem);
}

vmat_status vmat_configure_master(vmat_ctx *ctx) {
  const int64_t Va = ctx->Va > 0 ? ctx->Va : 1;
  int vpt = 4, nthr = 0;
  for (vpt = 4; vpt <= 32; vpt *= 2) {
    int64_t threads = (Va + vpt - 1) / vpt;
    int64_t per_sm = (threads + ctx->num_sms - 1) / ctx->num_sms;
    nthr = (int)(((per_sm + 31) / 32) * 32);
    if (nthr < 64) nthr = 64;
    if (nthr <= 512) break;
  }
  if (vpt > 32) return vmat_fail(ctx, VMAT_EINVAL, "too many active voxels for the master kernel");
  int64_t chunk = (int64_t)nthr * vpt;
  int grid = (int)((Va + chunk - 1) / chunk);
  size_t smem = master_smem_bytes(ctx->N, nthr);
  int nb = 0;
  cudaError_t e = vpt == 4    ? master_occupancy<4>(nthr, smem, &nb)
                  : vpt == 8  ? master_occupancy<8>(nthr, smem, &nb)
                  : vpt == 16 ? master_occupancy<16>(nthr, smem, &nb)
                              : master_occupancy<32>(nthr, smem, &nb);
  if (e != cudaSuccess) return vmat_cuda_fail(ctx, e, "master occupancy");
  if (nb < 1 || grid > nb * ctx->num_sms)
    return vmat_fail(ctx, VMAT_EINVAL, "master kernel cannot be co-resident (%d blocks/SM)", nb);
  ctx->master_vpt = vpt;
  ctx->master_block = nthr;
  ctx->master_grid = grid;
  ctx->master_smem = smem;
  ctx->Vpad = (int32_t)(grid * chunk);
  return VMAT_OK;
}

vmat_status vmat_launch_master(vmat_ctx *ctx, int max_iters, double kkt_tol, double rho_ref,
                               int set_rho_plan, double *rec_cost, double *rec_rho,
                               int32_t *rec_iters, int32_t *rec_status) {
  MasterArgs a;
  a.M = ctx->M;
  a.Vpad = ctx->Vpad;
  a.nslots = ctx->n_slots;
  a.N = ctx->N;
  a.cyclic = ctx->cyclic;
  a.max_iters = max_iters;
  a.set_rho_plan = set_rho_plan;
  a.slot_beam = ctx->slot_beam;
  a.sid = ctx->sid;
  a.tabf = ctx->tabf;
  a.tabd = ctx->tabd;
  a.theta = ctx->theta;
  a.gamma = ctx->gamma;
  a.kkt_tol = kkt_tol;
  a.rho_ref = rho_ref;
  a.y = ctx->y;
  a.rho_plan = ctx->rho_plan;
  a.part = ctx->red;
  a.gred = ctx->red + (size_t)ctx->master_grid * (ctx->N + PART_EXTRA);
  a.bar = ctx->bar;
  a.dstatus = ctx->dstatus;
  a.z_out = ctx->zact;
  a.fp_out = ctx->fpact;
  a.out = ctx->mout;
  a.rec_cost = rec_cost;
  a.rec_rho = rec_rho;
  a.rec_iters = rec_iters;
  a.rec_status = rec_status;
  a.inactive_cost = ctx->inactive_cost;
  a.wait_ns = 2000000000ull;  // 2 s per grid-wide wait
  if ((int64_t)ctx->master_grid * (ctx->N + PART_EXTRA) + ctx->N > ctx->red_len)
    return vmat_fail(ctx, VMAT_EINVAL, "reduction scratch too small");
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 4, ctx->stream));
  void *args[] = {&a};
  dim3 grid(ctx->master_grid), block(ctx->master_block);
  const void *fn = ctx->master_vpt == 4    ? (const void *)k_master<4>
                   : ctx->master_vpt == 8  ? (const void *)k_master<8>
                   : ctx->master_vpt == 16 ? (const void *)k_master<16>
                                           : (const void *)k_master<32>;
  // the dynamic shared-memory limit is a per-kernel, process-wide attribute:
  // set it for this context's launch (another context may have lowered it)
  VMAT_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ctx->master_smem));
  VMAT_CUDA(ctx, cudaLaunchCooperativeKernel(fn, grid, block, args, ctx->master_smem, ctx->stream));
  ctx->n_launches += 1;
  return VMAT_OK;
}

// ---------------------------------------------------------------- bounded-wait self-test
__global__ void k_grid_wait_probe(unsigned *bar, int *dstatus, unsigned long long wait_ns,
                                  int skip_one) {
  __shared__ int s_ok;
  if (skip_one && blockIdx.x == gridDim.x - 1) return;  // this CTA never arrives
  grid_sync(bar, dstatus, wait_ns, &s_ok);
}

extern "C" vmat_status vmat_selftest_grid_wait(vmat_ctx *ctx, int32_t skip_one, double wait_seconds) {
  if (!ctx) return VMAT_EINVAL;
  if (!(wait_seconds > 0.0 && wait_seconds <= 5.0))
    return vmat_fail(ctx, VMAT_EINVAL, "wait_seconds must be in (0, 5]");
  cudaStream_t st = ctx->stream;
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 8, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->dstatus, 0, 4, st));
  unsigned long long wait_ns = (unsigned long long)(wait_seconds * 1e9);
  int skip = skip_one ? 1 : 0;
  void *args[] = {&ctx->bar, &ctx->dstatus, &wait_ns, &skip};
  int grid = ctx->num_sms < 8 ? ctx->num_sms : 8;
  VMAT_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_grid_wait_probe, dim3(grid), dim3(32),
                                             args, 0, st));
  ctx->n_launches += 1;
  int ds = 0;
  VMAT_CUDA(ctx, cudaMemcpyAsync(&ds, ctx->dstatus, 4, cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  // leave the context usable
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 8, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->dstatus, 0, 4, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  if (ds == VMAT_ETIMEOUT) return vmat_fail(ctx, VMAT_ETIMEOUT, "grid wait ran out (as designed)");
  if (ds != 0) return vmat_fail(ctx, (vmat_status)ds, "grid wait: status %d", ds);
  return VMAT_OK;
}

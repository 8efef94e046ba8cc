// Master problem (Sec. 2.2): with the apertures fixed, minimise Eq. 3,
//   f(y) = sum_j F((M y)_j) + gamma * G(y),  y_k >= 0,
// over the beams that have a column, by gradient projection.  M[:, s] is the
// dose of the aperture added s-th (unit intensity), stored slot-major with
// a padded column stride Vpad.
//
// One cooperative launch runs the whole solve.  The padded voxels are cut
// into subtiles of ST = 4*threads voxels; CTA b owns the VPT/4 subtiles
// b, b+G, b+2G, ... (spread over the volume, so dense and sparse regions
// mix in every CTA) and thread t holds voxels 4t..4t+3 of each in registers
// (dose z, direction image w) for the whole solve.  A column is nonzero
// only near its aperture's beam path: per (column, subtile) flags let every
// pass skip all-zero subtiles.  Per iteration:
//   pass A   gradient M^T F'(z): F' of the CTA's subtiles goes to shared
//            memory; each warp streams whole (column, subtile) pairs with
//            many independent 16-byte loads per lane
//   reduce   per-slot CTA partials -> grid barrier -> warp-per-slot fixed-order
//            sums over CTAs -> grid barrier (deterministic, no float atomics)
//   step     every CTA forms the same d = P+(y - s g) - y (second
//            Barzilai-Borwein step s) from the same reduced gradient
//   pass B   z = M y (refreshed exactly) and w = M d, thread per voxel
//   search   phi'(t) = sum_j w_j F'(z_j + t w_j) + gamma*(dG(y).d + 2t G(d))
//            is piecewise linear and nondecreasing: each round evaluates it
//            at 16 points (FP32 per voxel, FP64 across warps and CTAs), one
//            grid reduction per round; stop once Newton steps from both ends
//            of the bracket agree (same linear piece: the secant is exact).
// Stop: rho = max_k |min(y_k, g_k)| <= tol * max(rho_start, rho_ref).
// The grid barrier is one counter whose top bit flips when every CTA has
// arrived; each wait is bounded in time and spins, after which the kernel
// records VMAT_ETIMEOUT and every CTA leaves.
#include <math.h>

#include "vmat_internal.cuh"

#define LS_POINTS 16
#define LS_ROUNDS 4
// per-CTA partial row: [N slots | 2 x 32 line-search values | cost | spare]
#define PART_EXTRA 72
#define LS_OFF(N, parity) ((N) + 32 * (parity))
#define COST_OFF(N) ((N) + 64)

struct MasterArgs {
  const float *M;
  const int32_t *tflag;  // [N][G*VPT/4] nonzero flags of the column subtiles
  int32_t Vpad, nslots, N, cyclic, max_iters, set_rho_plan;
  const int32_t *slot_beam;
  const uint8_t *sid;
  const float *tabf;
  const double *tabd;
  const double *theta;
  double gamma, kkt_tol, rho_ref;
  double *y;             // [N] in/out
  double *rho_plan;      // [1] read (max with rho_ref) and, if set_rho_plan, written
  double *part;          // [grid][N + PART_EXTRA]
  double *gred;          // [N]
  unsigned *bar;         // [1] grid barrier word
  int *dstatus;
  float *z_out, *fp_out;  // [Vpad]
  MasterOut *out;
  double *stats;         // [8] cumulative: ns in pass A+reduce, step, pass B, search; syncs; iters
  double *rec_cost, *rec_rho;
  int32_t *rec_iters, *rec_status;
  double inactive_cost;
  unsigned long long wait_ns;
};

// ---------------------------------------------------------------- grid barrier
// Every CTA adds 1 to the barrier word except CTA 0, which adds
// 0x80000000 - (G-1): the sum over a barrier is 0x80000000, so the top bit
// flips exactly when all have arrived and the low bits return to their
// previous value (no reset).  Returns false if a wait ran out or another CTA
// reported an error; the caller then leaves the kernel.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *dstatus, unsigned long long wait_ns,
                                          int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    unsigned old, cur;
    int ok = 1;
    __threadfence();  // the CTA's partials (ordered by the bar.sync above) before arriving
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(inc)
                 : "memory");
    const unsigned long long t0 = vmat_globaltimer();
    unsigned spins = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if ((old ^ cur) & 0x80000000u) break;
      if ((++spins & 63) == 0) {
        if (*(volatile int *)dstatus != 0) { ok = 0; break; }
        if (spins > (1u << 26) || vmat_globaltimer() - t0 > wait_ns) {
          atomicCAS(dstatus, 0, (int)VMAT_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    if (ok && *(volatile int *)dstatus != 0) ok = 0;
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

// Warp transpose-reduction: v[32] per lane in, lane l returns the warp sum of
// v[l] (31 shuffles for 32 sums).
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) {
    const bool upper = (lane & k) != 0;
#pragma unroll
    for (int i = 0; i < k; ++i) {
      const float send = upper ? v[i] : v[i + k];
      const float keep = upper ? v[i + k] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, k);
    }
  }
  return v[0];
}

// derivative of the smoothing term G (Eq. 2) at beam k, from inverse gaps
__device__ __forceinline__ double dG_inv(const double *y, const double *igl, const double *igr,
                                         int N, int k) {
  const int km = k > 0 ? k - 1 : N - 1, kp = k < N - 1 ? k + 1 : 0;
  return 2.0 * (y[k] - y[km]) * igl[k] - 2.0 * (y[kp] - y[k]) * igr[k];
}

// G(u) (Eq. 2) over all pairs from inverse gaps, by one warp; valid in every lane
__device__ __forceinline__ double G_inv(const double *u, const double *igr, int N) {
  const int lane = threadIdx.x & 31;
  double g = 0.0;
  for (int k = lane; k < N; k += 32) {
    const int kp = k < N - 1 ? k + 1 : 0;
    const double dd = u[kp] - u[k];
    g += dd * dd * igr[k];  // igr[N-1] is 0 on a path
  }
  return warp_sum(g);
}

// One line-search round at LS_POINTS trial points t.  Per voxel the round
// evaluates the increment of its phi' term over t = 0,
//   D_j(t) = 2 w_j [ (c_j(t) - c_j(0)) e_j + c_j(t) t w_j ],  e_j = z_j - T_j,
// (c = alpha below the threshold, beta above), which is O(t w_j^2) and free
// of the cancellation that phi' itself suffers near convergence, and the
// phi'' term 2 c_j(t) w_j^2.  Along the direction a voxel changes side at
// most once, at t_j = -e_j / w_j, and only if e_j and w_j have opposite
// signs; before it D_j(t) = 2 c_j(0) w_j^2 t, after it the term
// k_j (e_j + t w_j), k_j = 2 w_j (c_side - c_j(0)), is added.  So a voxel
// whose change lies before every trial point (or nowhere) adds a linear
// function of t, kept in three per-thread sums, and only voxels that change
// side between the first and last trial point are evaluated point by point.
// FP32 per voxel, FP32 within a warp, FP64 across warps and CTAs in a fixed
// order.  Out: s_res[0..15] = sum_j D_j(t_p), s_res[16..31] = sum_j
// 2 c_j(t_p) w_j^2.
template <int VPT>
__device__ __forceinline__ bool ls_round(const MasterArgs &a, const float (&z)[VPT],
                                         const float (&w)[VPT], const uint8_t (&sid)[VPT],
                                         const float *s_tab, const float *s_t, float *s_ls,
                                         double *s_res, int *s_ok, int parity, int stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  float t_first = s_t[0], t_last = s_t[0];
#pragma unroll
  for (int p = 1; p < LS_POINTS; ++p) {
    t_first = fminf(t_first, s_t[p]);
    t_last = fmaxf(t_last, s_t[p]);
  }
  float v[32];
#pragma unroll
  for (int p = 0; p < 32; ++p) v[p] = 0.f;
  float lin = 0.f;    // sum 2 c_j(0) w_j^2 over the thread's voxels
  float jump = 0.f;   // sum 2 w_j^2 (c_side - c_j(0)) over changes before t_first
  float at_first = 0.f;  // sum k_j (e_j + t_first w_j) over the same voxels
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const float wq = w[q];
    if (wq == 0.f) continue;
    const int id = sid[q];
    const float T = s_tab[id], al = s_tab[256 + id], be = s_tab[512 + id];
    const float e0 = z[q] - T;
    const float cw = wq > 0.f ? be : al;  // side taken at the threshold itself
    const float c0 = e0 > 0.f ? be : (e0 < 0.f ? al : cw);
    lin = fmaf(2.f * c0 * wq, wq, lin);
    const float dc = cw - c0;  // nonzero only if the voxel can change side
    if (dc == 0.f) continue;
    const float k = 2.f * wq * dc, dh = k * wq;
    const float e_first = fmaf(t_first, wq, e0);
    if (e_first * wq > 0.f) {  // changed side before every trial point
      jump += dh;
      at_first = fmaf(k, e_first, at_first);
      continue;
    }
    if (!(fmaf(t_last, wq, e0) * wq > 0.f)) continue;  // after every trial point
#pragma unroll
    for (int p = 0; p < LS_POINTS; ++p) {
      const float e = fmaf(s_t[p], wq, e0);
      if (e * wq > 0.f) {
        v[p] = fmaf(k, e, v[p]);
        v[LS_POINTS + p] += dh;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < LS_POINTS; ++p) {
    const float tp = s_t[p];
    v[p] += fmaf(lin, tp, fmaf(jump, tp - t_first, at_first));
    v[LS_POINTS + p] += lin + jump;
  }
  const float ws = warp_transpose_sum32(v);
  s_ls[warp * 32 + lane] = ws;
  __syncthreads();
  const int off = LS_OFF(a.N, parity);
  if (warp == 0) {
    double acc = 0.0;
    for (int q = 0; q < nwarp; ++q) acc += (double)s_ls[q * 32 + lane];
    a.part[(size_t)blockIdx.x * stride + off + lane] = acc;
  }
  if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_ok)) return false;
  // sum the CTAs' partials: thread (warp, lane) takes CTAs warp, warp + W, ...
  double acc = 0.0;
  for (int c = warp; c < (int)gridDim.x; c += nwarp)
    acc += __ldcg(a.part + (size_t)c * stride + off + lane);
  double *s_tmp = s_res + 32;  // [nwarp][32]
  s_tmp[warp * 32 + lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double r = 0.0;
    for (int q = 0; q < nwarp; ++q) r += s_tmp[q * 32 + lane];
    s_res[lane] = r;
  }
  __syncthreads();
  return true;
}

template <int VPT>
__global__ void __launch_bounds__(512, 1) k_master(MasterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, ns = a.nslots, tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const int stride = N + PART_EXTRA;
  constexpr int NG = VPT / 4;       // float4 groups per thread
  const int ST = nthr * 4;          // voxels per subtile
  const int G = gridDim.x, NS = G * NG;
  const int lane4 = ST / 128;       // float4s per lane when a warp streams a subtile
#define SUB_OFF(m) ((size_t)(blockIdx.x + G * (m)) * ST)

  double *s_y = (double *)smem;      // [N] per beam
  double *s_d = s_y + N;             // [N] per beam
  double *s_g = s_d + N;             // [N] per slot
  double *s_gold = s_g + N;          // [N] per slot
  double *s_dy = s_gold + N;         // [N] per slot
  double *s_igl = s_dy + N;          // [N] 1/gap to the left neighbour (0: none)
  double *s_igr = s_igl + N;         // [N] 1/gap to the right neighbour (0: none)
  double *s_dgy = s_igr + N;         // [N] per slot: dG(y) at the slot's beam
  double *s_sc = s_dgy + N;          // [32] CTA-wide scalars
  double *s_res = s_sc + 32;         // [32 + 16*32] line-search sums and scratch
  float *s_yf = (float *)(s_res + 32 + 16 * 32);  // [N] per slot
  float *s_df = s_yf + N;                         // [N] per slot
  float *s_tab = s_df + N;                        // [768]
  float *s_t = s_tab + 768;                       // [LS_POINTS] trial points
  float *s_ls = s_t + LS_POINTS;                  // [16][32] warp partials
  float *s_fp = s_ls + 16 * 32;                   // [NG][ST] F' of the CTA's subtiles
  float *s_pp = s_fp + NG * ST;                   // [N*NG] warp partial per (slot, subtile) pair
  int *s_i = (int *)(s_pp + N * NG);              // [8]: 1 nonzero slots, 2 nonzero pairs
  int *s_beam = s_i + 8;                          // [N] beam of slot
  int *s_nz = s_beam + N;                         // [N] slots with a nonzero subtile here
  int *s_mask = s_nz + N;                         // [N] per slot: bit m = subtile m nonzero
  int *s_pst = s_mask + N;                        // [N+1] first pair of each slot
  int *s_pair = s_pst + N + 1;                    // [N*NG] pairs s*8+m in slot order

  for (int q = tid; q < 768; q += nthr) s_tab[q] = a.tabf[q];
  for (int k = tid; k < N; k += nthr) {
    s_y[k] = a.y[k];
    s_d[k] = 0.0;
    const bool hl = k > 0 || a.cyclic, hr = k < N - 1 || a.cyclic;
    s_igl[k] = hl ? 1.0 / (k > 0 ? a.theta[k] - a.theta[k - 1] : a.theta[0] + 360.0 - a.theta[N - 1])
                  : 0.0;
    s_igr[k] = hr ? 1.0 / (k < N - 1 ? a.theta[k + 1] - a.theta[k] : a.theta[0] + 360.0 - a.theta[N - 1])
                  : 0.0;
  }
  for (int s = tid; s < ns; s += nthr) {
    s_beam[s] = a.slot_beam[s];
    s_dy[s] = 0.0;
    s_gold[s] = 0.0;
  }
  for (int s = tid; s < ns; s += nthr) {
    int mk = 0;
    for (int m = 0; m < NG; ++m)
      if (a.tflag[(size_t)s * NS + blockIdx.x + G * m]) mk |= 1 << m;
    s_mask[s] = mk;
  }
  __syncthreads();
  if (tid == 0) {  // nonzero columns and (column, subtile) pairs, in slot order
    int n = 0, np = 0;
    for (int s = 0; s < ns; ++s) {
      const int mk = s_mask[s];
      s_pst[s] = np;
      if (mk) s_nz[n++] = s;
      for (int m = 0; m < NG; ++m)
        if (mk >> m & 1) s_pair[np++] = s * 8 + m;
    }
    s_pst[ns] = np;
    s_i[1] = n;
    s_i[2] = np;
  }
  __syncthreads();
  for (int s = tid; s < ns; s += nthr) s_yf[s] = (float)s_y[s_beam[s]];
  const int nnzs = s_i[1], npairs = s_i[2];

  uint8_t my_sid[VPT];
#pragma unroll
  for (int m = 0; m < NG; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) my_sid[4 * m + q] = a.sid[SUB_OFF(m) + 4 * tid + q];
  float z[VPT], w[VPT];
  __syncthreads();

  // z = M y
#pragma unroll
  for (int v = 0; v < VPT; ++v) z[v] = 0.f;
#pragma unroll 4
  for (int q = 0; q < nnzs; ++q) {
    const int s = s_nz[q], mk = s_mask[s];
    const float *Ms = a.M + (size_t)s * a.Vpad;
    const float ys = s_yf[s];
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      if (!(mk >> m & 1)) continue;
      const float4 q = __ldg((const float4 *)(Ms + SUB_OFF(m)) + tid);
      z[4 * m] = fmaf(q.x, ys, z[4 * m]);
      z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]);
      z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]);
      z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]);
    }
  }

  int it = 0, status = VMAT_ENOTCONV, nsync = 0;
  double rho = 0.0, rho0 = 0.0, tol = 0.0;
  bool alive = true;
  int ls_parity = 0;
  unsigned long long tA = 0, tS = 0, tB = 0, tL = 0, c0 = 0;
  const bool timer = blockIdx.x == 0 && tid == 0;

  for (;;) {
    if (timer) c0 = vmat_globaltimer();
    // ---------------- pass A: per-slot CTA partials of M^T F'(z)
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      float4 f;
      int id = my_sid[4 * m];
      f.x = vmat_dF(z[4 * m], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      id = my_sid[4 * m + 1];
      f.y = vmat_dF(z[4 * m + 1], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      id = my_sid[4 * m + 2];
      f.z = vmat_dF(z[4 * m + 2], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      id = my_sid[4 * m + 3];
      f.w = vmat_dF(z[4 * m + 3], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      *(float4 *)(s_fp + m * ST + 4 * tid) = f;
    }
    __syncthreads();
    for (int q = warp; q < npairs; q += nwarp) {
      const int s = s_pair[q] >> 3, m = s_pair[q] & 7;
      const float4 *Ms = (const float4 *)(a.M + (size_t)s * a.Vpad + SUB_OFF(m));
      const float4 *F4 = (const float4 *)(s_fp + m * ST);
      float acc = 0.f;
#pragma unroll 8
      for (int i = 0; i < lane4; ++i) {
        const float4 q = __ldg(Ms + lane + 32 * i);
        const float4 f = F4[lane + 32 * i];
        acc = fmaf(q.x, f.x, acc);
        acc = fmaf(q.y, f.y, acc);
        acc = fmaf(q.z, f.z, acc);
        acc = fmaf(q.w, f.w, acc);
      }
      acc = warp_sumf(acc);
      if (lane == 0) s_pp[q] = acc;
    }
    __syncthreads();
    for (int s = tid; s < ns; s += nthr) {  // all-zero subtiles contribute exact zeros
      double acc = 0.0;
      for (int q = s_pst[s]; q < s_pst[s + 1]; ++q) acc += (double)s_pp[q];
      a.part[(size_t)blockIdx.x * stride + s] = acc;
    }
    ++nsync;
    if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }
    // fixed-order sums over CTAs: warp w of CTA b owns slot b + G*w
    for (int s = blockIdx.x + (int)gridDim.x * warp; s < ns; s += (int)gridDim.x * nwarp) {
      double acc = 0.0;
      for (int c = lane; c < (int)gridDim.x; c += 32) acc += __ldcg(a.part + (size_t)c * stride + s);
      acc = warp_sum(acc);
      if (lane == 0) a.gred[s] = acc;
    }
    ++nsync;
    if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }
    if (timer) { unsigned long long c1 = vmat_globaltimer(); tA += c1 - c0; c0 = c1; }

    // ---------------- gradient, residual, direction (same in every CTA)
    for (int s = tid; s < ns; s += nthr) {
      const double dg = dG_inv(s_y, s_igl, s_igr, N, s_beam[s]);
      s_dgy[s] = dg;
      s_g[s] = __ldcg(a.gred + s) + a.gamma * dg;
    }
    __syncthreads();
    if (warp == 0) {
      double r = 0.0, ym = 0.0, gm = 0.0, dyg = 0.0, dgg = 0.0;
      for (int s = lane; s < ns; s += 32) {
        const double yk = s_y[s_beam[s]], gk = s_g[s];
        r = fmax(r, fabs(fmin(yk, gk)));
        ym = fmax(ym, fabs(yk));
        gm = fmax(gm, fabs(gk));
        const double dg = gk - s_gold[s];
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
      const double ref = fmax(a.rho_ref, a.rho_plan ? *a.rho_plan : 0.0);
      tol = a.kkt_tol * fmax(fmax(rho0, ref), 1e-300);
    }
    if (rho <= tol) { status = VMAT_OK; break; }
    if (it >= a.max_iters) { status = VMAT_ENOTCONV; break; }
    const double step = s_sc[1];
    for (int s = tid; s < ns; s += nthr) {
      const int k = s_beam[s];
      const double yk = s_y[k];
      const double p = yk - step * s_g[s];
      const double dk = (p > 0.0 ? p : 0.0) - yk;
      s_d[k] = dk;
      s_df[s] = (float)dk;
      s_gold[s] = s_g[s];
    }
    __syncthreads();
    if (warp == 0) {  // g.d (full gradient: phi'(0)), dG(y).d and G(d)
      double gd = 0.0, g0 = 0.0;
      for (int s = lane; s < ns; s += 32) {
        const double dk = s_d[s_beam[s]];
        gd += s_dgy[s] * dk;
        g0 += s_g[s] * dk;
      }
      gd = warp_sum(gd);
      g0 = warp_sum(g0);
      const double Gd = G_inv(s_d, s_igr, N);
      if (lane == 0) { s_sc[2] = gd; s_sc[3] = Gd; s_sc[4] = g0; }
    }
    __syncthreads();
    const double gdot = s_sc[2], Gd = s_sc[3], phi0 = s_sc[4];
    if (timer) { unsigned long long c1 = vmat_globaltimer(); tS += c1 - c0; c0 = c1; }

    // ---------------- pass B: z = M y, w = M d
#pragma unroll
    for (int v = 0; v < VPT; ++v) { z[v] = 0.f; w[v] = 0.f; }
#pragma unroll 4
    for (int q = 0; q < nnzs; ++q) {
      const int s = s_nz[q], mk = s_mask[s];
      const float *Ms = a.M + (size_t)s * a.Vpad;
      const float ys = s_yf[s], ds = s_df[s];
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        if (!(mk >> m & 1)) continue;
        const float4 q = __ldg((const float4 *)(Ms + SUB_OFF(m)) + tid);
        z[4 * m] = fmaf(q.x, ys, z[4 * m]);         w[4 * m] = fmaf(q.x, ds, w[4 * m]);
        z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]); w[4 * m + 1] = fmaf(q.y, ds, w[4 * m + 1]);
        z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]); w[4 * m + 2] = fmaf(q.z, ds, w[4 * m + 2]);
        z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]); w[4 * m + 3] = fmaf(q.w, ds, w[4 * m + 3]);
      }
    }
    if (timer) { unsigned long long c1 = vmat_globaltimer(); tB += c1 - c0; c0 = c1; }

    // ---------------- exact line search on [0, 1]
    // phi'(t) = phi'(0) + sum_j D_j(t) + 2 gamma G(d) t, phi'(0) = g.d from the
    // reduced gradient; thread 0 keeps the bracket [lo, hi] (phi'(lo) < 0 <
    // phi'(hi)) and picks the trial points; all CTAs see the same sums.
    const double cg1 = 2.0 * a.gamma * Gd;
    double *s_ls_state = s_sc + 8;  // lo_t lo_f lo_h hi_t hi_f hi_h t done
    if (tid == 0) {
      s_ls_state[0] = 0.0; s_ls_state[1] = phi0; s_ls_state[2] = -1.0;
      s_ls_state[3] = 1.0; s_ls_state[4] = 0.0; s_ls_state[5] = -1.0;
      s_ls_state[6] = -1.0; s_ls_state[7] = phi0 < 0.0 ? 0.0 : 1.0;
      if (!(phi0 < 0.0)) s_ls_state[6] = 0.0;  // not a descent direction
    }
    __syncthreads();
    for (int r = 0; r < LS_ROUNDS && s_ls_state[7] == 0.0; ++r) {
      if (tid < LS_POINTS) {
        const double lo_t = s_ls_state[0], lo_f = s_ls_state[1], lo_h = s_ls_state[2];
        const double hi_t = s_ls_state[3], hi_f = s_ls_state[4], hi_h = s_ls_state[5];
        double tq;
        if (r == 0) {
          tq = (double)(tid + 1) / (double)LS_POINTS;  // 1/16 .. 1
        } else {
          const double span = hi_t - lo_t;
          if (tid == 0) tq = lo_h > 0.0 ? lo_t - lo_f / lo_h : -1.0;
          else if (tid == 1) tq = hi_h > 0.0 ? hi_t - hi_f / hi_h : -1.0;
          else tq = lo_t + span * (double)(tid - 1) / (double)(LS_POINTS - 1);
          if (!(tq > lo_t && tq < hi_t)) tq = lo_t + span * (tid == 0 ? 0.5 : 0.75);
        }
        s_t[tid] = (float)tq;
      }
      __syncthreads();
      ++nsync;
      if (!ls_round<VPT>(a, z, w, my_sid, s_tab, s_t, s_ls, s_res, s_i, ls_parity, stride)) {
        alive = false;
        break;
      }
      ls_parity ^= 1;
      if (tid == 0) {
        double lo_t = s_ls_state[0], lo_f = s_ls_state[1], lo_h = s_ls_state[2];
        double hi_t = s_ls_state[3], hi_f = s_ls_state[4], hi_h = s_ls_state[5];
        double t = -1.0;
        for (int p = 0; p < LS_POINTS; ++p) {
          const double tp = (double)s_t[p];
          const double f = phi0 + s_res[p] + cg1 * tp, h = s_res[LS_POINTS + p] + cg1;
          if (r == 0 && p == 0) lo_h = h;  // slope just right of 0 (first point's side pattern)
          if (r == 0 && p == LS_POINTS - 1) {
            if (f <= 0.0) { t = 1.0; break; }
            if (hi_h < 0.0) { hi_f = f; hi_h = h; }
          }
          if (f == 0.0) { t = tp; break; }
          if (f < 0.0 && tp > lo_t && tp < hi_t) { lo_t = tp; lo_f = f; lo_h = h; }
          if (f > 0.0 && tp < hi_t && tp > lo_t) { hi_t = tp; hi_f = f; hi_h = h; }
        }
        if (t < 0.0) {
          const double span = hi_t - lo_t;
          const double tsec = lo_t - lo_f * span / (hi_f - lo_f);
          const double na = lo_h > 0.0 ? lo_t - lo_f / lo_h : -1.0;
          const double nb = hi_h > 0.0 ? hi_t - hi_f / hi_h : -2.0;
          // both ends on one linear piece of phi' (their Newton steps agree): exact
          if (!(span > 0.0) || fabs(na - nb) <= 1e-6 * fabs(tsec) || span <= 1e-7 * hi_t ||
              r == LS_ROUNDS - 1)
            t = tsec;
        }
        s_ls_state[0] = lo_t; s_ls_state[1] = lo_f; s_ls_state[2] = lo_h;
        s_ls_state[3] = hi_t; s_ls_state[4] = hi_f; s_ls_state[5] = hi_h;
        if (t >= 0.0) { s_ls_state[6] = fmin(fmax(t, lo_t), 1.0); s_ls_state[7] = 1.0; }
      }
      __syncthreads();
    }
    if (!alive) break;
    const double t = s_ls_state[6] >= 0.0 ? s_ls_state[6] : s_ls_state[0];
    if (timer) { unsigned long long c1 = vmat_globaltimer(); tL += c1 - c0; c0 = c1; }
    if (t <= 0.0) { status = VMAT_ENOTCONV; break; }

    // ---------------- update
    for (int s = tid; s < ns; s += nthr) {
      const int k = s_beam[s];
      const double dy = t * s_d[k];
      s_dy[s] = dy;
      s_y[k] += dy;
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
#pragma unroll 4
  for (int q = 0; q < nnzs; ++q) {
    const int s = s_nz[q], mk = s_mask[s];
    const float *Ms = a.M + (size_t)s * a.Vpad;
    const float ys = s_yf[s];
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      if (!(mk >> m & 1)) continue;
      const float4 q = __ldg((const float4 *)(Ms + SUB_OFF(m)) + tid);
      z[4 * m] = fmaf(q.x, ys, z[4 * m]);
      z[4 * m + 1] = fmaf(q.y, ys, z[4 * m + 1]);
      z[4 * m + 2] = fmaf(q.z, ys, z[4 * m + 2]);
      z[4 * m + 3] = fmaf(q.w, ys, z[4 * m + 3]);
    }
  }
  double cst = 0.0;
#pragma unroll
  for (int m = 0; m < NG; ++m) {
    float zo[4], fo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = 4 * m + q, id = my_sid[v];
      fo[q] = vmat_dF(z[v], s_tab[id], s_tab[256 + id], s_tab[512 + id]);
      zo[q] = z[v];
      cst += vmat_F((double)z[v], a.tabd[id], a.tabd[256 + id], a.tabd[512 + id]);
    }
    const size_t off = SUB_OFF(m) + 4 * tid;
    *(float4 *)(a.z_out + off) = make_float4(zo[0], zo[1], zo[2], zo[3]);
    *(float4 *)(a.fp_out + off) = make_float4(fo[0], fo[1], fo[2], fo[3]);
  }
  cst = warp_sum(cst);
  if (lane == 0) s_res[32 + warp] = cst;
  __syncthreads();
  if (tid == 0) {
    double c = 0.0;
    for (int q = 0; q < nwarp; ++q) c += s_res[32 + q];
    a.part[(size_t)blockIdx.x * stride + COST_OFF(N)] = c;
  }
  ++nsync;
  if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) {
    if (blockIdx.x == 0 && tid == 0) a.out->status = VMAT_ETIMEOUT;
    return;
  }
  if (blockIdx.x == 0) {
    if (warp == 0) {
      double c = 0.0;
      for (int q = lane; q < (int)gridDim.x; q += 32)
        c += __ldcg(a.part + (size_t)q * stride + COST_OFF(N));
      c = warp_sum(c);
      const double G = G_inv(s_y, s_igr, N);
      if (lane == 0) {
        a.out->cost_active = c;
        a.out->smooth = G;
        a.out->rho = rho;
        a.out->rho0 = rho0;
        a.out->iters = it;
        a.out->status = status;
        if (a.set_rho_plan && a.rho_plan) *a.rho_plan = rho0;
        if (a.rec_cost) *a.rec_cost = c + a.inactive_cost + a.gamma * G;
        if (a.rec_rho) *a.rec_rho = rho;
        if (a.rec_iters) *a.rec_iters = it;
        if (a.rec_status) *a.rec_status = status;
        if (a.stats) {
          a.stats[0] += (double)tA;
          a.stats[1] += (double)tS;
          a.stats[2] += (double)tB;
          a.stats[3] += (double)tL;
          a.stats[4] += (double)nsync;
          a.stats[5] += (double)it;
        }
      }
    }
    for (int k = tid; k < N; k += nthr) a.y[k] = s_y[k];
  }
}

// ---------------------------------------------------------------- launch
static size_t master_smem_bytes(int N, int nthr, int vpt) {
  const size_t tile = (size_t)nthr * vpt, ng = vpt / 4;
  return (size_t)(8 * N + 32 + 32 + 16 * 32) * 8 +
         (size_t)(2 * N + 768 + LS_POINTS + 16 * 32) * 4 + tile * 4 + (size_t)N * ng * 4 +
         (size_t)(8 + 4 * N + 1 + N * ng) * 4 + 16;
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
  const int sms = ctx->sm_budget > 0 && ctx->sm_budget < ctx->num_sms ? ctx->sm_budget : ctx->num_sms;
  int vpt = 4, nthr = 0;
  for (vpt = 4; vpt <= 32; vpt *= 2) {
    int64_t threads = (Va + vpt - 1) / vpt;
    int64_t per_sm = (threads + sms - 1) / sms;
    nthr = (int)(((per_sm + 31) / 32) * 32);
    if (nthr < 64) nthr = 64;
    if (nthr <= 512) break;
  }
  if (vpt > 32) return vmat_fail(ctx, VMAT_EINVAL, "too many active voxels for the master kernel");
  int64_t chunk = (int64_t)nthr * vpt;
  int grid = (int)((Va + chunk - 1) / chunk);
  size_t smem = master_smem_bytes(ctx->N, nthr, vpt);
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

int64_t vmat_master_scratch(int grid, int N) { return (int64_t)grid * (N + PART_EXTRA) + N; }

vmat_status vmat_launch_master(vmat_ctx *ctx, int max_iters, double kkt_tol, double rho_ref,
                               int set_rho_plan, double *rec_cost, double *rec_rho,
                               int32_t *rec_iters, int32_t *rec_status) {
  MasterArgs a;
  a.M = ctx->M;
  a.tflag = ctx->tflag;
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
  a.stats = ctx->mstats;
  a.rec_cost = rec_cost;
  a.rec_rho = rec_rho;
  a.rec_iters = rec_iters;
  a.rec_status = rec_status;
  a.inactive_cost = ctx->inactive_cost;
  a.wait_ns = 2000000000ull;  // 2 s per grid-wide wait
  if (vmat_master_scratch(ctx->master_grid, ctx->N) > ctx->red_len)
    return vmat_fail(ctx, VMAT_EINVAL, "reduction scratch too small");
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 8, ctx->stream));
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
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = ctx->master_smem;
  lc.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident (the grid waits on itself)
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  VMAT_CUDA(ctx, cudaLaunchKernelExC(&lc, fn, args));
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
  // leave the context usable: a barrier word left mid-count is reset
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 8, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->dstatus, 0, 4, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  if (ds == VMAT_ETIMEOUT) return vmat_fail(ctx, VMAT_ETIMEOUT, "grid wait ran out (as designed)");
  if (ds != 0) return vmat_fail(ctx, (vmat_status)ds, "grid wait: status %d", ds);
  return VMAT_OK;
}

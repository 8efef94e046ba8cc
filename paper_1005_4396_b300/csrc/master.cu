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
// for the whole solve: the dose as its excess e = z - T over the voxel's
// threshold (Eq. 1 depends on z only through e) and the direction image w.  A column is nonzero
// only near its aperture's beam path: per (column, subtile) flags let every
// pass skip all-zero subtiles.  Per iteration:
//   pass A   gradient M^T F'(z): F' of the CTA's subtiles goes to shared
//            memory; each warp streams whole (column, subtile) pairs with
//            many independent 16-byte loads per lane; per lane, the four
//            products of each float4 are summed in FP32 and those block sums
//            compensated; then a compensated warp sum
//   reduce   per-slot CTA partials (FP32 rows) -> grid barrier -> every CTA
//            sums all rows in the same fixed order, compensated (one barrier;
//            deterministic, no float atomics)
//   step     every CTA forms the same d = P+(y - s g) - y from the same
//            reduced gradient; s is the adaptive Barzilai-Borwein step
//            (ABBmin, Frassoldati, Zanni and Zanghirati 2008): the long step
//            BB1 = dy.dy / dy.dg where it is close to the short one
//            BB2 = dy.dg / dg.dg, else the least BB2 of the last few
//            iterations; after 300 iterations of a solve BB2 alone (sixteen
//            seeded plans: 42% fewer iterations than BB2 alone)
//   pass B   w = M d, thread per voxel, column segments streamed through a
//            per-thread cp.async ring; e = M y - T is recomputed from y only
//            at the start and every 16th iteration (compensated, y as a float
//            pair; the solution's dose and F' are written from it) and
//            otherwise carried by the updates e += t w: the iterates then stay
//            consistent with the line that was searched, where a fresh FP32
//            product each iteration adds rounding noise to the gradient
//            differences the Barzilai-Borwein step is made of (3x more
//            iterations).  Gradient noise near the stopping tolerance is what
//            sets the iteration count: the excess form and the compensated
//            sums with the adaptive step below (which the noise of plain FP32
//            sums defeats) took a prostate plan from 21,400 to 11,700
//            iterations
//   search   phi'(t) = sum_j w_j F'(z_j + t w_j) + gamma*(dG(y).d + 2t G(d))
//            is piecewise linear and nondecreasing: each round evaluates it
//            at 16 points (FP32 per voxel, compensated FP32 across warps and
//            CTAs), one grid reduction per round; stop once Newton steps from both ends
//            of the bracket agree (same linear piece: the secant is exact).
//            Gradient projection takes the full step y + d first: the next
//            pass A computes the gradient there and, in the same reduction,
//            phi'(1); phi'(1) <= 0 makes t = 1 the minimiser (88% of a
//            prostate plan's iterations), so the iteration needs one grid
//            barrier.  Otherwise the rounds run from the saved point and the
//            point moves to y + t d before another pass A.  The iterates are
//            those of the line search at every step.
// Stop: rho = max_k |min(y_k, g_k)| <= tol * max(rho_start, rho_ref).
// The grid barrier is one counter whose top bit flips when every CTA has
// arrived; each wait is bounded in time and spins, after which the kernel
// records VMAT_ETIMEOUT and every CTA leaves.
#include <math.h>

#include "vmat_internal.cuh"

#define LS_POINTS 16
#define MAX_WARPS 32
#define LS_ROUNDS 4
// per-CTA partial row: [N slots | 2 x 32 line-search values | cost | spare]
#define PART_EXTRA 72
// Step rule of the gradient projection (the oracle uses the same rule):
// ABBmin with a memory of ABB_M short steps and switch ratio ABB_TAU for the
// first ABB_ITERS iterations of a solve, the short step BB2 after them.
#define ABB_M 3
#define ABB_TAU 0.5
#define ABB_ITERS 300
#define LS_OFF(N, parity) ((N) + 32 * (parity))
#define COST_OFF(N) ((N) + 64)

struct MasterArgs {
  const float *M;
  const float *Mlo;      // extended precision: [N][Vpad] each column entry minus its FP32 value
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
  float *gpart;          // [grid][(N+3)&~3] per-CTA gradient partials (16-byte aligned rows)
  unsigned *bar;         // [1] grid barrier word
  int *dstatus;
  float *z_out, *fp_out;  // [Vpad]
  float *fp_out_lo;       // extended precision: [Vpad] F' minus its FP32 value
  MasterOut *out;
  double *stats;         // [8] cumulative: ns in pass A+reduce, step, pass B, search; syncs; iters
  float *hpart;          // projected Newton: [grid][(N+1)(N+2)/2] per-CTA Gram partials
  float *hred;           // projected Newton: [(N+1)(N+2)/2] their sum (packed lower triangle)
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
                                          int *s_ok, unsigned long long *wait_acc = nullptr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long ta = wait_acc ? vmat_globaltimer() : 0ull;
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    unsigned old, cur;
    int ok = 1;
    // the release is cumulative: the CTA's partials, ordered before this
    // thread by the bar.sync above, are visible to every CTA that acquires
    // the flipped word (no separate fence needed)
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
    if (wait_acc) *wait_acc += vmat_globaltimer() - ta;  // arrival to release, as this CTA saw it
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

// Compensated FP32 accumulation (Neumaier's variant of Kahan summation): s
// holds the running sum, c the rounding error it has dropped; s + c carries
// about twice the precision of s, so a few hundred terms sum to FP64-like
// accuracy on the FP32 pipe (FP64 issues at a small fraction of its rate).
__device__ __forceinline__ void comp_add(float &s, float &c, float x) {
  const float t = __fadd_rn(s, x);
  c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
  s = t;
}

// F'(z) of Eq. 1 from the excess e = z - T of a voxel over its threshold
__device__ __forceinline__ float dF_e(float e, float al, float be) {
  return e > 0.f ? 2.f * be * e : (e < 0.f ? 2.f * al * e : 0.f);
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  const float t = __fadd_rn(a, b);
  const float bp = __fsub_rn(t, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bp)), __fsub_rn(b, bp));
  s = t;
}

// Extended precision: F'(z) = 2 c (eh + el) as a float pair (fh, fl), with
// the weight c = (ch + cl) of the voxel's side also a pair; the product's
// rounding error comes from an FMA, the small cross terms go to fl
__device__ __forceinline__ void dF_pair(float eh, float el, float alh, float all, float beh, float bel,
                                        float &fh, float &fl) {
  const bool over = eh > 0.f || (eh == 0.f && el > 0.f);
  const bool under = eh < 0.f || (eh == 0.f && el < 0.f);
  const float ch = over ? beh : (under ? alh : 0.f), cl = over ? bel : (under ? all : 0.f);
  const float c2 = 2.f * ch;  // exact
  fh = __fmul_rn(c2, eh);
  fl = __fmaf_rn(c2, eh, -fh) + 2.f * __fmaf_rn(ch, el, cl * eh);
}

// s + c += a * (bh + bl), compensated: the rounding error of a*bh comes
// exactly from an FMA, that of the sum from TwoSum (Knuth), and a*bl (bh + bl
// a float pair) goes to the correction term
__device__ __forceinline__ void dot2_add(float &s, float &c, float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  const float pe = __fmaf_rn(a, bh, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fmaf_rn(a, bl, __fadd_rn(e, pe)));
}

// s + c += q . f over a float4 (4 voxels of one column): the four products
// summed by one FMA chain in FP32, and that block sum added to (s, c)
// compensated (TwoSum).  The chain's few roundings, on four terms of
// neighbouring voxels, are the only error kept; over the ~500 blocks of a
// (column, subtile) pair they add up at random and stay below the rounding
// of the pair's result to FP32.  11 FP32 operations per 4 products, against
// 40 for products compensated one by one (TwoProduct and TwoSum each),
// which left the gradient pass bound by instruction issue.
__device__ __forceinline__ void dot4_add(float &s, float &c, const float4 &q, const float4 &f) {
  const float b = __fmaf_rn(q.w, f.w, __fmaf_rn(q.z, f.z, __fmaf_rn(q.y, f.y, __fmul_rn(q.x, f.x))));
  const float t = __fadd_rn(s, b);
  const float bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(b, bp));
  s = t;
  c = __fadd_rn(c, e);
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
// FP32 per voxel and within a warp, compensated FP32 across warps and CTAs
// in a fixed order.  Out, in lane l of warp 0 (lsv): sum_j D_j(t_l) for
// l < 16, sum_j 2 c_j(t_{l-16}) w_j^2 for l >= 16.
// The point-by-point sums live in a padded shared-memory row per thread
// (s_row, 33 floats), not in registers: they are touched only by the few
// voxels inside the bracket, and the registers stay free for z and w.
// structure id of the thread's voxel v (4 ids packed per word)
template <int NW>
__device__ __forceinline__ int sid_of(const uint32_t (&sidw)[NW], int v) {
  return (int)((sidw[v >> 2] >> (8 * (v & 3))) & 0xffu);
}

// The first half of a round: the thread's voxels (their excess from e0(v),
// their direction image w), the warp and CTA sums, and the CTA's 32 partials
// written to its row of a.part (parity selects one of two row halves, so that
// a round's partials are never overwritten while another CTA still reads the
// previous round's).
template <int VPT, typename E0>
__device__ __forceinline__ void ls_eval(const MasterArgs &a, E0 e0_of, const float (&w)[VPT],
                                        const uint32_t (&sid)[VPT / 4], const float *s_tab,
                                        const float *s_t, float *s_rows, float *s_ls, int parity,
                                        int stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  float t_first = s_t[0], t_last = s_t[0];
#pragma unroll
  for (int p = 1; p < LS_POINTS; ++p) {
    t_first = fminf(t_first, s_t[p]);
    t_last = fmaxf(t_last, s_t[p]);
  }
  float *v = s_rows + threadIdx.x * 33;  // all zero on entry; left zero on exit
  bool touched = false;
  float lin = 0.f;    // sum 2 c_j(0) w_j^2 over the thread's voxels
  float jump = 0.f;   // sum 2 w_j^2 (c_side - c_j(0)) over changes before t_first
  float at_first = 0.f;  // sum k_j (e_j + t_first w_j) over the same voxels
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const float wq = w[q];
    if (wq == 0.f) continue;
    const int id = sid_of(sid, q);
    const float al = s_tab[256 + id], be = s_tab[512 + id];
    const float e0 = e0_of(q);
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
    touched = true;
#pragma unroll
    for (int p = 0; p < LS_POINTS; ++p) {
      const float e = fmaf(s_t[p], wq, e0);
      if (e * wq > 0.f) {
        v[p] = fmaf(k, e, v[p]);
        v[LS_POINTS + p] += dh;
      }
    }
  }
  // lane l sums entry l of the warp's touched rows, in lane order
  // (conflict-free: row stride 33), and each touched row is zeroed again
  const unsigned rows = __ballot_sync(0xffffffffu, touched);
  float ws = 0.f;
  if (rows) {
    __syncwarp();
    const float *col = s_rows + warp * 32 * 33 + lane;
    for (unsigned m = rows; m; m &= m - 1) ws += col[(__ffs(m) - 1) * 33];
    __syncwarp();
    if (touched)
#pragma unroll
      for (int p = 0; p < 32; ++p) v[p] = 0.f;
  }
  lin = warp_sumf(lin);
  jump = warp_sumf(jump);
  at_first = warp_sumf(at_first);
  const float tp = s_t[lane & (LS_POINTS - 1)];
  ws += lane < LS_POINTS ? fmaf(lin, tp, fmaf(jump, tp - t_first, at_first)) : lin + jump;
  s_ls[warp * 32 + lane] = ws;
  __syncthreads();
  const int off = LS_OFF(a.N, parity);
  if (warp == 0) {  // the CTA's 32 sums, compensated over its warps, as FP32
    float cs = 0.f, cc = 0.f;
    for (int q = 0; q < nwarp; ++q) comp_add(cs, cc, s_ls[q * 32 + lane]);
    ((float *)(a.part + (size_t)blockIdx.x * stride + off))[lane] = __fadd_rn(cs, cc);
  }
}

// The second half, after the grid barrier: every CTA sums the CTAs' partials
// (warp w takes CTAs w, w + W, ..., 8 loads in flight per lane,
// compensated), then warp 0 combines the warps in order.  Out, in lane l of
// warp 0 (lsv): sum_j D_j(t_l) for l < 16, sum_j 2 c_j(t_{l-16}) w_j^2 for
// l >= 16.
__device__ __forceinline__ void ls_gather(const MasterArgs &a, double *s_res, int parity, int stride,
                                          double &lsv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int off = LS_OFF(a.N, parity);
  const int G = gridDim.x;
  float cs = 0.f, cc = 0.f;
  for (int c0 = warp; c0 < G; c0 += 8 * nwarp) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * nwarp;
      x[u] = c < G ? __ldcg((const float *)(a.part + (size_t)c * stride + off) + lane) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) comp_add(cs, cc, x[u]);
  }
  float2 *s_w2 = (float2 *)(s_res + 32);  // [nwarp][32]
  s_w2[warp * 32 + lane] = make_float2(cs, cc);
  __syncthreads();
  if (warp == 0) {
    float S = 0.f, C = 0.f;
    for (int q = 0; q < nwarp; ++q) {
      const float2 v = s_w2[q * 32 + lane];
      comp_add(S, C, v.x);
      C = __fadd_rn(C, v.y);
    }
    lsv = (double)S + (double)C;
  }
}

// One whole round: evaluation, grid barrier, gather.  Returns false if a wait
// ran out or another CTA reported an error.
template <int VPT, typename E0>
__device__ __forceinline__ bool ls_round(const MasterArgs &a, E0 e0_of, const float (&w)[VPT],
                                         const uint32_t (&sid)[VPT / 4], const float *s_tab,
                                         const float *s_t, float *s_rows, float *s_ls, double *s_res,
                                         int *s_ok, int parity, int stride, double &lsv,
                                         unsigned long long *wait_acc) {
  ls_eval<VPT>(a, e0_of, w, sid, s_tab, s_t, s_rows, s_ls, parity, stride);
  if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_ok, wait_acc)) return false;
  ls_gather(a, s_res, parity, stride, lsv);
  return true;
}

// Warp 0 after a round: lane p < 16 evaluates trial point p; the bracket
// moves to the largest point with phi' < 0 and the smallest with phi' > 0
// inside it (ties: lowest point index); every lane ends with the same state.
// phi'(t) = phi'(0) + sum_j D_j(t) + 2 gamma G(d) t with phi'(0) = g.d and
// G(d) from the warps' partials of the step phase (s_sc[32..], s_sc[48..]).
// State: lo_t lo_f lo_h hi_t hi_f hi_h t done; done with t once the
// minimiser is found (exact when both ends of the bracket lie on one linear
// piece of phi', else the secant after LS_ROUNDS rounds).
__device__ __forceinline__ void ls_bracket(int r, double lsv, const float *s_t, double *s_ls_state,
                                           const double *s_sc, int nwarp, double gamma) {
  const int lane = threadIdx.x & 31;
  // lane p < 16 evaluates trial point p; the bracket moves to the
  // largest point with phi' < 0 and the smallest with phi' > 0 inside
  // it (ties: lowest point index); every lane ends with the same state
  const unsigned FULL = 0xffffffffu;
  // the warps' phi'(0) and G(d) partials, in order (same values every round)
  float g0 = 0.f, gdd = 0.f;
  for (int q = 0; q < nwarp; ++q) {
    g0 += ((const float *)(s_sc + 32))[q];
    gdd += ((const float *)(s_sc + 48))[q];
  }
  const double phi0 = (double)g0, cg1 = 2.0 * gamma * (double)gdd;
  const int p = lane & (LS_POINTS - 1);
  const bool in = lane < LS_POINTS;
  const double tp = (double)s_t[p];
  const double f = phi0 + __shfl_sync(FULL, lsv, p) + cg1 * tp;
  const double h = __shfl_sync(FULL, lsv, p + LS_POINTS) + cg1;
  double lo_t = s_ls_state[0], lo_f = r == 0 ? phi0 : s_ls_state[1], lo_h = s_ls_state[2];
  double hi_t = s_ls_state[3], hi_f = s_ls_state[4], hi_h = s_ls_state[5];
  double t = -1.0;
  if (r == 0 && !(phi0 < 0.0)) t = 0.0;  // not a descent direction
  // an exact root among the points (round 0: before the full step t = 1)
  const unsigned zero = __ballot_sync(FULL, in && f == 0.0 && (r > 0 || p < LS_POINTS - 1));
  if (zero && t < 0.0) t = (double)s_t[__ffs(zero) - 1];
  if (r == 0) {
    lo_h = __shfl_sync(FULL, h, 0);  // slope just right of 0 (first point's side pattern)
    const double f1 = __shfl_sync(FULL, f, LS_POINTS - 1), h1 = __shfl_sync(FULL, h, LS_POINTS - 1);
    if (t < 0.0 && f1 <= 0.0) t = 1.0;
    if (hi_h < 0.0) { hi_f = f1; hi_h = h1; }
  }
  if (t < 0.0) {
    float key = (in && f < 0.0 && tp > lo_t && tp < hi_t) ? (float)tp : -1.f;
    int who = lane;
    for (int o = 16; o; o >>= 1) {
      const float k2 = __shfl_xor_sync(FULL, key, o);
      const int w2 = __shfl_xor_sync(FULL, who, o);
      if (k2 > key || (k2 == key && w2 < who)) { key = k2; who = w2; }
    }
    if (key >= 0.f) {
      lo_t = __shfl_sync(FULL, tp, who);
      lo_f = __shfl_sync(FULL, f, who);
      lo_h = __shfl_sync(FULL, h, who);
    }
    key = (in && f > 0.0 && tp > lo_t && tp < hi_t) ? (float)tp : 2.f;
    who = lane;
    for (int o = 16; o; o >>= 1) {
      const float k2 = __shfl_xor_sync(FULL, key, o);
      const int w2 = __shfl_xor_sync(FULL, who, o);
      if (k2 < key || (k2 == key && w2 < who)) { key = k2; who = w2; }
    }
    if (key <= 1.f) {
      hi_t = __shfl_sync(FULL, tp, who);
      hi_f = __shfl_sync(FULL, f, who);
      hi_h = __shfl_sync(FULL, h, who);
    }
    const double span = hi_t - lo_t;
    const double tsec = lo_t - lo_f * span / (hi_f - lo_f);
    // Newton steps from both ends (FP32: they only test agreement)
    const float na = lo_h > 0.0 ? (float)lo_t - (float)lo_f / (float)lo_h : -1.f;
    const float nb = hi_h > 0.0 ? (float)hi_t - (float)hi_f / (float)hi_h : -2.f;
    // both ends on one linear piece of phi' (their Newton steps agree): exact
    if (!(span > 0.0) || fabsf(na - nb) <= 1e-6f * fabsf((float)tsec) || span <= 1e-7 * hi_t ||
        r == LS_ROUNDS - 1)
      t = tsec;
  }
  if (lane == 0) {
    s_ls_state[0] = lo_t; s_ls_state[1] = lo_f; s_ls_state[2] = lo_h;
    s_ls_state[3] = hi_t; s_ls_state[4] = hi_f; s_ls_state[5] = hi_h;
    if (t >= 0.0) { s_ls_state[6] = fmin(fmax(t, lo_t), 1.0); s_ls_state[7] = 1.0; }
  }
}

// Trial points of round r, by threads 0..15 (FP32, as they are stored):
// round 0 at 1/16 .. 1; later rounds the Newton steps from both ends of the
// bracket and 14 points across it (a step outside it falls back to a point
// inside).  The caller synchronises before they are read.
__device__ __forceinline__ void ls_points(int r, float *s_t, const double *s_ls_state) {
  const int tid = threadIdx.x;
  if (tid >= LS_POINTS) return;
  float tq;
  if (r == 0) {
    tq = (float)(tid + 1) * (1.f / LS_POINTS);
  } else {
    const float lo_t = (float)s_ls_state[0], lo_f = (float)s_ls_state[1], lo_h = (float)s_ls_state[2];
    const float hi_t = (float)s_ls_state[3], hi_f = (float)s_ls_state[4], hi_h = (float)s_ls_state[5];
    const float span = hi_t - lo_t;
    if (tid == 0) tq = lo_h > 0.f ? lo_t - lo_f / lo_h : -1.f;
    else if (tid == 1) tq = hi_h > 0.f ? hi_t - hi_f / hi_h : -1.f;
    else tq = lo_t + span * (float)(tid - 1) * (1.f / (LS_POINTS - 1));
    if (!(tq > lo_t && tq < hi_t)) tq = lo_t + span * (tid == 0 ? 0.5f : 0.75f);
  }
  s_t[tid] = tq;
}

// Asynchronous 16-byte global -> shared copies (bypassing L1): a thread keeps
// several column segments in flight without holding them in registers.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One lane's share of a (column, subtile) pair in the gradient pass: all L
// float4 loads of the column issued at once, then summed against F' in
// shared memory
template <int L>
__device__ __forceinline__ void pair_dot(const float4 *Ms, const float4 *F4, int lane, float &acc,
                                         float &accc) {
  float4 q[L];
#pragma unroll
  for (int i = 0; i < L; ++i) q[i] = __ldg(Ms + lane + 32 * i);
#pragma unroll
  for (int i = 0; i < L; ++i) dot4_add(acc, accc, q[i], F4[lane + 32 * i]);
}

// Stages of the direction pass's copy pipeline: column segments in flight per thread
__host__ __device__ constexpr int master_pipe_stages(int vpt) { return vpt >= 16 ? 8 : 16; }

// Threads per CTA at most.  (768-thread CTAs at 4 voxels per thread, one
// subtile per CTA, measured slower on the prostate plan: 37.8 against 25.3 us
// per iteration; the CTAs holding the dense subtiles set the pace, and the
// per-warp combinations of the step and the sums grow with the warp count.)
__host__ __device__ constexpr int master_max_threads(int) { return 512; }

// Floats of the region holding the line-search rows ([nthr][33]); the
// direction pass runs its copy pipeline ([stages][nthr] float4) there, and
// the projected-Newton variant stages its Gram chunks ([64][N+8]) and its
// packed factor ((N+1)(N+2)/2) there.  A multiple of 4 (keeps what follows
// 16-byte aligned).
__host__ __device__ __forceinline__ int master_rows_len(int N, int nthr, int vpt, bool newton) {
  int r = max(33, 4 * master_pipe_stages(vpt)) * nthr;  // rows; direction-pass pipeline
  if (newton) {
    const int st = 64 * (N + 8) + 16 * nthr, fac = (N + 1) * (N + 2) / 2;  // staging + slice partials
    r = max(r, max(st, fac));
  }
  return (r + 3) & ~3;
}

// ---------------------------------------------------------------- projected Newton
// Packed lower triangle: entry (i, j), j <= i, at i(i+1)/2 + j.
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// Cholesky of the n x n leading block of the packed (n+1) x (n+1) matrix A
// whose last row holds a right-hand side b: afterwards A's rows 0..n-1 hold
// L below the diagonal (diagonal in dg), and row n holds y with L y = b (the
// forward substitution rides along).  Right-looking, one CTA barrier per
// pivot; the pivot column travels in a double-buffered copy (cb) so that the
// next column is gathered by the threads that update it.  Returns false in
// every thread if a pivot is not positive.
__device__ bool chol_packed_aug(float *A, int n, float *cb, float *dg) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5,
            nwarp = nthr >> 5;
  for (int i = tid; i <= n; i += nthr) cb[i] = A[pk(i, 0)];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const float *c = cb + (k & 1) * (n + 1);
    float *cn = cb + ((k + 1) & 1) * (n + 1);
    const float d = c[k];
    if (!(d > 0.f) || !isfinite(d)) return false;
    const float sq = sqrtf(d), isq = 1.f / sq, inv = 1.f / d;
    if (tid == 0) dg[k] = sq;
    for (int i = k + 1 + warp; i <= n; i += nwarp) {
      const float ci = c[i];
      if (lane == 0) A[pk(i, k)] = ci * isq;
      const float f = -ci * inv;
      const int jmax = i < n - 1 ? i : n - 1;
      float *row = A + pk(i, 0);
      for (int j = k + 1 + lane; j <= jmax; j += 32) {
        const float v = fmaf(f, c[j], row[j]);
        row[j] = v;
        if (j == k + 1) cn[i] = v;
      }
    }
    __syncthreads();
  }
  return true;
}

// e = M y - T for the thread's VPT voxels (4 per subtile, subtile m at
// off0 + m * mstride), compensated: starting from -T, every product of a
// column entry with y (a float pair) enters through dot2_add.  Near the
// solution many voxels sit close to their thresholds; there e is small and
// this keeps it exact to a few units of its own last place, where plain FP32
// sums of z would carry errors of the size of T's.  Each subtile's nonzero
// columns (ascending slots, the order of the direction pass's refresh) stream
// through the shared-memory ring `pipe` of STG copies per thread; the caller
// waits for the ring to drain before reusing it.
template <int VPT, bool XP, int STG>
__device__ __forceinline__ void excess_from_y(const MasterArgs &a, float *z, float *zlo,
                                              const uint32_t (&my_sid)[VPT / 4], const float *s_tab,
                                              const float *s_tablo, const int *s_mcnt,
                                              const int *s_mcols, int N, const float *s_yf,
                                              const float *s_ylo, float4 *pipe, size_t off0,
                                              size_t mstride) {
  constexpr int NG = VPT / 4;
  const int tid = threadIdx.x, nthr = blockDim.x;
#pragma unroll
  for (int m = 0; m < NG; ++m) {
    const int nm = s_mcnt[m];
    const int *cl = s_mcols + m * N;
    const float *src = a.M + off0 + m * mstride + 4 * tid;
    float zz[4], zc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      zz[q] = -s_tab[sid_of(my_sid, 4 * m + q)];
      zc[q] = XP ? -s_tablo[sid_of(my_sid, 4 * m + q)] : 0.f;  // extended: T as a float pair
    }
#pragma unroll
    for (int k = 0; k < STG; ++k) {
      if (k < nm) cp_async16(pipe + k * nthr + tid, src + (size_t)cl[k] * a.Vpad);
      cp_async_commit();
    }
    for (int q = 0; q < nm; ++q) {
      cp_async_wait<STG - 1>();
      const int slot = q & (STG - 1);
      const float4 v = pipe[slot * nthr + tid];
      const int sl = cl[q];
      const float ys = s_yf[sl], yl = s_ylo[sl];
      dot2_add(zz[0], zc[0], v.x, ys, yl);
      dot2_add(zz[1], zc[1], v.y, ys, yl);
      dot2_add(zz[2], zc[2], v.z, ys, yl);
      dot2_add(zz[3], zc[3], v.w, ys, yl);
      if (XP) {  // extended precision: the columns' low parts
        const float4 vl =
            __ldg((const float4 *)(a.Mlo + off0 + m * mstride + (size_t)sl * a.Vpad) + tid);
        zc[0] = fmaf(vl.x, ys, zc[0]);
        zc[1] = fmaf(vl.y, ys, zc[1]);
        zc[2] = fmaf(vl.z, ys, zc[2]);
        zc[3] = fmaf(vl.w, ys, zc[3]);
      }
      if (q + STG < nm) cp_async16(pipe + slot * nthr + tid, src + (size_t)cl[q + STG] * a.Vpad);
      cp_async_commit();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (XP)  // keep the excess as the pair (z, zlo)
        two_sum(zz[q], zc[q], z[4 * m + q], zlo[4 * m + q]);
      else
        z[4 * m + q] = __fadd_rn(zz[q], zc[q]);
    }
  }
}

// MAXT: the largest CTA the build serves.  Launches of at most 384 threads
// take a build bounded to 384 (up to 168 registers a thread, where 512
// threads allow 128 and the kernel would spill).
template <int VPT, bool NEWTON, bool XP, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_master(MasterArgs a) {
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
  int *s_slot = (int *)(s_igr + N);  // [N] slot of each beam, -1 if none (N doubles reserved)
  // per-warp scratch below is sized for up to MAX_WARPS warps per CTA
  double *s_sc = s_igr + 2 * N;      // [32 + 32] CTA-wide scalars, then per-warp phi'(0), G(d)
  double *s_res = s_sc + 64;         // [32 + 32*32] line-search sums and scratch
  const int Np = (N + 1) & ~1;                    // keeps the float region below 16-byte aligned
  double *s_ysave = s_res + 32 + MAX_WARPS * 32;  // [Np] gradient projection: y at the accepted point
  float *s_yf = (float *)(s_ysave + Np);          // [Np] per slot
  float *s_df = s_yf + Np;                        // [Np] per slot
  float *s_ylo = s_df + Np;                       // [Np4] low part of y
  float *s_tab = s_ylo + ((Np + 3) & ~3);         // [768]
  float *s_t = s_tab + 768;                       // [LS_POINTS] trial points
  float *s_ls = s_t + LS_POINTS;                  // [MAX_WARPS][32] warp partials
  // s_fp is 16-byte aligned for its float4 accesses: the doubles above take a
  // multiple of 16 bytes and the floats (2 Np + 1808) a multiple of 4
  float *s_fp = s_ls + MAX_WARPS * 32;  // [NG][ST] F' (pass A)
  float *s_rows = s_fp + NG * ST;                 // [nthr][33] line-search rows, kept zero between rounds
  const int rows_len = master_rows_len(N, nthr, VPT, NEWTON);
  float *s_pp = s_rows + rows_len;                // [N*NG] warp partial per (slot, subtile) pair
  int *s_i = (int *)(s_pp + N * NG);              // [8]: 2 nonzero pairs, 3 free slots (Newton)
  int *s_beam = s_i + 8;                          // [N] beam of slot
  int *s_mask = s_beam + N;                       // [N] per slot: bit m = subtile m nonzero
  int *s_pst = s_mask + N;                        // [N+1] first pair of each slot
  int *s_pair = s_pst + N + 1;                    // [N*NG] pairs s*8+m in slot order
  int *s_mcnt = s_pair + N * NG;                  // [8] nonzero columns of each own subtile
  int *s_mcols = s_mcnt + 8;                      // [NG][N] those columns (slots), ascending
  // projected Newton only (the launch sizes these for that variant)
  int *s_fidx = s_mcols + N * NG;                 // [N] free slots F, in slot order
  int *s_sub = s_fidx + N;                        // [N] F positions kept after dropping blocked ones
  int *s_ncol = s_sub + N;                        // [8] free columns nonzero in each own subtile
  int *s_cols = s_ncol + 8;                       // [NG][N] their F positions
  float *s_x = (float *)(s_cols + NG * N);        // [N] Newton step on F'
  float *s_dg = s_x + N;                          // [N] diagonal of the Cholesky factor
  float *s_cb = s_dg + N;                         // [2][N+1] pivot-column buffers
  // idle while the Newton step is formed, so aliased: sqrt(c_j) of the own
  // voxels on the F' tile, the staged Gram chunks and then the packed factor
  // on the line-search rows (which are zeroed again afterwards)
  float *s_sq = s_fp;                             // [NG][ST]
  float *s_A = s_rows;                            // [max(64 (N+8), (N+1)(N+2)/2)]
  // extended precision only (the launch sizes it for that variant), after
  // the last region the variant uses: low parts of F' and of T, alpha, beta
  float *s_xp = (float *)(((uintptr_t)(NEWTON ? (void *)(s_cb + 2 * (N + 1)) : (void *)(s_mcols + N * NG)) +
                           15) & ~(uintptr_t)15);
  float *s_fpl = s_xp;                            // [NG][ST] low part of F' (pass A)
  float *s_tablo = s_xp + NG * ST;                // [768] T, alpha, beta minus their FP32 values
  float *s_pplo = s_tablo + 768;                  // [N*NG] low part of each pair's dot product
  // gradient projection only: the excess at the accepted point, [VPT][nthr]
  // (and its low parts in extended precision), after the last region in use
  float *s_zsave = (float *)(((uintptr_t)(NEWTON ? (void *)(s_cb + 2 * (N + 1))
                                                 : (XP ? (void *)(s_pplo + N * NG) : (void *)(s_mcols + N * NG))) +
                              15) & ~(uintptr_t)15);
  float *s_zlsave = s_zsave + VPT * nthr;

  for (int q = tid; q < 768; q += nthr) s_tab[q] = a.tabf[q];
  if (XP)
    for (int q = tid; q < 768; q += nthr) s_tablo[q] = (float)(a.tabd[q] - (double)a.tabf[q]);
  for (int k = tid; k < N; k += nthr) {
    s_y[k] = a.y[k];
    s_d[k] = 0.0;
    const bool hl = k > 0 || a.cyclic, hr = k < N - 1 || a.cyclic;
    s_igl[k] = hl ? 1.0 / (k > 0 ? a.theta[k] - a.theta[k - 1] : a.theta[0] + 360.0 - a.theta[N - 1])
                  : 0.0;
    s_igr[k] = hr ? 1.0 / (k < N - 1 ? a.theta[k + 1] - a.theta[k] : a.theta[0] + 360.0 - a.theta[N - 1])
                  : 0.0;
  }
  for (int k = tid; k < N; k += nthr) s_slot[k] = -1;
  __syncthreads();
  for (int s = tid; s < ns; s += nthr) {
    s_beam[s] = a.slot_beam[s];
    s_slot[a.slot_beam[s]] = s;
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
  if (warp == 0) {  // nonzero (column, subtile) pairs and per-subtile column lists, in slot order
    const unsigned lt = (1u << lane) - 1u;
    int np = 0, cnt[NG];
#pragma unroll
    for (int m = 0; m < NG; ++m) cnt[m] = 0;
    for (int base = 0; base < ns; base += 32) {
      const int s = base + lane;
      const int mk = s < ns ? s_mask[s] : 0;
      const int pc = __popc(mk);
      int incl = pc;  // inclusive prefix of the pair counts over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (s < ns) {
        int p = np + incl - pc;
        s_pst[s] = p;
#pragma unroll
        for (int m = 0; m < NG; ++m)
          if (mk >> m & 1) s_pair[p++] = s * 8 + m;
      }
      np += __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        const unsigned b = __ballot_sync(0xffffffffu, mk >> m & 1);
        if (mk >> m & 1) s_mcols[m * N + cnt[m] + __popc(b & lt)] = s;
        cnt[m] += __popc(b);
      }
    }
    if (lane == 0) {
      s_pst[ns] = np;
      s_i[2] = np;
#pragma unroll
      for (int m = 0; m < NG; ++m) s_mcnt[m] = cnt[m];
    }
  }
  __syncthreads();
  for (int s = tid; s < ns; s += nthr) {
    const double yk = s_y[s_beam[s]];
    s_yf[s] = (float)yk;
    s_ylo[s] = (float)(yk - (double)(float)yk);
  }
  const int npairs = s_i[2];

  uint32_t my_sid[NG];
#pragma unroll
  for (int m = 0; m < NG; ++m) my_sid[m] = __ldg((const uint32_t *)(a.sid + SUB_OFF(m)) + tid);
  float z[VPT], w[VPT];
  float zl[XP ? VPT : 1];  // extended precision: low part of the excess
  __syncthreads();

  // the dose excess e = M y - T of the thread's voxels
  excess_from_y<VPT, XP, master_pipe_stages(VPT)>(a, z, XP ? zl : nullptr, my_sid, s_tab,
                                                   XP ? s_tablo : nullptr, s_mcnt, s_mcols, N, s_yf,
                                                   s_ylo, (float4 *)s_rows, SUB_OFF(0), G * ST);
  cp_async_wait<0>();
  __syncthreads();  // every thread's copies have landed before the rows are cleared
  for (int q = tid; q < 33 * nthr; q += nthr) s_rows[q] = 0.f;

  int it = 0, status = VMAT_ENOTCONV, nsync = 0;
  double rho = 0.0, rho0 = 0.0, tol = 0.0;
  double bb2_hist[ABB_M - 1];  // the last short steps, newest first (same in every thread)
#pragma unroll
  for (int q = 0; q < ABB_M - 1; ++q) bb2_hist[q] = INFINITY;
  bool alive = true;
  int ls_parity = 0;
  // gradient projection: while `trial` holds, z and s_y are the full step
  // (y + d, e + w) from the point saved in s_ysave / s_zsave, whose gradient
  // the pass computes together with the first line-search round along d
  bool trial = false;
  int gpar = 0;        // which of the two sets of gradient rows this pass writes
  int n_partial = 0;   // (CTA 0) steps whose exact minimiser was short of the full step
  // phase clocks of CTA 0, kept in shared memory (one thread uses them)
  // [6]: A, step, B, search, last, grid-barrier waits (included in the phases)
  unsigned long long *s_clk = (unsigned long long *)(s_sc + 24);
  const bool timer = blockIdx.x == 0 && tid == 0;
  if (timer)
    for (int q = 0; q < 6; ++q) s_clk[q] = 0;

  for (;;) {
    if (timer) s_clk[4] = vmat_globaltimer();
    // ---------------- pass A: per-slot CTA partials of M^T F'(z)
#pragma unroll
    for (int m = 0; m < NG; ++m) {
      float4 f;
      if (XP) {
        float fh[4], fl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int v = 4 * m + q, id = sid_of(my_sid, v);
          dF_pair(z[v], zl[XP ? v : 0], s_tab[256 + id], s_tablo[256 + id], s_tab[512 + id],
                  s_tablo[512 + id], fh[q], fl[q]);
        }
        f = make_float4(fh[0], fh[1], fh[2], fh[3]);
        *(float4 *)(s_fpl + m * ST + 4 * tid) = make_float4(fl[0], fl[1], fl[2], fl[3]);
      } else {
        int id = sid_of(my_sid, 4 * m);
        f.x = dF_e(z[4 * m], s_tab[256 + id], s_tab[512 + id]);
        id = sid_of(my_sid, 4 * m + 1);
        f.y = dF_e(z[4 * m + 1], s_tab[256 + id], s_tab[512 + id]);
        id = sid_of(my_sid, 4 * m + 2);
        f.z = dF_e(z[4 * m + 2], s_tab[256 + id], s_tab[512 + id]);
        id = sid_of(my_sid, 4 * m + 3);
        f.w = dF_e(z[4 * m + 3], s_tab[256 + id], s_tab[512 + id]);
      }
      *(float4 *)(s_fp + m * ST + 4 * tid) = f;
    }
    if (!NEWTON && trial) {
      // the line search's phi'(1) beyond phi'(0) + 2 gamma G(d): per voxel
      // D_j(1) = 2 c_j(0) w_j^2 + 2 w_j (c' - c_j(0)) (e_j + w_j) if the voxel
      // crosses its threshold before t = 1 (e_j + w_j is the excess now in z),
      // reduced with the gradient (slot ns of the CTA rows)
      float d1 = 0.f, d1c = 0.f;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const float wv = w[v];
        if (wv == 0.f) continue;
        const int id = sid_of(my_sid, v);
        const float al = s_tab[256 + id], be = s_tab[512 + id];
        const float e0 = s_zsave[v * nthr + tid], e1 = z[v];
        const float cw = wv > 0.f ? be : al;  // side taken at the threshold itself
        const float c0 = e0 > 0.f ? be : (e0 < 0.f ? al : cw);
        float dv = 2.f * c0 * wv * wv;
        const float dc = cw - c0;
        if (dc != 0.f && e1 * wv > 0.f) dv = fmaf(2.f * wv * dc, e1, dv);
        d1 += dv;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, d1, o), c2 = __shfl_xor_sync(0xffffffffu, d1c, o);
        comp_add(d1, d1c, s2);
        d1c = __fadd_rn(d1c, c2);
      }
      if (lane == 0) ((float2 *)(s_res + 32))[warp] = make_float2(d1, d1c);
    }
    __syncthreads();
    for (int q = warp; q < npairs; q += nwarp) {
      const int s = s_pair[q] >> 3, m = s_pair[q] & 7;
      const float4 *Ms = (const float4 *)(a.M + (size_t)s * a.Vpad + SUB_OFF(m));
      const float4 *F4 = (const float4 *)(s_fp + m * ST);
      float acc = 0.f, accc = 0.f;
      if (XP) {  // F' and the column entries as pairs
        const float4 *L4 = (const float4 *)(s_fpl + m * ST);
        const float4 *Ml = (const float4 *)(a.Mlo + (size_t)s * a.Vpad + SUB_OFF(m));
#pragma unroll 4
        for (int i = 0; i < lane4; ++i) {
          const float4 q = __ldg(Ms + lane + 32 * i), ql = __ldg(Ml + lane + 32 * i);
          const float4 f = F4[lane + 32 * i], fl = L4[lane + 32 * i];
          dot2_add(acc, accc, q.x, f.x, fl.x);
          dot2_add(acc, accc, q.y, f.y, fl.y);
          dot2_add(acc, accc, q.z, f.z, fl.z);
          dot2_add(acc, accc, q.w, f.w, fl.w);
          accc = fmaf(ql.x, f.x, fmaf(ql.y, f.y, fmaf(ql.z, f.z, fmaf(ql.w, f.w, accc))));
        }
      } else {
        // the lane's whole share of the pair (lane4 = threads / 32 float4
        // loads) in flight at once: a runtime trip count below a loop's
        // unroll factor would issue the loads one at a time
        switch (lane4) {
#define PAIR_DOT_CASE(L) \
  case L: pair_dot<L>(Ms, F4, lane, acc, accc); break;
          PAIR_DOT_CASE(8) PAIR_DOT_CASE(9) PAIR_DOT_CASE(10) PAIR_DOT_CASE(11) PAIR_DOT_CASE(12)
          PAIR_DOT_CASE(13) PAIR_DOT_CASE(14) PAIR_DOT_CASE(15) PAIR_DOT_CASE(16)
#undef PAIR_DOT_CASE
          default:
#pragma unroll 8
            for (int i = 0; i < lane4; ++i) {
              const float4 q = __ldg(Ms + lane + 32 * i);
              dot4_add(acc, accc, q, F4[lane + 32 * i]);
            }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, acc, o), c2 = __shfl_xor_sync(0xffffffffu, accc, o);
        comp_add(acc, accc, s2);
        accc = __fadd_rn(accc, c2);
      }
      if (lane == 0) {
        if (XP) {  // the pair's dot product stays a (value, correction) pair
          two_sum(acc, accc, s_pp[q], s_pplo[q]);
        } else {
          s_pp[q] = __fadd_rn(acc, accc);
        }
      }
    }
    __syncthreads();
    const int fstride = (N + 4) & ~3;  // slots, then (gradient projection) phi'(1) at slot ns
    // two sets of rows, alternating from one gradient pass to the next: the
    // gradient projection passes only one grid barrier per iteration, so a
    // CTA may write this pass's row while another still reads the last one
    float *gp = a.gpart + (size_t)gpar * 2 * G * fstride;
    float *grow = gp + (size_t)blockIdx.x * fstride;
    // extended precision: the low parts of the CTA rows follow all G rows
    float *growlo = gp + (size_t)(G + blockIdx.x) * fstride;
    for (int s = tid; s < ((ns + 4) & ~3); s += nthr) {  // all-zero subtiles contribute exact zeros
      float cs = 0.f, cc = 0.f;
      if (s < ns) {
        for (int q = s_pst[s]; q < s_pst[s + 1]; ++q) {
          comp_add(cs, cc, s_pp[q]);
          if (XP) cc = __fadd_rn(cc, s_pplo[q]);
        }
      } else if (s == ns && !NEWTON && trial) {
        for (int q = 0; q < nwarp; ++q) {
          const float2 v = ((const float2 *)(s_res + 32))[q];
          comp_add(cs, cc, v.x);
          cc = __fadd_rn(cc, v.y);
        }
      }
      if (XP) {
        two_sum(cs, cc, grow[s], growlo[s]);
      } else {
        grow[s] = __fadd_rn(cs, cc);
      }
    }
    ++nsync;
    if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i, timer ? s_clk + 5 : nullptr)) { alive = false; break; }
    {  // every CTA sums every CTA's row in the same fixed order (compensated):
       // warp w takes CTAs w, w + W, ... (8 loads in flight per lane), lane l
       // slots 4l..4l+3 of each 128-slot chunk; then the warps are combined
      const int n4 = (ns + 4) >> 2;     // the slots and slot ns
      float2 *s_gw = (float2 *)s_rows;  // [nwarp][128] (the rows are free until pass B)
      for (int c4 = 0; c4 < n4; c4 += 32) {
        const int j = c4 + lane;
        float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
        constexpr int GB = VPT >= 16 ? 4 : 8;  // loads in flight per lane (registers are tight at 16+)
        for (int c0 = warp; c0 < G; c0 += GB * nwarp) {
          float4 xv[GB];
#pragma unroll
          for (int u = 0; u < GB; ++u) {
            const int c = c0 + u * nwarp;
            xv[u] = (c < G && j < n4) ? __ldcg((const float4 *)(gp + (size_t)c * fstride) + j)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < GB; ++u) {
            comp_add(S[0], C[0], xv[u].x);
            comp_add(S[1], C[1], xv[u].y);
            comp_add(S[2], C[2], xv[u].z);
            comp_add(S[3], C[3], xv[u].w);
          }
          if (XP) {  // the CTA rows' low parts
#pragma unroll
            for (int u = 0; u < GB; ++u) {
              const int c = c0 + u * nwarp;
              const float4 lo = (c < G && j < n4)
                                    ? __ldcg((const float4 *)(gp + (size_t)(G + c) * fstride) + j)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
              C[0] = __fadd_rn(C[0], lo.x);
              C[1] = __fadd_rn(C[1], lo.y);
              C[2] = __fadd_rn(C[2], lo.z);
              C[3] = __fadd_rn(C[3], lo.w);
            }
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) s_gw[warp * 128 + 4 * lane + e] = make_float2(S[e], C[e]);
        __syncthreads();
        for (int t = tid; t < 128 && 4 * c4 + t <= ns; t += nthr) {
          float gs = 0.f, gc = 0.f;
          for (int q = 0; q < nwarp; ++q) {
            const float2 v = s_gw[q * 128 + t];
            comp_add(gs, gc, v.x);
            gc = __fadd_rn(gc, v.y);
          }
          if (4 * c4 + t < ns) s_g[4 * c4 + t] = (double)gs + (double)gc;  // M^T F'(z) of slot 4 c4 + t
          else s_sc[16] = (double)gs + (double)gc;  // sum_j D_j(1) (gradient projection)
        }
        __syncthreads();
      }
    }
    gpar ^= 1;
    if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[0] += c1 - s_clk[4]; s_clk[4] = c1; }

    // ---------------- gradient projection: the exact line search along d.
    // phi'(t) is nondecreasing, so t = 1 is its minimiser on [0, 1] exactly
    // when phi'(1) = g.d + sum_j D_j(1) + 2 gamma G(d) <= 0 (most iterations);
    // then the gradient just formed is the gradient at the new point and the
    // step follows at once.  Otherwise the search runs its rounds from the
    // saved point, the point moves to y + t d and a gradient pass follows.
    if (!NEWTON && trial) {
      double *s_ls_state = s_sc + 8;  // lo_t lo_f lo_h hi_t hi_f hi_h t done
      if (tid == 0) {  // phi'(0) and G(d) from the warps' partials of the step phase, in order
        float g0 = 0.f, gdd = 0.f;
        for (int q = 0; q < nwarp; ++q) {
          g0 += ((const float *)(s_sc + 32))[q];
          gdd += ((const float *)(s_sc + 48))[q];
        }
        const double phi0 = (double)g0, f1 = phi0 + s_sc[16] + 2.0 * a.gamma * (double)gdd;
        s_sc[17] = !(phi0 < 0.0) ? -1.0 : (f1 <= 0.0 ? 1.0 : 0.0);
      }
      __syncthreads();
      const double verdict = s_sc[17];
      const bool full = verdict > 0.0;
      if (verdict == 0.0) {
#pragma unroll
        for (int p = 0; p < 33; ++p) s_rows[tid * 33 + p] = 0.f;  // the gradient sum used them
        for (int r = 0; r < LS_ROUNDS && s_ls_state[7] == 0.0; ++r) {
          ls_points(r, s_t, s_ls_state);
          __syncthreads();
          ++nsync;
          double lsv = 0.0;
          if (!ls_round<VPT>(a, [&](int q) { return s_zsave[q * nthr + tid]; }, w, my_sid, s_tab, s_t,
                             s_rows, s_ls, s_res, s_i, ls_parity, stride, lsv, timer ? s_clk + 5 : nullptr)) {
            alive = false;
            break;
          }
          ls_parity ^= 1;
          if (warp == 0) ls_bracket(r, lsv, s_t, s_ls_state, s_sc, nwarp, a.gamma);
          __syncthreads();
        }
        if (!alive) break;
      }
      const double t = full ? 1.0 : (verdict < 0.0 ? 0.0 : (s_ls_state[6] >= 0.0 ? s_ls_state[6] : s_ls_state[0]));
      const float tf = (float)t;
      if (!full) {
        // back to the saved point and along d by t (t <= 0: stay there)
        const float tm = t > 0.0 ? tf : 0.f;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const float zs = s_zsave[v * nthr + tid];
          if (XP) {  // (z, zl) = saved + tf w, the product's rounding error from an FMA
            const float p = __fmul_rn(tm, w[v]), pe = __fmaf_rn(tm, w[v], -p);
            float sh, se;
            two_sum(zs, p, sh, se);
            two_sum(sh, __fadd_rn(s_zlsave[v * nthr + tid], __fadd_rn(se, pe)), z[v], zl[XP ? v : 0]);
          } else {
            z[v] = fmaf(tm, w[v], zs);
          }
        }
        for (int s = tid; s < ns; s += nthr) {
          const int k = s_beam[s];
          const double ys = s_ysave[k];
          if (!(t > 0.0)) {
            s_y[k] = ys;
          } else if (XP) {  // a full step onto the bound lands on 0 exactly; never below it
            const double yn = ys + (double)tf * (double)s_df[s];
            s_y[k] = (yn <= 0.0 || (t == 1.0 && s_d[k] == -ys)) ? 0.0 : yn;
          } else {
            s_y[k] = ys + t * s_d[k];
          }
        }
        if (timer) ++n_partial;
      }
      if (!(t > 0.0)) {
        __syncthreads();
        status = VMAT_ENOTCONV;
        break;
      }
      // the move just made, for the next Barzilai-Borwein step; y as a float
      // pair only before an iteration that refreshes e from it
      ++it;
      const bool pair_now = (it & 15) == 15;
      for (int s = tid; s < ns; s += nthr) {
        const int k = s_beam[s];
        s_dy[s] = XP ? (double)tf * (double)s_df[s] : t * s_d[k];
        if (pair_now) {
          s_yf[s] = (float)s_y[k];
          s_ylo[s] = (float)(s_y[k] - (double)s_yf[s]);
        }
      }
      trial = false;
      __syncthreads();
      if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[3] += c1 - s_clk[4]; s_clk[4] = c1; }
      if (!full) continue;  // the gradient at y + t d
    }

    // ---------------- gradient, residual, direction (same in every CTA)
    // y, g and d are formed in FP64, spread over all threads.  The KKT
    // residual and the magnitudes are maxima, taken exactly on the bit
    // patterns of the FP64 values (integer compares; y >= 0 always); the
    // Barzilai-Borwein inner products, phi'(0) = g.d (all terms <= 0) and G(d)
    // are taken in FP32.  Reductions: warp butterflies, then every thread
    // combines the warps' values in the same order.
    {
      const unsigned FULL = 0xffffffffu;
      const unsigned long long ABS = 0x7fffffffffffffffull;
      unsigned long long rb = 0, yb = 0, gb = 0;
      float dyg = 0.f, dgg = 0.f, dyy = 0.f;
      for (int s = tid; s < ns; s += nthr) {
        const int k = s_beam[s];
        const double gk = s_g[s] + a.gamma * dG_inv(s_y, s_igl, s_igr, N, k);
        s_g[s] = gk;
        const unsigned long long ybits = (unsigned long long)__double_as_longlong(s_y[k]) & ABS;
        const unsigned long long gbits = (unsigned long long)__double_as_longlong(gk);
        const unsigned long long gabs = gbits & ABS;
        rb = max(rb, (gbits >> 63) ? gabs : min(ybits, gabs));  // |min(y, g)|
        yb = max(yb, ybits);
        gb = max(gb, gabs);
        const float dgk = (float)(gk - s_gold[s]), dyk = (float)s_dy[s];
        dyg = fmaf(dyk, dgk, dyg);
        dgg = fmaf(dgk, dgk, dgg);
        dyy = fmaf(dyk, dyk, dyy);
      }
      for (int o = 16; o; o >>= 1) {
        rb = max(rb, __shfl_xor_sync(FULL, rb, o));
        yb = max(yb, __shfl_xor_sync(FULL, yb, o));
        gb = max(gb, __shfl_xor_sync(FULL, gb, o));
        dyg += __shfl_xor_sync(FULL, dyg, o);
        dgg += __shfl_xor_sync(FULL, dgg, o);
        dyy += __shfl_xor_sync(FULL, dyy, o);
      }
      unsigned long long *s_ru = (unsigned long long *)(s_res + 32);  // [3][MAX_WARPS]
      float *s_rf = (float *)(s_res + 32 + 3 * MAX_WARPS);            // [3][MAX_WARPS]
      if (lane == 0) {
        s_ru[warp] = rb;
        s_ru[MAX_WARPS + warp] = yb;
        s_ru[2 * MAX_WARPS + warp] = gb;
        s_rf[warp] = dyg;
        s_rf[MAX_WARPS + warp] = dgg;
        s_rf[2 * MAX_WARPS + warp] = dyy;
      }
      __syncthreads();
      // one thread combines the warps and takes the scalar decisions (FP64
      // issues at 1/64 of the FP32 rate on this GPU: redundant copies of this
      // logic in every thread cost ~1 us per iteration); the others read them
      if (tid == 0) {
        rb = yb = gb = 0;
        dyg = dgg = dyy = 0.f;
        for (int q = 0; q < nwarp; ++q) {
          rb = max(rb, s_ru[q]);
          yb = max(yb, s_ru[MAX_WARPS + q]);
          gb = max(gb, s_ru[2 * MAX_WARPS + q]);
          dyg += s_rf[q];
          dgg += s_rf[MAX_WARPS + q];
          dyy += s_rf[2 * MAX_WARPS + q];
        }
        rho = __longlong_as_double((long long)rb);
        if (it == 0) {
          rho0 = rho;
          const double ref = fmax(a.rho_ref, a.rho_plan ? *a.rho_plan : 0.0);
          tol = a.kkt_tol * fmax(fmax(rho0, ref), 1e-300);
        }
        double step = 0.0, verdict = 0.0;
        if (rho <= tol) {
          verdict = 1.0;
        } else if (it >= a.max_iters) {
          verdict = 2.0;
        } else if (it == 0) {
          step = fmax(__longlong_as_double((long long)yb), 1.0) /
                 fmax(__longlong_as_double((long long)gb), 1e-300);
        } else {
          // adaptive Barzilai-Borwein (ABBmin): where the two BB steps differ by
          // more than the factor ABB_TAU the least of the last ABB_M short (BB2)
          // steps, else the long (BB1) step; BB2 alone once a solve has taken
          // ABB_ITERS iterations (the rare solves where the adaptive rule
          // stalls then finish at BB2's pace)
          const double bb2 = (dyg > 0.f && dgg >= 1e-30f) ? (double)(dyg / dgg) : 1e12;
          const double bb1 = dyg > 0.f ? (double)(dyy / dyg) : 1e12;
          double hmin = bb2;
#pragma unroll
          for (int q = 0; q < ABB_M - 1; ++q) hmin = fmin(hmin, bb2_hist[q]);
#pragma unroll
          for (int q = ABB_M - 2; q > 0; --q) bb2_hist[q] = bb2_hist[q - 1];
          bb2_hist[0] = bb2;
          step = it >= ABB_ITERS ? bb2 : (bb2 < ABB_TAU * bb1 ? hmin : bb1);
        }
        s_sc[18] = fmin(fmax(step, 1e-12), 1e12);
        s_sc[19] = verdict;
        s_sc[20] = rho;
        s_sc[21] = rho0;
      }
      __syncthreads();
      rho = s_sc[20];
      rho0 = s_sc[21];
      if (s_sc[19] == 1.0) { status = VMAT_OK; break; }
      if (s_sc[19] == 2.0) { status = VMAT_ENOTCONV; break; }
      const double step = s_sc[18];
      bool newton_ok = false;
      if (NEWTON) {
        // ---- projected Newton: the Hessian of Eq. 3 on the free set
        // F = {y > 0 or g < 0} is M_F^T C M_F + 2 gamma L_FF (C = 2 alpha_j or
        // 2 beta_j by side, L the Laplacian of G); each CTA forms its voxels'
        // part of the Gram matrix of A = M_F sqrt(C), the CTAs' parts are
        // summed in a fixed order, and every CTA solves the same system.
        const int HPM = (N + 1) * (N + 2) / 2;
        if (tid == 0) {
          int nf = 0;
          for (int s = 0; s < ns; ++s)
            if (s_y[s_beam[s]] > 0.0 || s_g[s] < 0.0) s_fidx[nf++] = s;
          s_i[3] = nf;
          for (int m = 0; m < NG; ++m) {
            int c = 0;
            for (int q = 0; q < nf; ++q)
              if (s_mask[s_fidx[q]] >> m & 1) s_cols[m * N + c++] = q;
            s_ncol[m] = c;
          }
        }
#pragma unroll
        for (int m = 0; m < NG; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int v = 4 * m + q, id = sid_of(my_sid, v);
            const float e = z[v];
            s_sq[m * ST + 4 * tid + q] = sqrtf(2.f * (e > 0.f ? s_tab[512 + id] : s_tab[256 + id]));
          }
        __syncthreads();
        const int nf = s_i[3];
        if (nf > 0) {
          float *hp = a.hpart + (size_t)blockIdx.x * HPM;
          for (int q = tid; q < nf * (nf + 1) / 2; q += nthr) hp[q] = 0.f;
          float *s_part = s_A + 64 * (N + 8);  // [nthr][16] partial blocks of the voxel slices
          for (int m = 0; m < NG; ++m) {
            const int nm = s_ncol[m];
            if (nm == 0) continue;
            const int P = (nm + 3) >> 2, ldA = 4 * P + 4, nblk = P * (P + 1) / 2;
            const int *cols = s_cols + m * N;
            // KS voxel slices per 4x4 block when there are fewer blocks than
            // threads; the slices' partial blocks are added in slice order
            int KS = 1;
            while (KS < 8 && nblk * KS * 2 <= nthr) KS *= 2;
            const int bpr = nthr / KS, ks = tid / bpr, bl = tid - ks * bpr;
            for (int blk0 = 0; blk0 < nblk; blk0 += bpr) {
              const int blk = blk0 + bl;
              const bool act = ks < KS && blk < nblk;
              int bi = 0, bj = 0;
              if (act) {  // block (bi <= bj) of the upper triangle, row-major
                int r = 0, rem = blk;
                while (rem >= P - r) { rem -= P - r; ++r; }
                bi = r;
                bj = r + rem;
              }
              float acc[4][4];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = 0.f;
              for (int v0 = 0; v0 < ST; v0 += 64) {
                __syncthreads();
                for (int idx = tid; idx < 4 * P * 64; idx += nthr) {  // chunk of A^T: [voxel][column]
                  const int row = idx >> 6, v = idx & 63;
                  float val = 0.f;
                  if (row < nm)
                    val = __ldg(a.M + (size_t)s_fidx[cols[row]] * a.Vpad + SUB_OFF(m) + v0 + v) *
                          s_sq[m * ST + v0 + v];
                  s_A[v * ldA + row] = val;
                }
                __syncthreads();
                if (act) {
#pragma unroll 4
                  for (int v = ks; v < 64; v += KS) {
                    const float4 xa = *(const float4 *)(s_A + v * ldA + 4 * bi);
                    const float4 ya = *(const float4 *)(s_A + v * ldA + 4 * bj);
                    const float xs[4] = {xa.x, xa.y, xa.z, xa.w}, ys[4] = {ya.x, ya.y, ya.z, ya.w};
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                      for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fmaf(xs[ii], ys[jj], acc[ii][jj]);
                  }
                }
              }
              if (KS > 1) {
                if (act)
#pragma unroll
                  for (int e = 0; e < 16; ++e) s_part[tid * 16 + e] = acc[e >> 2][e & 3];
                __syncthreads();
                if (act && ks == 0)
                  for (int q = 1; q < KS; ++q)
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[e >> 2][e & 3] += s_part[(q * bpr + bl) * 16 + e];
              }
              if (act && ks == 0)
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                  for (int jj = 0; jj < 4; ++jj) {
                    const int ra = 4 * bi + ii, rb = 4 * bj + jj;
                    if (ra < nm && rb < nm && (bi != bj || ii <= jj))
                      hp[pk(cols[rb], cols[ra])] += acc[ii][jj];  // cols ascending: F position ra <= rb
                  }
            }
            __syncthreads();
          }
        }
        ++nsync;
        if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }
        if (nf > 0) {  // CTA b sums its share of the entries over the CTAs (compensated, fixed order)
          const int HPF = nf * (nf + 1) / 2, per = (HPF + G - 1) / G;
          const int q0 = blockIdx.x * per, q1 = min(HPF, q0 + per);
          float2 *s_w2 = (float2 *)(s_res + 32);  // [nwarp][32]
          for (int e0 = q0; e0 < q1; e0 += 32) {
            const int e = e0 + lane;
            float cs = 0.f, cc = 0.f;
            for (int c0 = warp; c0 < G; c0 += 8 * nwarp) {
              float xv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int c = c0 + u * nwarp;
                xv[u] = (c < G && e < q1) ? __ldcg(a.hpart + (size_t)c * HPM + e) : 0.f;
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) comp_add(cs, cc, xv[u]);
            }
            s_w2[warp * 32 + lane] = make_float2(cs, cc);
            __syncthreads();
            if (warp == 0 && e < q1) {
              float S = 0.f, C = 0.f;
              for (int q = 0; q < nwarp; ++q) {
                const float2 v = s_w2[q * 32 + lane];
                comp_add(S, C, v.x);
                C = __fadd_rn(C, v.y);
              }
              a.hred[e] = __fadd_rn(S, C);
            }
            __syncthreads();
          }
        }
        ++nsync;
        if (!grid_sync(a.bar, a.dstatus, a.wait_ns, s_i)) { alive = false; break; }
        // ---- solve H_F'F' x = -g_F', F' = F without the variables at zero
        // that the step would push below zero; then the longest step in [0, 1]
        // that keeps y >= 0 (ratio test; a per-variable projection of a step
        // scaled by a full inverse Hessian need not descend).  Any failure:
        // the gradient-projection step.
        int n = nf;
        for (int q = tid; q < nf; q += nthr) s_sub[q] = q;
        __syncthreads();
        bool solved = false;
        for (int rep = 0; rep < 8 && n > 0; ++rep) {
          const int tot = (n + 1) * (n + 2) / 2;
          for (int q = tid; q < tot; q += nthr) {
            int i = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
            while (pk(i, 0) > q) --i;
            while (pk(i + 1, 0) <= q) ++i;
            const int j = q - pk(i, 0);
            float v;
            if (i == n) {
              v = j == n ? 0.f : -(float)s_g[s_fidx[s_sub[j]]];
            } else {
              const int fi = s_sub[i], fj = s_sub[j];
              const int ki = s_beam[s_fidx[fi]], kj = s_beam[s_fidx[fj]];
              double lap = 0.0;  // Laplacian of G (Eq. 2) at (ki, kj)
              if (ki == kj) {
                lap = s_igl[ki] + s_igr[ki];
              } else {
                if (kj == (ki + 1) % N) lap -= s_igr[ki];
                if (ki == (kj + 1) % N) lap -= s_igr[kj];
              }
              v = __ldcg(a.hred + pk(fi, fj)) + (float)(2.0 * a.gamma * lap);
              if (i == j) v *= 1.f + 1e-6f;
            }
            s_A[q] = v;
          }
          __syncthreads();
          if (!chol_packed_aug(s_A, n, s_cb, s_dg)) break;
          if (warp == 0) {  // back substitution L^T x = y
            for (int k = n - 1; k >= 0; --k) {
              float acc = 0.f;
              for (int i = k + 1 + lane; i < n; i += 32) acc = fmaf(s_A[pk(i, k)], s_x[i], acc);
              acc = warp_sumf(acc);
              if (lane == 0) s_x[k] = (s_A[pk(n, k)] - acc) / s_dg[k];
              __syncwarp();
            }
          }
          __syncthreads();
          if (tid == 0) {  // drop variables at zero that the step pushes below zero
            int nk = 0;
            for (int i = 0; i < n; ++i) {
              const int fi = s_sub[i];
              if (!(s_y[s_beam[s_fidx[fi]]] <= 0.0 && s_x[i] < 0.f)) {
                s_sub[nk] = fi;
                s_x[nk] = s_x[i];
                ++nk;
              }
            }
            s_i[4] = nk;
          }
          __syncthreads();
          const int nk = s_i[4];
          if (nk == n) { solved = true; break; }
          n = nk;
        }
        if (solved) {
          // ratio test in FP64: tmax = min(1, min_{x_i < 0} y_i / -x_i), a
          // minimum of non-negative doubles taken on their bit patterns;
          // d = tmax x on F', 0 elsewhere, kept only if it descends (g.d < 0)
          unsigned long long tb = __double_as_longlong(1.0);
          for (int i = tid; i < n; i += nthr) {
            const double xi = (double)s_x[i];
            if (xi < 0.0) {
              const double r = s_y[s_beam[s_fidx[s_sub[i]]]] / -xi;
              tb = min(tb, (unsigned long long)__double_as_longlong(r));
            }
          }
          for (int o = 16; o; o >>= 1) tb = min(tb, __shfl_xor_sync(FULL, tb, o));
          unsigned long long *s_tb = (unsigned long long *)(s_res + 32);  // [nwarp]
          if (lane == 0) s_tb[warp] = tb;
          for (int s = tid; s < ns; s += nthr) s_d[s_beam[s]] = 0.0;
          __syncthreads();
          tb = s_tb[0];
          for (int q = 1; q < nwarp; ++q) tb = min(tb, s_tb[q]);
          const double tmax = __longlong_as_double((long long)tb);
          float gd = 0.f;
          for (int i = tid; i < n; i += nthr) {
            const int sl = s_fidx[s_sub[i]];
            const double di = tmax * (double)s_x[i];
            s_d[s_beam[sl]] = di;
            gd = fmaf((float)s_g[sl], (float)di, gd);
          }
          for (int o = 16; o; o >>= 1) gd += __shfl_xor_sync(FULL, gd, o);
          float *s_gd = (float *)(s_res + 32 + MAX_WARPS);  // [nwarp]
          if (lane == 0) s_gd[warp] = gd;
          __syncthreads();
          gd = 0.f;
          for (int q = 0; q < nwarp; ++q) gd += s_gd[q];
          newton_ok = tmax > 0.0 && gd < 0.f;  // same in every thread
          __syncthreads();
        }
        for (int q = tid; q < rows_len; q += nthr) s_rows[q] = 0.f;  // the line search needs them zero
      }
      float g0 = 0.f;
      for (int s = tid; s < ns; s += nthr) {
        const int k = s_beam[s];
        const double yk = s_y[k], gk = s_g[s];
        double dk;
        if (newton_ok) {
          dk = s_d[k];
        } else {
          const double p = yk - step * gk;
          dk = (p > 0.0 ? p : 0.0) - yk;
          s_d[k] = dk;
        }
        s_df[s] = (float)dk;
        s_gold[s] = gk;
        g0 = fmaf((float)gk, (float)dk, g0);
      }
      if (tid == 0) {  // line-search bracket [0, 1]; phi'(0) is filled in by warp 0
        double *st = s_sc + 8;
        st[0] = 0.0; st[1] = 0.0; st[2] = -1.0; st[3] = 1.0;
        st[4] = 0.0; st[5] = -1.0; st[6] = -1.0; st[7] = 0.0;
      }
      __syncthreads();
      float gdd = 0.f;  // G(d) over the beam pairs (unoccupied beams have d = 0)
      for (int k = tid; k < N; k += nthr) {
        const int kp = k < N - 1 ? k + 1 : 0;  // s_igr[N-1] = 0 on a path
        const float dd = (float)(s_d[kp] - s_d[k]);
        gdd = fmaf(dd * dd, (float)s_igr[k], gdd);
      }
      for (int o = 16; o; o >>= 1) {
        g0 += __shfl_xor_sync(FULL, g0, o);
        gdd += __shfl_xor_sync(FULL, gdd, o);
      }
      if (lane == 0) {  // summed over warps by warp 0 in the line search
        ((float *)(s_sc + 32))[warp] = g0;        // s_sc[32..47]
        ((float *)(s_sc + 48))[warp] = gdd;       // s_sc[48..63]
      }
    }
    if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[1] += c1 - s_clk[4]; s_clk[4] = c1; }

    // ---------------- pass B: w = M d (and z = M y)
    // per own subtile, the thread streams its 16 bytes of each nonzero column
    // through a private ring of shared-memory slots (STG copies in flight;
    // the columns are mostly L2-resident, so latency bounds this pass)
    // the excess e is carried by the updates e += t w; every 16th iteration it
    // is recomputed from y so that FP32 rounding cannot accumulate
    if (MAXT <= 384 && !XP) {
      // (the 384-thread build, with registers to spare) the segments in
      // batches of BQ plain 16-byte loads per thread, all in flight at once,
      // then summed in column order: the same sums as the ring below
      const bool refresh = (it & 15) == 15;
      constexpr int BQ = 6;  // (4..12 measured on the prostate plan: 6 is the fastest)
      const size_t vp4 = (size_t)a.Vpad / 4;
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        const int nm = s_mcnt[m];
        const int *cl = s_mcols + m * N;
        const float4 *src = (const float4 *)(a.M + SUB_OFF(m)) + tid;
        float4 ww = make_float4(0.f, 0.f, 0.f, 0.f), zz = ww, zc4 = ww;
        if (refresh) {
          zz.x = -s_tab[sid_of(my_sid, 4 * m)];
          zz.y = -s_tab[sid_of(my_sid, 4 * m + 1)];
          zz.z = -s_tab[sid_of(my_sid, 4 * m + 2)];
          zz.w = -s_tab[sid_of(my_sid, 4 * m + 3)];
        }
        for (int q0 = 0; q0 < nm; q0 += BQ) {
          float4 v[BQ];
#pragma unroll
          for (int u = 0; u < BQ; ++u)
            if (q0 + u < nm) v[u] = __ldcg(src + (size_t)cl[q0 + u] * vp4);
#pragma unroll
          for (int u = 0; u < BQ; ++u) {
            if (q0 + u < nm) {
              const int sl = cl[q0 + u];
              const float ds = s_df[sl];
              if (refresh) {
                const float ys = s_yf[sl], yl = s_ylo[sl];
                dot2_add(zz.x, zc4.x, v[u].x, ys, yl);
                dot2_add(zz.y, zc4.y, v[u].y, ys, yl);
                dot2_add(zz.z, zc4.z, v[u].z, ys, yl);
                dot2_add(zz.w, zc4.w, v[u].w, ys, yl);
              }
              ww.x = fmaf(v[u].x, ds, ww.x);
              ww.y = fmaf(v[u].y, ds, ww.y);
              ww.z = fmaf(v[u].z, ds, ww.z);
              ww.w = fmaf(v[u].w, ds, ww.w);
            }
          }
        }
        if (refresh) {
          z[4 * m] = __fadd_rn(zz.x, zc4.x); z[4 * m + 1] = __fadd_rn(zz.y, zc4.y);
          z[4 * m + 2] = __fadd_rn(zz.z, zc4.z); z[4 * m + 3] = __fadd_rn(zz.w, zc4.w);
        }
        w[4 * m] = ww.x; w[4 * m + 1] = ww.y; w[4 * m + 2] = ww.z; w[4 * m + 3] = ww.w;
      }
#pragma unroll
      for (int p = 0; p < 33; ++p) s_rows[tid * 33 + p] = 0.f;
    } else {
      const bool refresh = (it & 15) == 15;  // (iteration 0 starts from a fresh e; the update
                                              // before a refresh forms y as a float pair)
      constexpr int STG = master_pipe_stages(VPT);
      float4 *pipe = (float4 *)s_rows;  // [STG][nthr], slot k of thread t at k*nthr + t
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        const int nm = s_mcnt[m];
        const int *cl = s_mcols + m * N;
        const float *src = a.M + SUB_OFF(m) + 4 * tid;
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f), ww = zz;
#pragma unroll
        for (int k = 0; k < STG; ++k) {
          if (k < nm) cp_async16(pipe + k * nthr + tid, src + (size_t)cl[k] * a.Vpad);
          cp_async_commit();
        }
        if (refresh) {
          float4 zc4 = zz;
          zz.x = -s_tab[sid_of(my_sid, 4 * m)];
          zz.y = -s_tab[sid_of(my_sid, 4 * m + 1)];
          zz.z = -s_tab[sid_of(my_sid, 4 * m + 2)];
          zz.w = -s_tab[sid_of(my_sid, 4 * m + 3)];
          if (XP) {  // T as a float pair
            zc4.x = -s_tablo[sid_of(my_sid, 4 * m)];
            zc4.y = -s_tablo[sid_of(my_sid, 4 * m + 1)];
            zc4.z = -s_tablo[sid_of(my_sid, 4 * m + 2)];
            zc4.w = -s_tablo[sid_of(my_sid, 4 * m + 3)];
          }
          for (int q = 0; q < nm; ++q) {
            cp_async_wait<STG - 1>();
            const int slot = q & (STG - 1);
            const float4 v = pipe[slot * nthr + tid];
            const int sl = cl[q];
            const float ys = s_yf[sl], yl = s_ylo[sl], ds = s_df[sl];
            dot2_add(zz.x, zc4.x, v.x, ys, yl); ww.x = fmaf(v.x, ds, ww.x);
            dot2_add(zz.y, zc4.y, v.y, ys, yl); ww.y = fmaf(v.y, ds, ww.y);
            dot2_add(zz.z, zc4.z, v.z, ys, yl); ww.z = fmaf(v.z, ds, ww.z);
            dot2_add(zz.w, zc4.w, v.w, ys, yl); ww.w = fmaf(v.w, ds, ww.w);
            if (XP) {  // the columns' low parts
              const float4 vl =
                  __ldg((const float4 *)(a.Mlo + SUB_OFF(m) + (size_t)sl * a.Vpad) + tid);
              zc4.x = fmaf(vl.x, ys, zc4.x); ww.x = fmaf(vl.x, ds, ww.x);
              zc4.y = fmaf(vl.y, ys, zc4.y); ww.y = fmaf(vl.y, ds, ww.y);
              zc4.z = fmaf(vl.z, ys, zc4.z); ww.z = fmaf(vl.z, ds, ww.z);
              zc4.w = fmaf(vl.w, ys, zc4.w); ww.w = fmaf(vl.w, ds, ww.w);
            }
            if (q + STG < nm) cp_async16(pipe + slot * nthr + tid, src + (size_t)cl[q + STG] * a.Vpad);
            cp_async_commit();
          }
          if (XP) {
            two_sum(zz.x, zc4.x, z[4 * m], zl[XP ? 4 * m : 0]);
            two_sum(zz.y, zc4.y, z[4 * m + 1], zl[XP ? 4 * m + 1 : 0]);
            two_sum(zz.z, zc4.z, z[4 * m + 2], zl[XP ? 4 * m + 2 : 0]);
            two_sum(zz.w, zc4.w, z[4 * m + 3], zl[XP ? 4 * m + 3 : 0]);
          } else {
            z[4 * m] = __fadd_rn(zz.x, zc4.x); z[4 * m + 1] = __fadd_rn(zz.y, zc4.y);
            z[4 * m + 2] = __fadd_rn(zz.z, zc4.z); z[4 * m + 3] = __fadd_rn(zz.w, zc4.w);
          }
        } else {
          for (int q = 0; q < nm; ++q) {
            cp_async_wait<STG - 1>();
            const int slot = q & (STG - 1);
            const float4 v = pipe[slot * nthr + tid];
            const float ds = s_df[cl[q]];
            ww.x = fmaf(v.x, ds, ww.x);
            ww.y = fmaf(v.y, ds, ww.y);
            ww.z = fmaf(v.z, ds, ww.z);
            ww.w = fmaf(v.w, ds, ww.w);
            if (XP) {  // the columns' low parts
              const float4 vl =
                  __ldg((const float4 *)(a.Mlo + SUB_OFF(m) + (size_t)cl[q] * a.Vpad) + tid);
              ww.x = fmaf(vl.x, ds, ww.x);
              ww.y = fmaf(vl.y, ds, ww.y);
              ww.z = fmaf(vl.z, ds, ww.z);
              ww.w = fmaf(vl.w, ds, ww.w);
            }
            if (q + STG < nm) cp_async16(pipe + slot * nthr + tid, src + (size_t)cl[q + STG] * a.Vpad);
            cp_async_commit();
          }
        }
        w[4 * m] = ww.x; w[4 * m + 1] = ww.y; w[4 * m + 2] = ww.z; w[4 * m + 3] = ww.w;
      }
      cp_async_wait<0>();
      __syncthreads();  // every thread's copies have landed before the rows are reused
#pragma unroll
      for (int p = 0; p < 33; ++p) s_rows[tid * 33 + p] = 0.f;
    }
    if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[2] += c1 - s_clk[4]; s_clk[4] = c1; }

    // ---------------- gradient projection: save the point and take the full
    // step; the next gradient pass evaluates line-search round 0 along d
    if (!NEWTON) {
      for (int s = tid; s < ns; s += nthr) {
        const int k = s_beam[s];
        const double ys = s_y[k];
        s_ysave[k] = ys;
        if (XP) {  // a full step onto the bound lands on 0 exactly; never below it
          const double yn = ys + (double)s_df[s];
          s_y[k] = (yn <= 0.0 || s_d[k] == -ys) ? 0.0 : yn;
        } else {
          s_y[k] = ys + s_d[k];
        }
      }
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        s_zsave[v * nthr + tid] = z[v];
        if (XP) {
          s_zlsave[v * nthr + tid] = zl[XP ? v : 0];
          float sh, se;
          two_sum(z[v], w[v], sh, se);
          two_sum(sh, __fadd_rn(zl[XP ? v : 0], se), z[v], zl[XP ? v : 0]);
        } else {
          z[v] = fmaf(1.f, w[v], z[v]);
        }
      }
      trial = true;
      __syncthreads();
      if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[3] += c1 - s_clk[4]; s_clk[4] = c1; }
      continue;
    }

    // ---------------- exact line search on [0, 1]
    // phi'(t) = phi'(0) + sum_j D_j(t) + 2 gamma G(d) t, phi'(0) = g.d from the
    // reduced gradient; warp 0 keeps the bracket [lo, hi] (phi'(lo) < 0 <
    // phi'(hi)) and threads 0..15 pick the trial points; all CTAs see the
    // same sums and take the same decisions.
    double *s_ls_state = s_sc + 8;  // lo_t lo_f lo_h hi_t hi_f hi_h t done
    for (int r = 0; r < LS_ROUNDS && s_ls_state[7] == 0.0; ++r) {
      ls_points(r, s_t, s_ls_state);
      __syncthreads();
      ++nsync;
      double lsv = 0.0;
      if (!ls_round<VPT>(a, [&](int q) { return z[q]; }, w, my_sid, s_tab, s_t, s_rows, s_ls, s_res,
                         s_i, ls_parity, stride, lsv, timer ? s_clk + 5 : nullptr)) {
        alive = false;
        break;
      }
      ls_parity ^= 1;
      if (warp == 0) ls_bracket(r, lsv, s_t, s_ls_state, s_sc, nwarp, a.gamma);
      __syncthreads();
    }
    if (!alive) break;
    const double t = s_ls_state[6] >= 0.0 ? s_ls_state[6] : s_ls_state[0];
    if (timer) { const unsigned long long c1 = vmat_globaltimer(); s_clk[3] += c1 - s_clk[4]; s_clk[4] = c1; }
    if (t <= 0.0) { status = VMAT_ENOTCONV; break; }

    // ---------------- update
    // (y as a float pair is read only by the refresh of e in the next
    // direction pass, so it is formed only before such an iteration)
    const bool pair_next = ((it + 1) & 15) == 15;
    const float tf = (float)t;
    for (int s = tid; s < ns; s += nthr) {
      const int k = s_beam[s];
      // extended precision: y moves by exactly the FP32 step and direction
      // that the excess update below applies (both factors are floats, so
      // their product is exact in FP64)
      const double dy = XP ? (double)tf * (double)s_df[s] : t * s_d[k];
      s_dy[s] = dy;
      if (XP) {  // a full step onto the bound lands on 0 exactly; never below it
        const double yn = s_y[k] + dy;
        s_y[k] = (yn <= 0.0 || (t == 1.0 && s_d[k] == -s_y[k])) ? 0.0 : yn;
      } else {
        s_y[k] = NEWTON ? fmax(s_y[k] + dy, 0.0) : s_y[k] + dy;  // ratio test in FP64: clamp -0
      }
      if (pair_next) {
        s_yf[s] = (float)s_y[k];
        s_ylo[s] = (float)(s_y[k] - (double)s_yf[s]);
      }
    }
    if (XP) {  // (z, zl) += tf w, the product's rounding error from an FMA
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const float p = __fmul_rn(tf, w[v]), pe = __fmaf_rn(tf, w[v], -p);
        float sh, se;
        two_sum(z[v], p, sh, se);
        two_sum(sh, __fadd_rn(zl[XP ? v : 0], __fadd_rn(se, pe)), z[v], zl[XP ? v : 0]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < VPT; ++v) z[v] = fmaf(tf, w[v], z[v]);
    }
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

  // ---------------- final dose, derivative and cost at the solution, from
  // the carried excess (recomputed from y at the start and every 16th
  // iteration, updated exactly along every step): z = e + T
  __syncthreads();
  double cst = 0.0;
#pragma unroll
  for (int m = 0; m < NG; ++m) {
    float zo[4], fo[4], flo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = 4 * m + q, id = sid_of(my_sid, v);
      fo[q] = dF_e(z[v], s_tab[256 + id], s_tab[512 + id]);
      if (XP) {  // z = (eh + el) + T with T = T_hi + T_lo, in FP64; F' as a pair
        dF_pair(z[v], zl[XP ? v : 0], s_tab[256 + id], s_tablo[256 + id], s_tab[512 + id],
                s_tablo[512 + id], fo[q], flo[q]);
        const double zd = ((double)z[v] + (double)zl[XP ? v : 0]) + ((double)s_tab[id] + (double)s_tablo[id]);
        zo[q] = (float)zd;
        cst += vmat_F(zd, a.tabd[id], a.tabd[256 + id], a.tabd[512 + id]);
      } else {
        zo[q] = __fadd_rn(z[v], s_tab[id]);
        // cost against the FP64 threshold: z = e + T in the FP32 threshold, exactly
        cst += vmat_F((double)z[v] + (double)s_tab[id], a.tabd[id], a.tabd[256 + id], a.tabd[512 + id]);
      }
    }
    const size_t off = SUB_OFF(m) + 4 * tid;
    *(float4 *)(a.z_out + off) = make_float4(zo[0], zo[1], zo[2], zo[3]);
    *(float4 *)(a.fp_out + off) = make_float4(fo[0], fo[1], fo[2], fo[3]);
    if (XP) *(float4 *)(a.fp_out_lo + off) = make_float4(flo[0], flo[1], flo[2], flo[3]);
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
          a.stats[0] += (double)s_clk[0];
          a.stats[1] += (double)s_clk[1];
          a.stats[2] += (double)s_clk[2];
          a.stats[3] += (double)s_clk[3];
          a.stats[4] += (double)nsync;
          a.stats[5] += (double)it;
          a.stats[6] += (double)s_clk[5];
          a.stats[7] += (double)n_partial;
        }
      }
    }
    for (int k = tid; k < N; k += nthr) a.y[k] = s_y[k];
  }
}

// ---------------------------------------------------------------- launch
static size_t master_smem_bytes(int N, int nthr, int vpt, bool newton, bool xp) {
  const size_t ng = vpt / 4;
  size_t b = (size_t)(8 * N + 64 + 32 + MAX_WARPS * 32 + ((N + 1) & ~1)) * 8 +  // doubles: y d g gold dy
                                                                                 // igl igr slot sc res ysave
             (size_t)(2 * ((N + 1) & ~1) + ((((N + 1) & ~1) + 3) & ~3) + 768 + LS_POINTS + MAX_WARPS * 32) * 4 +
             (size_t)nthr * vpt * 4 +                          // F' tile
             (size_t)master_rows_len(N, nthr, vpt, newton) * 4 +  // line-search rows, pipeline, Newton
             (size_t)N * ng * 4 +                              // pair partials
             (size_t)(8 + 3 * N + 1 + N * ng) * 4 +            // i beam mask pst pair
             (size_t)(8 + N * ng) * 4;                          // per-subtile column lists
  if (newton) b += (size_t)(2 * N + 8 + ng * N) * 4 + (size_t)(2 * N + 2 * (N + 1)) * 4;
  if (xp) b += 16 + (size_t)nthr * vpt * 4 + 768 * 4 + (size_t)N * ng * 4;  // alignment, low parts:
                                                                            // F', T/alpha/beta, pairs
  if (!newton) b += 16 + (size_t)nthr * vpt * 4 * (xp ? 2 : 1);  // excess at the accepted point
  return b + 16;
}

// The master kernel for a launch shape and variant; nullptr where the
// variant is not built (extended precision stops at 16 voxels per thread).
// The FP32 gradient projection at 4 or 8 voxels per thread has a build for
// CTAs of at most 384 threads.
static const void *master_fn(int vpt, bool newton, bool xp, int nthr) {
  constexpr int M = master_max_threads(0);
  if (!newton && !xp && nthr <= 384) {
    if (vpt == 4) return (const void *)k_master<4, false, false, 384>;
    if (vpt == 8) return (const void *)k_master<8, false, false, 384>;
  }
#define VMAT_MFN(V)                                                                              \
  if (vpt == V)                                                                                 \
    return newton ? (xp ? (const void *)k_master<V, true, true, M> : (const void *)k_master<V, true, false, M>) \
                  : (xp ? (const void *)k_master<V, false, true, M> : (const void *)k_master<V, false, false, M>);
  VMAT_MFN(4)
  VMAT_MFN(8)
  VMAT_MFN(16)
#undef VMAT_MFN
  if (vpt == 32 && !xp)
    return newton ? (const void *)k_master<32, true, false, M> : (const void *)k_master<32, false, false, M>;
  return nullptr;
}

static cudaError_t master_occupancy_any(int vpt, bool newton, bool xp, int nthr, size_t smem, int *nb) {
  const void *fn = master_fn(vpt, newton, xp, nthr);
  if (!fn) {
    *nb = 0;
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, fn, nthr, smem);
}

// Launch shape: the fewest voxels per thread (4, 8, 16, 32) that fit the
// SMs with 512-thread CTAs, then threads per CTA chosen so that the CTAs
// cover the voxels with one CTA on (nearly) every SM, but never fewer than
// 256 threads (small problems then take fewer CTAs: 8 warps per CTA hide the
// pass latencies that 2-5 warps do not) and 512 from 16 voxels per thread on.
// The column passes are bound per SM (each warp's pairs in series, the
// direction pass's copies and shared-memory traffic), so spreading the voxels
// over all SMs shortens them more than the extra CTA rows lengthen the
// cross-CTA sums (prostate: 145 CTAs of 384 threads, 25.4 us per iteration
// against 28.7 us with 109 CTAs of 512); more voxels per thread (16, 32)
// lengthen every per-voxel pass.
vmat_status vmat_configure_master(vmat_ctx *ctx) {
  const int64_t Va = ctx->Va > 0 ? ctx->Va : 1;
  const int sms = ctx->sm_budget > 0 && ctx->sm_budget < ctx->num_sms ? ctx->sm_budget : ctx->num_sms;
  const int target = sms;
  int vpt = 4;
  for (; vpt <= 32; vpt *= 2) {
    const int64_t cap = (int64_t)vpt * master_max_threads(vpt);
    if ((Va + cap - 1) / cap <= sms) break;
  }
  if (vpt > 32) return vmat_fail(ctx, VMAT_EINVAL, "too many active voxels for the master kernel");
  const int64_t per = (Va + (int64_t)vpt * target - 1) / ((int64_t)vpt * target);
  int nthr = (int)(((per + 31) / 32) * 32);
  if (nthr < 256) nthr = 256;  // small problems: fewer CTAs of at least 8 warps
  if (nthr > master_max_threads(vpt) || vpt >= 16)  // at 16+ voxels per thread every warp counts
    nthr = master_max_threads(vpt);
  int64_t chunk = (int64_t)nthr * vpt;
  int grid = (int)((Va + chunk - 1) / chunk);
  const bool xp = ctx->master_xp != 0;
  if (xp && !master_fn(vpt, false, true, nthr))
    return vmat_fail(ctx, VMAT_EINVAL,
                     "extended-precision master: at most 16 active voxels per thread (%lld active "
                     "voxels need %d)", (long long)Va, vpt);
  size_t smem = master_smem_bytes(ctx->N, nthr, vpt, false, xp);
  size_t smem_pn = master_smem_bytes(ctx->N, nthr, vpt, true, xp);
  int nb = 0;
  cudaError_t e = master_occupancy_any(vpt, false, xp, nthr, smem, &nb);
  if (e != cudaSuccess) return vmat_cuda_fail(ctx, e, "master occupancy");
  if (nb < 1 || grid > nb * ctx->num_sms)
    return vmat_fail(ctx, VMAT_EINVAL, "master kernel cannot be co-resident (%d blocks/SM)", nb);
  if (ctx->master_method == VMAT_MASTER_PROJECTED_NEWTON) {
    int optin = 0;
    VMAT_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (smem_pn > (size_t)optin)
      return vmat_fail(ctx, VMAT_EINVAL,
                       "projected-Newton master needs %zu B of shared memory per CTA (%d beams); "
                       "the device allows %d", smem_pn, ctx->N, optin);
    e = master_occupancy_any(vpt, true, xp, nthr, smem_pn, &nb);
    if (e != cudaSuccess) return vmat_cuda_fail(ctx, e, "projected-Newton master occupancy");
    if (nb < 1 || grid > nb * ctx->num_sms)
      return vmat_fail(ctx, VMAT_EINVAL, "projected-Newton master cannot be co-resident");
  }
  ctx->master_vpt = vpt;
  ctx->master_block = nthr;
  ctx->master_grid = grid;
  ctx->master_smem = smem;
  ctx->master_smem_pn = smem_pn;
  ctx->Vpad = (int32_t)(grid * chunk);
  return VMAT_OK;
}

// doubles: per-CTA partial rows [grid][N + PART_EXTRA], then (16-byte
// aligned) the per-CTA gradient partial rows [2 * grid][(N+3)&~3] floats
int64_t vmat_master_scratch(int grid, int N) {
  // the gradient rows twice: value rows, then (extended precision) their low parts
  // (two sets of them: one per parity of the gradient pass)
  return (int64_t)grid * (N + PART_EXTRA) + 2 + ((int64_t)4 * grid * ((N + 4) & ~3) + 1) / 2;
}

int64_t vmat_hessian_len(int N) { return (int64_t)(N + 1) * (N + 2) / 2; }

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
  {
    const uintptr_t gp = (uintptr_t)(ctx->red + (size_t)ctx->master_grid * (ctx->N + PART_EXTRA));
    a.gpart = (float *)((gp + 15) & ~(uintptr_t)15);
  }
  a.bar = ctx->bar;
  a.dstatus = ctx->dstatus;
  a.z_out = ctx->zact;
  a.fp_out = ctx->fpact;
  a.Mlo = ctx->master_xp ? ctx->Mlo : nullptr;
  a.fp_out_lo = ctx->master_xp ? ctx->fplo : nullptr;
  if (ctx->master_xp && (!ctx->Mlo || !ctx->fplo))
    return vmat_fail(ctx, VMAT_ESTATE, "extended-precision buffers missing");
  a.out = ctx->mout;
  a.stats = ctx->mstats;
  const bool pn = ctx->master_method == VMAT_MASTER_PROJECTED_NEWTON;
  if (pn && !ctx->hbuf) return vmat_fail(ctx, VMAT_ESTATE, "projected-Newton scratch missing");
  a.hpart = pn ? ctx->hbuf : nullptr;
  a.hred = pn ? ctx->hbuf + (size_t)ctx->master_grid * vmat_hessian_len(ctx->N) : nullptr;
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
  const void *fn = master_fn(ctx->master_vpt, pn, ctx->master_xp != 0, ctx->master_block);
  if (!fn) return vmat_fail(ctx, VMAT_EINVAL, "no master kernel for this launch shape and precision");
  const size_t smem = pn ? ctx->master_smem_pn : ctx->master_smem;
  // the dynamic shared-memory limit is a per-kernel, process-wide attribute:
  // set it for this context's launch (another context may have lowered it)
  VMAT_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = smem;
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

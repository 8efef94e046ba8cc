// Pricing subproblem (Sec. 2.2) and aperture columns.
//
// k_pricing: one CTA per beam without an aperture.  Thread 0 finds the
// nearest beams with apertures on each side (ring or path order); each leaf
// row gets limits l in [Llo, Lhi], r in [Rlo, Rhi] (a leaf may move at most
// s columns per angle step from the neighbour's), then ONE left-to-right
// pass over its C beamlets: P[0] = 0, P[c+1] = P[c] + g_c in FP32; for each
// r the best left leaf is the feasible l of largest P[l] (ties: largest l);
// the row keeps the least P[r] - P[l], then the shortest interval, then the
// smallest l.  The aperture price sums the row values in FP64, row order;
// with smoothing-aware pricing it then adds gamma * dG/dy_k of Eq. 2 at the
// current y (the exact reduced cost of the new column, see smoothing_slope).
// A row is tiny (C <= 128) and its sequential order fixes ties exactly, so
// the scan stays sequential per thread; all rows of a beam run in parallel.
// k_select: least aperture price over free beams (ties: lowest beam), and
// the least price of the others.
// k_aperture: M[:, slot] = sum over open beamlets of the chosen aperture of
// D_i,: (in FP32; with the extended-precision master in FP64 and kept as a
// float pair), by one thread per voxel over its voxel-major row (sorted by
// beamlet, so the beam's entries are one contiguous run found by bisection).
#include <math.h>

#include "vmat_internal.cuh"

// dG/dy_k of Eq. 2 at y: the pair (k-1, k) contributes 2 (y_k - y_{k-1}) / gap,
// the pair (k, k+1) -2 (y_{k+1} - y_k) / gap (on a ring the wrap pair joins
// beams N-1 and 0, gap theta_0 + 360 - theta_{N-1}); the two are combined as
// (0 + left) - right, each rounded once, FP64.  A beam without an aperture
// has y_k = 0, so this is -2 times its neighbours' intensities over the gaps.
__device__ __forceinline__ double smoothing_slope(const double *__restrict__ y,
                                                  const double *__restrict__ theta, int N,
                                                  int cyclic, int k) {
  if (N < 2) return 0.0;
  double out = 0.0;
  if (k > 0 || cyclic) {
    const int a = k > 0 ? k - 1 : N - 1;
    const double gap = a + 1 < N ? theta[a + 1] - theta[a] : theta[0] + 360.0 - theta[N - 1];
    out = __dadd_rn(out, __ddiv_rn(__dmul_rn(2.0, __dsub_rn(y[k], y[a])), gap));
  }
  if (k < N - 1 || cyclic) {
    const int b = k + 1 < N ? k + 1 : 0;
    const double gap = k + 1 < N ? theta[k + 1] - theta[k] : theta[0] + 360.0 - theta[N - 1];
    out = __dsub_rn(out, __ddiv_rn(__dmul_rn(2.0, __dsub_rn(y[b], y[k])), gap));
  }
  return out;
}

__global__ void __launch_bounds__(128) k_pricing(const float *__restrict__ g,
                                                 const uint8_t *__restrict__ occ,
                                                 const int16_t *__restrict__ lleaf,
                                                 const int16_t *__restrict__ rleaf, int N, int R,
                                                 int C, int s, int cyclic, double *ap_price,
                                                 int16_t *ap_l, int16_t *ap_r,
                                                 const double *__restrict__ y,
                                                 const double *__restrict__ theta, double gamma,
                                                 int smooth) {
  const int k = blockIdx.x;
  __shared__ int nb[2], dist[2];
  __shared__ float rowv[VMAT_MAX_ROWS];
  __shared__ int rowok[VMAT_MAX_ROWS];
  if (occ[k]) {
    if (threadIdx.x == 0) ap_price[k] = INFINITY;
    return;
  }
  if (threadIdx.x == 0) {
    for (int side = 0; side < 2; ++side) {
      nb[side] = -1;
      dist[side] = 0;
      const int step = side == 0 ? -1 : 1;
      for (int d = 1; d < N; ++d) {
        int q = k + step * d;
        if (cyclic) q = ((q % N) + N) % N;
        else if (q < 0 || q >= N) break;
        if (occ[q]) {
          nb[side] = q;
          dist[side] = d;
          break;
        }
      }
    }
  }
  __syncthreads();
  for (int row = threadIdx.x; row < R; row += blockDim.x) {
    int llo = 0, lhi = C, rlo = 0, rhi = C;
    for (int side = 0; side < 2; ++side) {
      if (nb[side] < 0) continue;
      const int m = s * dist[side];
      const int ln = lleaf[nb[side] * R + row], rn = rleaf[nb[side] * R + row];
      llo = max(llo, ln - m);
      lhi = min(lhi, ln + m);
      rlo = max(rlo, rn - m);
      rhi = min(rhi, rn + m);
    }
    const float *gr = g + ((int64_t)k * R + row) * C;
    float P = 0.f, Pbest = 0.f, bv = 0.f;
    int lbest = -1, bl = 0, br = 0, found = 0;
    for (int c = 0; c <= C; ++c) {
      if (c > 0) P = __fadd_rn(P, gr[c - 1]);
      if (c >= llo && c <= lhi && (lbest < 0 || P >= Pbest)) {
        Pbest = P;
        lbest = c;
      }
      if (c >= rlo && c <= rhi && lbest >= 0) {
        const float v = __fsub_rn(P, Pbest);
        const int len = c - lbest;
        if (!found || v < bv || (v == bv && len < br - bl)) {
          bv = v;
          bl = lbest;
          br = c;
          found = 1;
        }
      }
    }
    rowv[row] = bv;
    rowok[row] = found;
    ap_l[k * R + row] = (int16_t)bl;
    ap_r[k * R + row] = (int16_t)br;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0;
    int ok = 1;
    for (int row = 0; row < R; ++row) {
      ok &= rowok[row];
      p += (double)rowv[row];
    }
    if (smooth) p = __dadd_rn(p, __dmul_rn(smoothing_slope(y, theta, N, cyclic, k), gamma));
    ap_price[k] = ok ? p : NAN;
  }
}

// Writes the selection; when rec_* are given, also the per-iteration record.
__global__ void __launch_bounds__(256) k_select(const double *__restrict__ ap_price,
                                                const uint8_t *__restrict__ occ,
                                                const int16_t *__restrict__ ap_l,
                                                const int16_t *__restrict__ ap_r, int N, int R,
                                                SelRec *sel, int16_t *sel_l, int16_t *sel_r,
                                                int32_t *rec_k, double *rec_p, double *rec_p2) {
  __shared__ double sp[256];
  __shared__ int sk[256], sbad[256];
  __shared__ int kbest;
  const int t = threadIdx.x;
  double bp = INFINITY;
  int bk = -1, bad = 0;
  for (int k = t; k < N; k += blockDim.x) {
    if (occ[k]) continue;
    double p = ap_price[k];
    if (isnan(p)) { bad = 1; continue; }
    if (bk < 0 || p < bp) { bp = p; bk = k; }  // k ascending per thread: ties keep the lower
  }
  sp[t] = bp; sk[t] = bk; sbad[t] = bad;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (t < o) {
      double p2 = sp[t + o];
      int k2 = sk[t + o];
      if (k2 >= 0 && (sk[t] < 0 || p2 < sp[t] || (p2 == sp[t] && k2 < sk[t]))) {
        sp[t] = p2;
        sk[t] = k2;
      }
      sbad[t] |= sbad[t + o];
    }
    __syncthreads();
  }
  if (t == 0) kbest = sk[0];
  const int anybad = sbad[0];
  __syncthreads();
  const int kb = kbest;
  // least price among the other free beams
  double q = INFINITY;
  for (int k = t; k < N; k += blockDim.x) {
    if (occ[k] || k == kb) continue;
    double p = ap_price[k];
    if (!isnan(p) && p < q) q = p;
  }
  __syncthreads();
  sp[t] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (t < o) sp[t] = fmin(sp[t], sp[t + o]);
    __syncthreads();
  }
  if (t == 0) {
    SelRec r;
    r.k = kb;
    r.status = (kb < 0 || anybad) ? (int)VMAT_ESTATE : 0;
    r.p = kb >= 0 ? ap_price[kb] : INFINITY;
    r.p2 = sp[0];
    *sel = r;
    if (rec_k) *rec_k = kb;
    if (rec_p) *rec_p = r.p;
    if (rec_p2) *rec_p2 = r.p2;
  }
  if (kb >= 0)
    for (int row = t; row < R; row += blockDim.x) {
      sel_l[row] = ap_l[kb * R + row];
      sel_r[row] = ap_r[kb * R + row];
    }
}

vmat_status vmat_launch_pricing_rec(vmat_ctx *ctx, const float *g, int32_t *rec_k, double *rec_p,
                                    double *rec_p2) {
  k_pricing<<<ctx->N, 64, 0, ctx->stream>>>(g, ctx->occ, ctx->lleaf, ctx->rleaf, ctx->N, ctx->R,
                                            ctx->C, ctx->step, ctx->cyclic, ctx->ap_price,
                                            ctx->ap_l, ctx->ap_r, ctx->y, ctx->theta, ctx->gamma,
                                            ctx->price_smoothing);
  k_select<<<1, 256, 0, ctx->stream>>>(ctx->ap_price, ctx->occ, ctx->ap_l, ctx->ap_r, ctx->N,
                                       ctx->R, ctx->sel, ctx->sel_l, ctx->sel_r, rec_k, rec_p,
                                       rec_p2);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 2;
  return VMAT_OK;
}

vmat_status vmat_launch_pricing(vmat_ctx *ctx, const float *g) {
  return vmat_launch_pricing_rec(ctx, g, nullptr, nullptr, nullptr);
}

// replace the selection by a forced aperture (replay)
__global__ void k_force(const int32_t *fk, const int16_t *fl, const int16_t *fr, int t, int R,
                        SelRec *sel, int16_t *sel_l, int16_t *sel_r) {
  if (threadIdx.x == 0) {
    sel->k = fk[t];
    sel->status = 0;
  }
  for (int row = threadIdx.x; row < R; row += blockDim.x) {
    sel_l[row] = fl[(int64_t)t * R + row];
    sel_r[row] = fr[(int64_t)t * R + row];
  }
}

vmat_status vmat_launch_force(vmat_ctx *ctx, const int32_t *fk, const int16_t *fl,
                              const int16_t *fr, int t) {
  k_force<<<1, 128, 0, ctx->stream>>>(fk, fl, fr, t, ctx->R, ctx->sel, ctx->sel_l, ctx->sel_r);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  return VMAT_OK;
}

// ---------------------------------------------------------------- aperture column
template <typename TV>
__global__ void __launch_bounds__(256) k_aperture(const int64_t *__restrict__ ptr,
                                                  const int32_t *__restrict__ col,
                                                  const TV *__restrict__ val,
                                                  const float *__restrict__ scale, int use_scale,
                                                  int32_t Va, int32_t Vpad, int R, int C,
                                                  const SelRec *__restrict__ sel,
                                                  const int16_t *__restrict__ sl,
                                                  const int16_t *__restrict__ sr,
                                                  float *__restrict__ Mcol,
                                                  float *__restrict__ Mcol_lo, int tile,
                                                  int32_t *__restrict__ tflag,
                                                  const uint16_t *__restrict__ boff, int N1) {
  __shared__ int16_t L[VMAT_MAX_ROWS], Rr[VMAT_MAX_ROWS];
  __shared__ int sk;
  if (threadIdx.x == 0) sk = sel->status == 0 ? sel->k : -1;
  for (int row = threadIdx.x; row < R; row += blockDim.x) {
    L[row] = sl[row];
    Rr[row] = sr[row];
  }
  __syncthreads();
  const int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Vpad) return;
  const int k = sk;
  if (a >= Va || k < 0) {
    Mcol[a] = 0.f;
    if (Mcol_lo) Mcol_lo[a] = 0.f;
    return;  // padding and failed selections leave the tile flags alone
  }
  const int32_t RC = R * C, lo = k * RC, hi = lo + RC;
  int64_t b = ptr[a], end;
  if (boff) {  // the row's entries of beam k, from the offsets table
    const uint16_t *o = boff + (size_t)a * N1 + k;
    end = b + o[1];
    b += o[0];
  } else {
    int64_t e = ptr[a + 1];
    end = e;
    while (b < e) {  // first entry with beamlet >= lo
      int64_t m = (b + e) >> 1;
      if (col[m] < lo) b = m + 1;
      else e = m;
    }
  }
  float accf = 0.f;   // FP32 sum in beamlet order
  double acc = 0.0;   // extended precision: FP64 sum, kept as a float pair
  for (int64_t q = b; q < end; ++q) {
    const int32_t i = col[q];
    if (i >= hi) break;
    const int32_t rc = i - lo, row = rc / C, c = rc - row * C;
    if (c >= L[row] && c < Rr[row]) {
      const float v = vmat_ld(val, q);
      if (Mcol_lo) acc += use_scale ? (double)v * (double)scale[i] : (double)v;
      else accf += use_scale ? v * scale[i] : v;
    }
  }
  if (Mcol_lo) {
    accf = (float)acc;
    Mcol_lo[a] = (float)(acc - (double)accf);
  }
  Mcol[a] = accf;
  // mark the master subtile holding voxel a as nonzero for this column
  // (subtiles are whole multiples of 128 voxels: a warp never straddles two)
  if (__any_sync(__activemask(), accf != 0.f) && (threadIdx.x & 31) == __ffs(__activemask()) - 1)
    atomicOr(tflag + a / tile, 1);
}

// Offsets of each beam's entries in each voxel-major row: boff[a][k] = the
// number of entries of row a with beamlet < k * RC (k = 0..N; rows are sorted
// by beamlet).  One warp per row; entry e writes the offsets of the beams
// from the previous entry's beam (exclusive) to its own.  Rows longer than
// 65,535 entries do not fit and set *overflow.
__global__ void __launch_bounds__(256) k_beam_offsets(const int64_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ col, int32_t Va,
                                                      int N, unsigned long long rc_magic,
                                                      uint16_t *__restrict__ boff, int *overflow) {
  const int lane = threadIdx.x & 31;
  const int32_t a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a >= Va) return;
  const int64_t s = ptr[a], t = ptr[a + 1];
  if (t - s > 65535) {
    if (lane == 0) atomicExch(overflow, 1);
    return;
  }
  uint16_t *o = boff + (size_t)a * (N + 1);
  for (int64_t e = s + lane; e < t; e += 32) {
    const int bcur = (int)(((unsigned long long)(unsigned)col[e] * rc_magic) >> 40);
    const int bprev = e == s ? -1 : (int)(((unsigned long long)(unsigned)col[e - 1] * rc_magic) >> 40);
    for (int k = bprev + 1; k <= bcur; ++k) o[k] = (uint16_t)(e - s);
  }
  if (lane == 0) {
    const int blast = t > s ? (int)(((unsigned long long)(unsigned)col[t - 1] * rc_magic) >> 40) : -1;
    for (int k = blast + 1; k <= N; ++k) o[k] = (uint16_t)(t - s);
  }
}

vmat_status vmat_build_beam_offsets(vmat_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  const int RC = ctx->R * ctx->C;
  const unsigned long long magic = ((1ull << 40) + (unsigned long long)RC - 1) / (unsigned long long)RC;
  int *flag = (int *)(ctx->pstat + 5);  // the live-row count word, free outside a price call
  VMAT_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->vm_boff, (size_t)(ctx->Va > 0 ? ctx->Va : 1) * (ctx->N + 1)));
  if (ctx->Va > 0) {
    k_beam_offsets<<<(unsigned)((ctx->Va + 7) / 8), 256, 0, st>>>(ctx->vm_ptr, ctx->vm_col, ctx->Va, ctx->N,
                                                                  magic, ctx->vm_boff, flag);
    ctx->n_launches += 1;
  }
  int h = 0;
  VMAT_CUDA(ctx, cudaGetLastError());
  VMAT_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  if (h) {  // a row too long for 16-bit offsets: the aperture kernel bisects instead
    cudaFree(ctx->vm_boff);
    ctx->device_bytes -= (int64_t)((size_t)ctx->Va * (ctx->N + 1) * sizeof(uint16_t));
    ctx->vm_boff = nullptr;
  }
  return VMAT_OK;
}

// commit the selected aperture as plan column `slot`
__global__ void k_commit(const SelRec *sel, const int16_t *sl, const int16_t *sr, int R, int slot,
                         uint8_t *occ, int16_t *lleaf, int16_t *rleaf, int32_t *slot_beam,
                         double *y, int *dstatus, const int32_t *tf, int nsub,
                         int32_t *rec_subtiles) {
  if (rec_subtiles) {  // nonzero subtiles of the new column
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int q = threadIdx.x; q < nsub; q += blockDim.x) c += tf[q] != 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *rec_subtiles = cnt;
  }
  const int k = sel->status == 0 ? sel->k : -1;
  if (k < 0) {
    if (threadIdx.x == 0) atomicCAS(dstatus, 0, (int)VMAT_ESTATE);
    return;
  }
  for (int row = threadIdx.x; row < R; row += blockDim.x) {
    lleaf[k * R + row] = sl[row];
    rleaf[k * R + row] = sr[row];
  }
  if (threadIdx.x == 0) {
    occ[k] = 1;
    slot_beam[slot] = k;
    y[k] = 0.0;
  }
}

vmat_status vmat_launch_add_column(vmat_ctx *ctx, int slot, int32_t *rec_subtiles) {
  cudaStream_t st = ctx->stream;
  float *Mcol = ctx->M + (size_t)slot * ctx->Vpad;
  float *Mcol_lo = ctx->Mlo ? ctx->Mlo + (size_t)slot * ctx->Vpad : nullptr;
  const int nsub = ctx->master_grid * (ctx->master_vpt / 4);
  int32_t *tf = ctx->tflag + (size_t)slot * nsub;
  const int tile = ctx->master_block * 4;  // master subtile
  VMAT_CUDA(ctx, cudaMemsetAsync(tf, 0, (size_t)nsub * 4, st));
  unsigned nb = (unsigned)((ctx->Vpad + 255) / 256);
  int us = ctx->dt != VMAT_F32;
#define VMAT_AP_ARGS                                                                              \
  ctx->vm_ptr, ctx->vm_col, (const TV *)ctx->vm_val, ctx->scale, us, ctx->Va, ctx->Vpad, ctx->R, \
      ctx->C, ctx->sel, ctx->sel_l, ctx->sel_r, Mcol, Mcol_lo, tile, tf, ctx->vm_boff, ctx->N + 1
  if (ctx->dt == VMAT_F32) {
    typedef float TV;
    k_aperture<TV><<<nb, 256, 0, st>>>(VMAT_AP_ARGS);
  } else if (ctx->dt == VMAT_F16) {
    typedef __half TV;
    k_aperture<TV><<<nb, 256, 0, st>>>(VMAT_AP_ARGS);
  } else {
    typedef __nv_bfloat16 TV;
    k_aperture<TV><<<nb, 256, 0, st>>>(VMAT_AP_ARGS);
  }
#undef VMAT_AP_ARGS
  k_commit<<<1, 128, 0, st>>>(ctx->sel, ctx->sel_l, ctx->sel_r, ctx->R, slot, ctx->occ, ctx->lleaf,
                              ctx->rleaf, ctx->slot_beam, ctx->y, ctx->dstatus, tf, nsub,
                              rec_subtiles);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 2;
  return VMAT_OK;
}

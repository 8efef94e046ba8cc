// Sparse products with D (Sec. 2.1 dose model, Sec. 2.2 prices).
//
//   price  g_i = s_i * sum_j Dhat_ij f_j     beamlet-major CSR, warp per row
//   dose   z_j = sum_i Dhat_ij (s_i x_i)     voxel-major CSR, warp per row,
//          fused epilogue: F'(z_j) and the FP64 cost sum_j F(z_j) (Eq. 1)
//   batched forms over 32 fluence vectors (lane = vector) for the
//   differentiable forward and its adjoint, on row tiles of D (tiles.cu).
// D is streamed once per call (16-byte loads, evict-first); the dense vector
// that is gathered (f or x, at most a few MB) stays resident in L2.
// Dhat = D for FP32 storage; F16/BF16 store D_ij / s_i.
//
// Prices from the live voxels.  Eq. 1 is one-sided: F'(z_j) = 0 wherever a
// voxel meets its threshold from the allowed side, which at a master
// solution holds for all but ~1-2% of the voxels (the target and the few
// organ or tissue voxels above their thresholds).  g = D F' then only needs
// the voxel-major rows of the voxels with F'_j != 0: each entry D_ij F'_j
// (an exact FP64 product of two floats) is rounded once to a fixed-point
// grid of step 2^-S and added to beamlet i's 64-bit integer accumulator.
// Integer addition is associative, so the sums do not depend on the order
// in which the live rows' entries arrive (deterministic, although the adds
// are atomic), and S is chosen per call from max|F'| and the largest row sum
// of D so that no partial sum can overflow: every price carries an absolute
// error below (entries of its row) x 2^-(S+1) ~ 1e-15 of that bound, below
// the FP32 rounding of the result.  When the live rows hold more than 1/16
// of D's entries the beamlet-major row products run instead.
#include <algorithm>

#include "vmat_internal.cuh"

#define WARPS_PER_BLOCK 8

template <typename TV>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ float4 ld(const float *p) { return __ldcs((const float4 *)p); }
};
template <>
struct Vec4<__half> {
  static __device__ __forceinline__ float4 ld(const __half *p) {
    uint2 u = __ldcs((const uint2 *)p);
    __half2 a = *(__half2 *)&u.x, b = *(__half2 *)&u.y;
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
};
template <>
struct Vec4<__nv_bfloat16> {
  static __device__ __forceinline__ float4 ld(const __nv_bfloat16 *p) {
    uint2 u = __ldcs((const uint2 *)p);
    __nv_bfloat162 a = *(__nv_bfloat162 *)&u.x, b = *(__nv_bfloat162 *)&u.y;
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
};

__device__ __forceinline__ float ld_stream(const float *p, int64_t e) { return __ldcs(p + e); }
__device__ __forceinline__ float ld_stream(const __half *p, int64_t e) { return __half2float(p[e]); }
__device__ __forceinline__ float ld_stream(const __nv_bfloat16 *p, int64_t e) {
  return __bfloat162float(p[e]);
}

// sum over entries [e0, e1) of val[e] * vec[col[e]] by one warp (lane partials)
template <typename TV>
__device__ __forceinline__ float warp_row_dot(const int32_t *__restrict__ col,
                                              const TV *__restrict__ val,
                                              const float *__restrict__ vec, int64_t e0, int64_t e1,
                                              int lane) {
  float acc = 0.f;
  int64_t ea = (e0 + 3) & ~(int64_t)3;
  if (ea > e1) ea = e1;
  if (e0 + lane < ea) acc = ld_stream(val, e0 + lane) * __ldg(vec + __ldcs(col + e0 + lane));
  const int64_t eb = ea + ((e1 - ea) & ~(int64_t)3);
  for (int64_t e = ea + 4 * lane; e < eb; e += 128) {
    int4 c = __ldcs((const int4 *)(col + e));
    float4 v = Vec4<TV>::ld(val + e);
    acc = fmaf(v.x, __ldg(vec + c.x), acc);
    acc = fmaf(v.y, __ldg(vec + c.y), acc);
    acc = fmaf(v.z, __ldg(vec + c.z), acc);
    acc = fmaf(v.w, __ldg(vec + c.w), acc);
  }
  if (eb + lane < e1) acc = fmaf(ld_stream(val, eb + lane), __ldg(vec + __ldcs(col + eb + lane)), acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// ---------------------------------------------------------------- price
// mode 0: all beams; 1: beams with mask[k] != 0; 2: beams with mask[k] == 0

// Extended precision (the master's F' as the pair f + flo): g_i = s_i *
// sum_j Dhat_ij (f_j + flo_j) accumulated in FP64, one warp per row, lanes
// combined in a fixed order; g is rounded to FP32 once.
template <typename TV>
__global__ void __launch_bounds__(256) k_price_xp(const int64_t *__restrict__ ptr,
                                                  const int32_t *__restrict__ col,
                                                  const TV *__restrict__ val,
                                                  const float *__restrict__ scale, int use_scale,
                                                  const float *__restrict__ f,
                                                  const float *__restrict__ flo,
                                                  const uint8_t *__restrict__ mask, int mode, int RC,
                                                  int64_t B, float *__restrict__ g) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (i >= B) return;
  if (mode) {
    bool m = mask[i / RC] != 0;
    if (m != (mode == 1)) return;
  }
  double acc = 0.0;
  for (int64_t e = __ldg(ptr + i) + lane; e < __ldg(ptr + i + 1); e += 32) {
    const int32_t c = __ldcs(col + e);
    acc = fma((double)ld_stream(val, e), (double)__ldg(f + c) + (double)__ldg(flo + c), acc);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) g[i] = (float)(use_scale ? acc * (double)scale[i] : acc);
}

// ---------------------------------------------------------------- live-voxel prices
// stat: [0] bits of max |f_j| (non-negative floats order like their bits),
// [1] entries of the rows with f_j != 0, [5] number of those rows (these
// three cleared before each call); [2] calls that took the live-voxel form,
// [3] calls, [4] entries read by the live-voxel calls (cumulative).
__device__ __forceinline__ bool price_sparse(const unsigned long long *stat, const double *rowsum_max,
                                             int path, int64_t nnz, int &S) {
  const double bound = (double)__uint_as_float((unsigned)stat[0]) * rowsum_max[0];
  int e = 0;
  frexp(bound, &e);  // bound < 2^e
  S = bound > 0.0 ? 62 - e : 0;
  if (!isfinite(bound)) return false;  // non-finite prices come from the row products
  return path == VMAT_PRICE_LIVE || (path == VMAT_PRICE_AUTO && stat[1] * 16 <= (unsigned long long)nnz);
}

// beam of beamlet i: floor(i / RC) as (i * ceil(2^40 / RC)) >> 40, exact for
// i < 2^23 and RC < 2^17 (the error i * delta / 2^40 < 2^-17 < 1 / RC)
__device__ __forceinline__ int beam_of(unsigned i, unsigned long long rc_magic) {
  return (int)(((unsigned long long)i * rc_magic) >> 40);
}

__device__ __forceinline__ bool mask_selected(const uint8_t *mask, int mode, int k) {
  return mode == 0 || ((mask[k] != 0) == (mode == 1));
}

// round(d * f * 2^S) for finite floats d >= 0 and f, from the exact 48-bit
// product of their significands (integer pipe; no FP64): ties away from zero.
// The caller's S keeps |d f| 2^S below 2^62.
__device__ __forceinline__ long long fixp_mul(float d, float f, int S) {
  const unsigned bd = __float_as_uint(d), bf = __float_as_uint(f);
  int ed = (int)((bd >> 23) & 0xffu), ef = (int)((bf >> 23) & 0xffu);
  unsigned md = bd & 0x7fffffu, mf = bf & 0x7fffffu;
  if (ed) md |= 0x800000u; else ed = 1;  // subnormals: no implicit bit, exponent of 1
  if (ef) mf |= 0x800000u; else ef = 1;
  const unsigned long long p = (unsigned long long)md * mf;  // d f = p 2^(ed + ef - 300)
  const int sh = ed + ef - 300 + S;
  unsigned long long v;
  if (sh >= 0) v = p << sh;
  else if (sh > -63) v = (p + (1ull << (-sh - 1))) >> (-sh);
  else v = 0ull;
  return (bf >> 31) ? -(long long)v : (long long)v;
}

// max |f|, the live rows' entry count and the list of live rows (in whatever
// order the warps append them: the integer sums do not depend on it)
__global__ void __launch_bounds__(256) k_price_scan(const float *__restrict__ f,
                                                    const int64_t *__restrict__ vm_ptr, int32_t Va,
                                                    unsigned long long *stat, int32_t *live) {
  const int lane = threadIdx.x & 31;
  unsigned fb = 0;
  unsigned long long n = 0;
  for (int32_t a0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; a0 < Va; a0 += gridDim.x * blockDim.x) {
    const int32_t a = a0 + lane;
    const float v = a < Va ? f[a] : 0.f;
    const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
    if (v != 0.f) {
      fb = max(fb, __float_as_uint(fabsf(v)));
      n += (unsigned long long)(vm_ptr[a + 1] - vm_ptr[a]);
    }
    if (m) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(stat + 5, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (v != 0.f) live[base + __popc(m & ((1u << lane) - 1u))] = a;
    }
  }
  for (int o = 16; o; o >>= 1) {
    fb = max(fb, __shfl_xor_sync(0xffffffffu, fb, o));
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if (lane == 0 && n) {
    atomicMax(stat, (unsigned long long)fb);
    atomicAdd(stat + 1, n);
  }
}

// one warp per live row at a time (4 entries per lane in flight): each entry
// of a selected beam goes to its beamlet's fixed-point accumulator
template <typename TV>
__global__ void __launch_bounds__(256) k_price_live(const int64_t *__restrict__ vm_ptr,
                                                    const int32_t *__restrict__ vm_col,
                                                    const TV *__restrict__ vm_val,
                                                    const float *__restrict__ f,
                                                    const int32_t *__restrict__ live,
                                                    const uint8_t *__restrict__ mask, int mode,
                                                    unsigned long long rc_magic,
                                                    const unsigned long long *__restrict__ stat,
                                                    const double *__restrict__ rowsum_max, int path,
                                                    int64_t nnz, unsigned long long *acc) {
  int S;
  if (!price_sparse(stat, rowsum_max, path, nnz, S)) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5), nlive = (int64_t)stat[5];
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nlive; q += nw) {
    const int32_t a = live[q];
    const float fv = f[a];
    const int64_t e1 = vm_ptr[a + 1];
    for (int64_t e = vm_ptr[a] + lane; e < e1; e += 128) {
      int32_t i[4];
      float d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = e + 32 * u < e1;
        i[u] = in ? __ldcs(vm_col + e + 32 * u) : -1;
        d[u] = in ? ld_stream(vm_val, e + 32 * u) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i[u] < 0 || !mask_selected(mask, mode, beam_of((unsigned)i[u], rc_magic))) continue;
        const long long v = fixp_mul(d[u], fv, S);
        if (v) atomicAdd(acc + i[u], (unsigned long long)v);
      }
    }
  }
}

// ---------------------------------------------------------------- price rows
// Row products (warp per beamlet row, grid-stride) unless the call took the
// live-voxel form; then each thread converts (and clears) the accumulators of
// its beamlets.
template <typename TV>
__global__ void __launch_bounds__(256) k_price_rows(const int64_t *__restrict__ ptr,
                                                    const int32_t *__restrict__ col,
                                                    const TV *__restrict__ val,
                                                    const float *__restrict__ scale, int use_scale,
                                                    const float *__restrict__ f,
                                                    const uint8_t *__restrict__ mask, int mode, int RC,
                                                    int64_t B, unsigned long long *stat,
                                                    const double *__restrict__ rowsum_max, int path,
                                                    int64_t nnz, unsigned long long *acc,
                                                    float *__restrict__ g) {
  int S;
  const bool sparse = price_sparse(stat, rowsum_max, path, nnz, S);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    stat[3] += 1;
    if (sparse) {
      stat[2] += 1;
      stat[4] += stat[1];
    }
  }
  if (sparse) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B;
         i += (int64_t)gridDim.x * blockDim.x) {
      if (!mask_selected(mask, mode, (int)(i / RC))) continue;
      const long long v = (long long)acc[i];
      acc[i] = 0ull;
      const double p = ldexp((double)v, -S);
      g[i] = (float)(use_scale ? p * (double)scale[i] : p);
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t i = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); i < B; i += nw) {
    if (!mask_selected(mask, mode, (int)(i / RC))) continue;
    const float a = warp_row_dot<TV>(col, val, f, __ldg(ptr + i), __ldg(ptr + i + 1), lane);
    if (lane == 0) g[i] = use_scale ? a * scale[i] : a;
  }
}

// largest row sum of Dhat (FP64), for the fixed-point scale of the live-voxel prices
template <typename TV>
__global__ void k_row_sum_max(const int64_t *__restrict__ ptr, const TV *__restrict__ val, int64_t B,
                              unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (i >= B) return;
  double s = 0.0;
  for (int64_t e = ptr[i] + lane; e < ptr[i + 1]; e += 32) s += (double)vmat_ld(val, e);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

vmat_status vmat_row_sum_max(vmat_ctx *ctx) {
  const unsigned nb = (unsigned)((ctx->B + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  unsigned long long *out = (unsigned long long *)ctx->rowsum_max;
  VMAT_CUDA(ctx, cudaMemsetAsync(out, 0, 8, ctx->stream));
  if (nb == 0) return VMAT_OK;
  if (ctx->dt == VMAT_F32)
    k_row_sum_max<float><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, (const float *)ctx->bm_val, ctx->B, out);
  else if (ctx->dt == VMAT_F16)
    k_row_sum_max<__half><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, (const __half *)ctx->bm_val, ctx->B, out);
  else
    k_row_sum_max<__nv_bfloat16><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, (const __nv_bfloat16 *)ctx->bm_val,
                                                               ctx->B, out);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  return VMAT_OK;
}

__global__ void k_gather_active(const float *__restrict__ full, const int32_t *__restrict__ act,
                                int32_t Va, int32_t Vpad, float *__restrict__ out) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < Vpad) out[a] = a < Va ? full[act[a]] : 0.f;
}

vmat_status vmat_launch_price(vmat_ctx *ctx, const float *f_act, const uint8_t *mask, int mode,
                              float *g, const float *f_lo) {
  const int64_t B = ctx->B;
  unsigned nb = (unsigned)((B + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  const int RC = ctx->R * ctx->C;
  int us = ctx->dt != VMAT_F32;
  if (f_lo) {
    if (ctx->dt == VMAT_F32)
      k_price_xp<float><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, ctx->bm_col, (const float *)ctx->bm_val,
                                                     ctx->scale, us, f_act, f_lo, mask, mode, RC, B, g);
    else if (ctx->dt == VMAT_F16)
      k_price_xp<__half><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, ctx->bm_col, (const __half *)ctx->bm_val,
                                                      ctx->scale, us, f_act, f_lo, mask, mode, RC, B, g);
    else
      k_price_xp<__nv_bfloat16><<<nb, 256, 0, ctx->stream>>>(ctx->bm_ptr, ctx->bm_col,
                                                             (const __nv_bfloat16 *)ctx->bm_val,
                                                             ctx->scale, us, f_act, f_lo, mask, mode,
                                                             RC, B, g);
  } else {
    // live-voxel form (or the row products when the live rows are not sparse)
    cudaStream_t st = ctx->stream;
    unsigned long long *stat = ctx->pstat;
    VMAT_CUDA(ctx, cudaMemsetAsync(stat, 0, 16, st));
    VMAT_CUDA(ctx, cudaMemsetAsync(stat + 5, 0, 8, st));
    const unsigned nscan = (unsigned)std::min<int64_t>((ctx->Va + 255) / 256, 4 * ctx->num_sms);
    k_price_scan<<<nscan > 0 ? nscan : 1, 256, 0, st>>>(f_act, ctx->vm_ptr, ctx->Va, stat, ctx->plive);
    const int path = ctx->price_path;
    const unsigned nlive = (unsigned)(8 * ctx->num_sms);  // persistent warps over the live rows
    const unsigned nrows = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, 32 * ctx->num_sms));
    const unsigned long long rc_magic = ((1ull << 40) + (unsigned long long)RC - 1) / (unsigned long long)RC;
#define VMAT_PRICE_LAUNCH(TV)                                                                          \
  k_price_live<TV><<<nlive, 256, 0, st>>>(ctx->vm_ptr, ctx->vm_col, (const TV *)ctx->vm_val, f_act,   \
                                          ctx->plive, mask, mode, rc_magic, stat, ctx->rowsum_max,    \
                                          path, ctx->nnz, ctx->pacc);                                 \
  k_price_rows<TV><<<nrows, 256, 0, st>>>(ctx->bm_ptr, ctx->bm_col, (const TV *)ctx->bm_val, ctx->scale, \
                                       us, f_act, mask, mode, RC, B, stat, ctx->rowsum_max, path,     \
                                       ctx->nnz, ctx->pacc, g)
    if (ctx->dt == VMAT_F32) {
      VMAT_PRICE_LAUNCH(float);
    } else if (ctx->dt == VMAT_F16) {
      VMAT_PRICE_LAUNCH(__half);
    } else {
      VMAT_PRICE_LAUNCH(__nv_bfloat16);
    }
#undef VMAT_PRICE_LAUNCH
    ctx->n_launches += 2;
  }
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  return VMAT_OK;
}

vmat_status vmat_gather_active(vmat_ctx *ctx, const float *full, float *act) {
  k_gather_active<<<(ctx->Vpad + 255) / 256, 256, 0, ctx->stream>>>(full, ctx->act_vox, ctx->Va,
                                                                    ctx->Vpad, act);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  return VMAT_OK;
}

// ---------------------------------------------------------------- dose
template <typename TV>
__global__ void __launch_bounds__(256) k_dose(const int64_t *__restrict__ ptr,
                                              const int32_t *__restrict__ col,
                                              const TV *__restrict__ val,
                                              const float *__restrict__ x, int32_t Va,
                                              const int32_t *__restrict__ act,
                                              const uint8_t *__restrict__ sid,
                                              const float *__restrict__ tabf,
                                              const double *__restrict__ tabd,
                                              float *__restrict__ z_full,
                                              float *__restrict__ fp_full,
                                              double *__restrict__ part) {
  __shared__ double s_cost[WARPS_PER_BLOCK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t a = blockIdx.x * WARPS_PER_BLOCK + warp;
  double c = 0.0;
  if (a < Va) {
    float z = warp_row_dot<TV>(col, val, x, __ldg(ptr + a), __ldg(ptr + a + 1), lane);
    if (lane == 0) {
      int q = sid[a];
      int32_t j = act[a];
      if (z_full) z_full[j] = z;
      if (fp_full) fp_full[j] = vmat_dF(z, tabf[q], tabf[256 + q], tabf[512 + q]);
      c = vmat_F((double)z, tabd[q], tabd[256 + q], tabd[512 + q]);
    }
  }
  if (lane == 0) s_cost[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0 && part) {
    double s = 0.0;
    for (int q = 0; q < WARPS_PER_BLOCK; ++q) s += s_cost[q];
    part[blockIdx.x] = s;
  }
}

// z = 0 and F'(0) on voxels that D never reaches
__global__ void k_fill_inactive(const int32_t *__restrict__ vox2act,
                                const uint8_t *__restrict__ sid_full, const float *__restrict__ tabf,
                                int32_t V, float *z_full, float *fp_full) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= V || vox2act[j] >= 0) return;
  int q = sid_full[j];
  if (z_full) z_full[j] = 0.f;
  if (fp_full) fp_full[j] = vmat_dF(0.f, tabf[q], tabf[256 + q], tabf[512 + q]);
}

__global__ void k_scale_fluence(const float *__restrict__ x, const float *__restrict__ s, int64_t B,
                                float *__restrict__ xs) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) xs[i] = x[i] * s[i];
}

// fixed-order sum of n partials by one block
__global__ void k_sum_partials(const double *__restrict__ part, int64_t n, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

vmat_status vmat_launch_dose(vmat_ctx *ctx, const float *x, float *z_full, float *fp_full,
                             double *cost_dev) {
  cudaStream_t st = ctx->stream;
  const float *xin = x;
  if (ctx->dt != VMAT_F32) {
    k_scale_fluence<<<(unsigned)((ctx->B + 255) / 256), 256, 0, st>>>(x, ctx->scale, ctx->B, ctx->xs);
    xin = ctx->xs;
  }
  unsigned nb = (unsigned)((ctx->Va + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  if (nb == 0) nb = 1;
  if ((int64_t)nb + 1 > ctx->red_len) return vmat_fail(ctx, VMAT_EINVAL, "scratch too small");
  double *part = cost_dev ? ctx->red : nullptr;
#define VMAT_DOSE_ARGS                                                                        \
  ctx->vm_ptr, ctx->vm_col, (const TV *)ctx->vm_val, xin, ctx->Va, ctx->act_vox, ctx->sid, \
      ctx->tabf, ctx->tabd, z_full, fp_full, part
  if (ctx->dt == VMAT_F32) {
    typedef float TV;
    k_dose<TV><<<nb, 256, 0, st>>>(VMAT_DOSE_ARGS);
  } else if (ctx->dt == VMAT_F16) {
    typedef __half TV;
    k_dose<TV><<<nb, 256, 0, st>>>(VMAT_DOSE_ARGS);
  } else {
    typedef __nv_bfloat16 TV;
    k_dose<TV><<<nb, 256, 0, st>>>(VMAT_DOSE_ARGS);
  }
#undef VMAT_DOSE_ARGS
  if (z_full || fp_full)
    k_fill_inactive<<<(ctx->V + 255) / 256, 256, 0, st>>>(ctx->vox2act, ctx->sid_full, ctx->tabf,
                                                          ctx->V, z_full, fp_full);
  if (cost_dev) k_sum_partials<<<1, 256, 0, st>>>(part, nb, cost_dev);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1 + (ctx->dt != VMAT_F32) + ((z_full || fp_full) ? 1 : 0) + (cost_dev ? 1 : 0);
  return VMAT_OK;
}

// ---------------------------------------------------------------- batched (32 vectors)
// 8 consecutive values (one union entry of a row tile, 16- or 32-byte aligned)
__device__ __forceinline__ void load8(const float *p, float (&v)[8]) {
  const float4 a = __ldcs((const float4 *)p), b = __ldcs((const float4 *)p + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const __half *p, float (&v)[8]) {
  const uint4 u = __ldcs((const uint4 *)p);
  const __half2 *h = (const __half2 *)&u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __half22float2(h[q]);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}
__device__ __forceinline__ void load8(const __nv_bfloat16 *p, float (&v)[8]) {
  const uint4 u = __ldcs((const uint4 *)p);
  const __nv_bfloat162 *h = (const __nv_bfloat162 *)&u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __bfloat1622float2(h[q]);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}

// Row-tiled batched product (tiles.cu): one warp per tile of 8 rows, lane =
// vector.  The warp stages 32 union entries at a time (column, 8 values as
// floats, times the column's scale for reduced-precision dose) in shared
// memory, then for each entry gathers the dense operand's 128-byte row once
// and updates all 8 rows; each row sums its own entries in the CSR's
// column order.
template <typename TV>
__device__ __forceinline__ void tile_rows32(const RowTiles &t, const TV *__restrict__ uval,
                                            const float *__restrict__ colscale,
                                            const float *__restrict__ X, int64_t tile, int lane,
                                            int32_t *s_c, float4 *s_v, float (&acc)[8]) {
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = 0.f;
  const int64_t e0 = t.uptr[tile], e1 = t.uptr[tile + 1];
  for (int64_t base = e0; base < e1; base += 32) {
    const int n = (int)min((int64_t)32, e1 - base);
    if (lane < n) {
      const int32_t c = __ldcs(t.ucol + base + lane);
      float v[8];
      load8(uval + (base + lane) * 8, v);
      if (colscale) {
        const float sc = __ldg(colscale + c);
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] *= sc;
      }
      s_c[lane] = c;
      s_v[2 * lane] = make_float4(v[0], v[1], v[2], v[3]);
      s_v[2 * lane + 1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    __syncwarp();
#pragma unroll 4
    for (int q = 0; q < n; ++q) {
      const float x = __ldg(X + (size_t)s_c[q] * 32 + lane);
      const float4 a = s_v[2 * q], b = s_v[2 * q + 1];
      acc[0] = fmaf(a.x, x, acc[0]);
      acc[1] = fmaf(a.y, x, acc[1]);
      acc[2] = fmaf(a.z, x, acc[2]);
      acc[3] = fmaf(a.w, x, acc[3]);
      acc[4] = fmaf(b.x, x, acc[4]);
      acc[5] = fmaf(b.y, x, acc[5]);
      acc[6] = fmaf(b.z, x, acc[6]);
      acc[7] = fmaf(b.w, x, acc[7]);
    }
    __syncwarp();
  }
}

template <typename TV>
__global__ void __launch_bounds__(256) k_dose32t(RowTiles t, const float *__restrict__ scale,
                                                 int use_scale, const float *__restrict__ X,
                                                 int32_t Va, const int32_t *__restrict__ act,
                                                 const uint8_t *__restrict__ sid,
                                                 const float *__restrict__ tabf,
                                                 const double *__restrict__ tabd, float *Z,
                                                 float *Fp, double *part) {
  __shared__ int32_t s_c[WARPS_PER_BLOCK][32];
  __shared__ float4 s_v[WARPS_PER_BLOCK][64];
  __shared__ double s_cost[WARPS_PER_BLOCK][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
  double c = 0.0;
  if (tile < t.n_tiles) {
    float acc[8];
    tile_rows32<TV>(t, (const TV *)t.uval, use_scale ? scale : nullptr, X, tile, lane, s_c[warp],
                    s_v[warp], acc);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t a = tile * 8 + r;
      if (a < Va) {
        const int q = sid[a];
        const size_t j = (size_t)act[a];
        Z[j * 32 + lane] = acc[r];
        if (Fp) Fp[j * 32 + lane] = vmat_dF(acc[r], tabf[q], tabf[256 + q], tabf[512 + q]);
        c += vmat_F((double)acc[r], tabd[q], tabd[256 + q], tabd[512 + q]);
      }
    }
  }
  s_cost[warp][lane] = c;
  __syncthreads();
  if (part && threadIdx.x < 32) {
    double sum = 0.0;
    for (int w = 0; w < WARPS_PER_BLOCK; ++w) sum += s_cost[w][threadIdx.x];
    part[(size_t)blockIdx.x * 32 + threadIdx.x] = sum;
  }
}

template <typename TV>
__global__ void __launch_bounds__(256) k_price32t(RowTiles t, const float *__restrict__ scale,
                                                  int use_scale, const float *__restrict__ Fa,
                                                  int64_t B, const float *__restrict__ colw,
                                                  float *__restrict__ G) {
  __shared__ int32_t s_c[WARPS_PER_BLOCK][32];
  __shared__ float4 s_v[WARPS_PER_BLOCK][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
  if (tile >= t.n_tiles) return;
  float acc[8];
  tile_rows32<TV>(t, (const TV *)t.uval, nullptr, Fa, tile, lane, s_c[warp], s_v[warp], acc);
  const float cw = colw ? colw[lane] : 1.f;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = tile * 8 + r;
    if (i < B) {
      float g = acc[r];
      if (use_scale) g *= scale[i];
      if (colw) g *= cw;
      G[(size_t)i * 32 + lane] = g;
    }
  }
}

__global__ void k_fill_inactive32(const int32_t *__restrict__ vox2act,
                                  const uint8_t *__restrict__ sid_full,
                                  const float *__restrict__ tabf, int32_t V, float *Z, float *Fp) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)V * 32) return;
  int32_t j = (int32_t)(t >> 5);
  if (vox2act[j] >= 0) return;
  int q = sid_full[j];
  Z[t] = 0.f;
  if (Fp) Fp[t] = vmat_dF(0.f, tabf[q], tabf[256 + q], tabf[512 + q]);
}

// per-vector fixed-order sums of nb x 32 partials
__global__ void k_sum_partials32(const double *__restrict__ part, int64_t nb, double *out) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t q = w; q < nb; q += 8) s += part[q * 32 + lane];
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q][lane];
    out[lane] = t;
  }
}

__global__ void k_gather_active32(const float *__restrict__ full, const int32_t *__restrict__ act,
                                  int32_t Va, float *__restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)Va * 32) return;
  out[t] = full[(size_t)act[t >> 5] * 32 + (t & 31)];
}

vmat_status vmat_launch_dose_batch32(vmat_ctx *ctx, const float *X, float *Z, float *Fp,
                                     double *cost_dev) {
  cudaStream_t st = ctx->stream;
  unsigned nb = (unsigned)((ctx->Va + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  if (nb == 0) nb = 1;
  if ((int64_t)nb * 32 + 64 > ctx->red_len) return vmat_fail(ctx, VMAT_EINVAL, "scratch too small");
  double *part = cost_dev ? ctx->red : nullptr;
  int us = ctx->dt != VMAT_F32;
  vmat_status ts = vmat_ensure_row_tiles(ctx, true);
  if (ts != VMAT_OK) return ts;
  // one block per 8 tiles of 8 active voxels: fewer partial rows than the
  // warp-per-voxel form, so the scratch check above covers them
  nb = (unsigned)((ctx->vtiles.n_tiles + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  if (nb == 0) nb = 1;
#define VMAT_D32_ARGS                                                                    \
  ctx->vtiles, ctx->scale, us, X, ctx->Va, ctx->act_vox, ctx->sid, ctx->tabf, ctx->tabd, Z, \
      Fp, part
  if (ctx->dt == VMAT_F32) {
    typedef float TV;
    k_dose32t<TV><<<nb, 256, 0, st>>>(VMAT_D32_ARGS);
  } else if (ctx->dt == VMAT_F16) {
    typedef __half TV;
    k_dose32t<TV><<<nb, 256, 0, st>>>(VMAT_D32_ARGS);
  } else {
    typedef __nv_bfloat16 TV;
    k_dose32t<TV><<<nb, 256, 0, st>>>(VMAT_D32_ARGS);
  }
#undef VMAT_D32_ARGS
  k_fill_inactive32<<<(unsigned)(((int64_t)ctx->V * 32 + 255) / 256), 256, 0, st>>>(
      ctx->vox2act, ctx->sid_full, ctx->tabf, ctx->V, Z, Fp);
  if (cost_dev) k_sum_partials32<<<1, 256, 0, st>>>(part, nb, cost_dev);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 2 + (cost_dev ? 1 : 0);
  return VMAT_OK;
}

vmat_status vmat_launch_price_batch32(vmat_ctx *ctx, const float *Fp, const float *colw, float *G) {
  cudaStream_t st = ctx->stream;
  if (!ctx->fa32) VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->fa32, (size_t)(ctx->Va > 0 ? ctx->Va : 1) * 32));
  float *Fa = ctx->fa32;
  k_gather_active32<<<(unsigned)(((int64_t)ctx->Va * 32 + 255) / 256 + 1), 256, 0, st>>>(
      Fp, ctx->act_vox, ctx->Va, Fa);
  vmat_status ts = vmat_ensure_row_tiles(ctx, false);
  if (ts != VMAT_OK) return ts;
  unsigned nb = (unsigned)((ctx->btiles.n_tiles + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
  if (nb == 0) nb = 1;
  int us = ctx->dt != VMAT_F32;
  if (ctx->dt == VMAT_F32)
    k_price32t<float><<<nb, 256, 0, st>>>(ctx->btiles, ctx->scale, us, Fa, ctx->B, colw, G);
  else if (ctx->dt == VMAT_F16)
    k_price32t<__half><<<nb, 256, 0, st>>>(ctx->btiles, ctx->scale, us, Fa, ctx->B, colw, G);
  else
    k_price32t<__nv_bfloat16><<<nb, 256, 0, st>>>(ctx->btiles, ctx->scale, us, Fa, ctx->B, colw, G);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 2;
  return VMAT_OK;
}

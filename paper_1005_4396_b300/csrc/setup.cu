// Context creation: validation, the storage forms of D on the device, and the
// plan-state buffers.  D arrives as a beamlet-major CSR on the host (Sec. 2.1:
// D_ij is the dose to voxel j from beamlet i at unit intensity); the device
// keeps it twice over the compacted set of voxels that D reaches:
//   beamlet-major  (row i: the voxels of beamlet i)  for prices g = D f,
//   voxel-major    (row j: the beamlets reaching j, sorted by beamlet, hence
//                   grouped by beam) for doses z = D^T x and aperture columns.
// F16/BF16 storage scales each beamlet row by s_i = max_j D_ij.
#include <cub/cub.cuh>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "vmat_internal.cuh"

static thread_local std::string g_create_error;

vmat_status vmat_fail(vmat_ctx *ctx, vmat_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_error = buf;
  return st;
}

vmat_status vmat_cuda_fail(vmat_ctx *ctx, cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a non-sticky launch error so the context stays usable
  return vmat_fail(ctx, e == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

extern "C" const char *vmat_last_error(const vmat_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

// ---------------------------------------------------------------- kernels
// One warp per beamlet row: entries strictly ascending, inside the grid,
// finite and positive.  Sets *bad on the first violation found.
template <typename TV>
__global__ void k_validate_rows(const int64_t *ptr, const int32_t *vox, const TV *val, int64_t B,
                                int32_t V, int *bad) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= B) return;
  int64_t e0 = ptr[i], e1 = ptr[i + 1];
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    int32_t v = vox[e];
    double d = (double)val[e];
    bool ok = v >= 0 && v < V && isfinite(d) && d > 0.0 && (e == e0 || vox[e - 1] < v);
    if (!ok) atomicExch(bad, 1);
  }
}

__global__ void k_mark_active(const int32_t *vox, int64_t nnz, int32_t *flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    flag[vox[e]] = 1;
}

__global__ void k_compact(const int32_t *flag, const int32_t *excl, int32_t V, int32_t *vox2act,
                          int32_t *act_vox) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= V) return;
  if (flag[j]) {
    vox2act[j] = excl[j];
    act_vox[excl[j]] = j;
  } else {
    vox2act[j] = -1;
  }
}

__global__ void k_remap_cols(int32_t *vox, int64_t nnz, const int32_t *vox2act) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    vox[e] = vox2act[vox[e]];
}

// One warp per beamlet row: per-beamlet scale (max of the row; 1 for F32
// storage), the stored value val/scale, and the transpose sort key
// (active voxel << 32 | beamlet).
template <typename TIN, typename TOUT>
__global__ void k_rows_convert(const int64_t *ptr, const int32_t *col, const TIN *val, int64_t B,
                               int use_scale, float *scale, TOUT *out, unsigned long long *key,
                               int32_t *idx) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= B) return;
  int64_t e0 = ptr[i], e1 = ptr[i + 1];
  float s = 1.0f;
  if (use_scale) {
    double m = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) m = fmax(m, (double)val[e]);
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s = e1 > e0 ? (float)m : 1.0f;
    if (lane == 0) scale[i] = s;
  }
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    double v = (double)val[e];
    if (use_scale) v = v / (double)s;
    out[e] = (TOUT)(float)v;
    key[e] = ((unsigned long long)(uint32_t)col[e] << 32) | (unsigned long long)(uint32_t)i;
    idx[e] = (int32_t)e;
  }
}

template <typename TV>
__global__ void k_transpose_fill(const unsigned long long *key, const int32_t *idx, const TV *bm_val,
                                 int64_t nnz, int32_t *vm_col, TV *vm_val, int64_t *vm_ptr,
                                 int32_t Va) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long k = key[e];
    int32_t a = (int32_t)(k >> 32);
    vm_col[e] = (int32_t)(k & 0xffffffffull);
    vm_val[e] = bm_val[idx[e]];
    if (e == 0 || (int32_t)(key[e - 1] >> 32) != a) vm_ptr[a] = e;
    if (e == nnz - 1) vm_ptr[Va] = nnz;
  }
}

__global__ void k_active_sid(const uint8_t *sid_full, const int32_t *act_vox, int32_t Va,
                             int32_t Vpad, uint8_t *sid) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Vpad) return;
  sid[a] = a < Va ? sid_full[act_vox[a]] : (uint8_t)VMAT_NULL_STRUCT;
}

// sum of F(0) over voxels that D never reaches (their dose is always 0)
__global__ void k_inactive_cost(const uint8_t *sid_full, const int32_t *vox2act, int32_t V,
                                const double *tab, double *part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < V; j += gridDim.x * blockDim.x)
    if (vox2act[j] < 0) {
      int q = sid_full[j];
      s += vmat_F(0.0, tab[q], tab[256 + q], tab[512 + q]);
    }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_fixed(const double *part, int n, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// ---------------------------------------------------------------- create
namespace {
struct Tmp {
  std::vector<void *> p;
  ~Tmp() {
    for (void *q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t alloc(T **q, size_t n) {
    cudaError_t e = cudaMalloc((void **)q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e == cudaSuccess) p.push_back(*q);
    return e;
  }
};
}  // namespace

static vmat_status validate_host(const vmat_problem *P) {
  if (!P) return vmat_fail(nullptr, VMAT_EINVAL, "problem is NULL");
  if (P->n_vox <= 0 || P->n_angles <= 0 || P->n_rows <= 0 || P->n_cols <= 0)
    return vmat_fail(nullptr, VMAT_EINVAL, "sizes must be positive");
  if (P->n_angles > VMAT_MAX_ANGLES || P->n_rows > VMAT_MAX_ROWS || P->n_cols > VMAT_MAX_COLS)
    return vmat_fail(nullptr, VMAT_EINVAL, "at most %d beams, %d rows, %d columns",
                     VMAT_MAX_ANGLES, VMAT_MAX_ROWS, VMAT_MAX_COLS);
  if (!P->theta_deg || !P->struct_id || !P->T || !P->alpha || !P->beta || !P->row_ptr ||
      (P->nnz > 0 && (!P->vox_idx || !P->val)))
    return vmat_fail(nullptr, VMAT_EINVAL, "NULL array in problem");
  if (P->n_struct <= 0 || P->n_struct > 255)
    return vmat_fail(nullptr, VMAT_EINVAL, "n_struct must be in [1, 255]");
  if (P->nnz < 0 || P->nnz >= (int64_t)INT32_MAX)
    return vmat_fail(nullptr, VMAT_EINVAL, "nnz must be in [0, 2^31-1)");
  if (P->val_dtype != VMAT_F64 && P->val_dtype != VMAT_F32)
    return vmat_fail(nullptr, VMAT_EINVAL, "val_dtype must be VMAT_F64 or VMAT_F32");
  if (!(P->gamma >= 0.0) || !isfinite(P->gamma)) return vmat_fail(nullptr, VMAT_EINVAL, "gamma");
  if (P->max_leaf_step < 0) return vmat_fail(nullptr, VMAT_EINVAL, "max_leaf_step < 0");
  for (int k = 0; k < P->n_angles; ++k) {
    double t = P->theta_deg[k];
    if (!(t >= 0.0 && t < 360.0) || (k > 0 && !(t > P->theta_deg[k - 1])))
      return vmat_fail(nullptr, VMAT_EINVAL, "theta must be strictly increasing in [0, 360)");
  }
  for (int q = 0; q < P->n_struct; ++q)
    if (!isfinite(P->T[q]) || !(P->alpha[q] >= 0.0) || !(P->beta[q] >= 0.0) ||
        !isfinite(P->alpha[q]) || !isfinite(P->beta[q]))
      return vmat_fail(nullptr, VMAT_EINVAL, "structure %d: T, alpha, beta must be finite, weights >= 0", q);
  for (int64_t j = 0; j < P->n_vox; ++j)
    if (P->struct_id[j] >= P->n_struct)
      return vmat_fail(nullptr, VMAT_EINVAL, "struct_id[%lld] >= n_struct", (long long)j);
  const int64_t B = (int64_t)P->n_angles * P->n_rows * P->n_cols;
  if (P->row_ptr[0] != 0 || P->row_ptr[B] != P->nnz)
    return vmat_fail(nullptr, VMAT_EINVAL, "row_ptr must start at 0 and end at nnz");
  for (int64_t i = 0; i < B; ++i)
    if (P->row_ptr[i + 1] < P->row_ptr[i])
      return vmat_fail(nullptr, VMAT_EINVAL, "row_ptr must be non-decreasing");
  return VMAT_OK;
}

template <typename TOUT>
static vmat_status build_storage(vmat_ctx *ctx, Tmp &tmp, const int32_t *colv, const void *val_in,
                                 vmat_dtype in_dt) {
  const int64_t nnz = ctx->nnz, B = ctx->B;
  cudaStream_t st = ctx->stream;
  int use_scale = ctx->dt != VMAT_F32;
  TOUT *bm_val, *vm_val;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &bm_val, nnz));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &vm_val, nnz));
  ctx->bm_val = bm_val;
  ctx->vm_val = vm_val;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->scale, B));
  if (!use_scale) {
    std::vector<float> ones(B, 1.0f);
    VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->scale, ones.data(), B * sizeof(float),
                                   cudaMemcpyHostToDevice, st));
    VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  }
  unsigned long long *key, *key2;
  int32_t *idx, *idx2;
  VMAT_CUDA(ctx, tmp.alloc(&key, nnz));
  VMAT_CUDA(ctx, tmp.alloc(&key2, nnz));
  VMAT_CUDA(ctx, tmp.alloc(&idx, nnz));
  VMAT_CUDA(ctx, tmp.alloc(&idx2, nnz));
  unsigned nb = (unsigned)((B + 7) / 8);
  if (in_dt == VMAT_F64)
    k_rows_convert<double, TOUT><<<nb, 256, 0, st>>>(ctx->bm_ptr, colv, (const double *)val_in, B,
                                                     use_scale, ctx->scale, bm_val, key, idx);
  else
    k_rows_convert<float, TOUT><<<nb, 256, 0, st>>>(ctx->bm_ptr, colv, (const float *)val_in, B,
                                                    use_scale, ctx->scale, bm_val, key, idx);
  VMAT_CUDA(ctx, cudaGetLastError());
  int end_bit = 32;
  while ((1ll << (end_bit - 32)) < (long long)ctx->Va) ++end_bit;
  size_t tbytes = 0;
  VMAT_CUDA(ctx, cub::DeviceRadixSort::SortPairs(nullptr, tbytes, key, key2, idx, idx2, (int)nnz,
                                                 0, end_bit, st));
  void *tst;
  VMAT_CUDA(ctx, tmp.alloc((char **)&tst, tbytes));
  VMAT_CUDA(ctx, cub::DeviceRadixSort::SortPairs(tst, tbytes, key, key2, idx, idx2, (int)nnz, 0,
                                                 end_bit, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->vm_ptr, ctx->Va + 1));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->vm_ptr, 0, ((size_t)ctx->Va + 1) * 8, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->vm_col, nnz));
  if (nnz > 0)
    k_transpose_fill<TOUT><<<4 * ctx->num_sms, 256, 0, st>>>(key2, idx2, bm_val, nnz, ctx->vm_col,
                                                             vm_val, ctx->vm_ptr, ctx->Va);
  VMAT_CUDA(ctx, cudaGetLastError());
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  return VMAT_OK;
}

// Buffers whose size follows the master kernel's tiling (padded voxel count,
// grid): structure ids of the active voxels, the aperture-dose matrix and its
// subtile flags, plan dose and derivative, reduction scratch.
static vmat_status alloc_xp(vmat_ctx *ctx);

static vmat_status alloc_tiled(vmat_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  const int32_t Vpad = ctx->Vpad;
  const int N = ctx->N;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->sid, Vpad));
  k_active_sid<<<(Vpad + 255) / 256, 256, 0, st>>>(ctx->sid_full, ctx->act_vox, ctx->Va, Vpad, ctx->sid);
  VMAT_CUDA(ctx, cudaGetLastError());
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->M, (size_t)N * Vpad));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->M, 0, (size_t)N * Vpad * 4, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->tflag, (size_t)N * ctx->master_grid * (ctx->master_vpt / 4)));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->zact, Vpad));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->fpact, Vpad));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->fgather, Vpad));
  // scratch: master partials [grid][N+extra] + reduced gradient [N]; dose
  // partials [ceil(Va/8)] and batched [ceil(Va/8)][32]; result slots at the end
  int64_t nbv = ((int64_t)ctx->Va + 7) / 8 + 1;
  int64_t need = vmat_master_scratch(ctx->master_grid, N);
  if (nbv * 32 > need) need = nbv * 32;
  ctx->red_len = need + 128;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->red, ctx->red_len));
  if (ctx->master_method == VMAT_MASTER_PROJECTED_NEWTON) {
    ctx->hbuf_len = (int64_t)(ctx->master_grid + 1) * vmat_hessian_len(N);
    VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->hbuf, ctx->hbuf_len));
  }
  if (ctx->master_xp) return alloc_xp(ctx);
  return VMAT_OK;
}

// Extended-precision master: the low parts of the columns and of F'.
static vmat_status alloc_xp(vmat_ctx *ctx) {
  if (!ctx->Mlo) {
    VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->Mlo, (size_t)ctx->N * ctx->Vpad));
    VMAT_CUDA(ctx, cudaMemsetAsync(ctx->Mlo, 0, (size_t)ctx->N * ctx->Vpad * 4, ctx->stream));
  }
  if (!ctx->fplo) {
    VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->fplo, (size_t)ctx->Vpad));
    VMAT_CUDA(ctx, cudaMemsetAsync(ctx->fplo, 0, (size_t)ctx->Vpad * 4, ctx->stream));
  }
  return VMAT_OK;
}

static void free_xp(vmat_ctx *ctx) {
  if (ctx->Mlo) {
    cudaFree(ctx->Mlo);
    ctx->Mlo = nullptr;
    ctx->device_bytes -= (int64_t)ctx->N * ctx->Vpad * 4;
  }
  if (ctx->fplo) {
    cudaFree(ctx->fplo);
    ctx->fplo = nullptr;
    ctx->device_bytes -= (int64_t)ctx->Vpad * 4;
  }
}

static void free_tiled(vmat_ctx *ctx) {
  free_xp(ctx);
  void **ptrs[] = {(void **)&ctx->sid, (void **)&ctx->M, (void **)&ctx->tflag, (void **)&ctx->zact,
                   (void **)&ctx->fpact, (void **)&ctx->fgather, (void **)&ctx->red};
  size_t bytes[] = {(size_t)ctx->Vpad, (size_t)ctx->N * ctx->Vpad * 4,
                    (size_t)ctx->N * ctx->master_grid * (ctx->master_vpt / 4) * 4,
                    (size_t)ctx->Vpad * 4, (size_t)ctx->Vpad * 4, (size_t)ctx->Vpad * 4,
                    (size_t)ctx->red_len * 8};
  for (int q = 0; q < 7; ++q)
    if (*ptrs[q]) {
      cudaFree(*ptrs[q]);
      *ptrs[q] = nullptr;
      ctx->device_bytes -= (int64_t)bytes[q];
    }
  if (ctx->hbuf) {
    cudaFree(ctx->hbuf);
    ctx->hbuf = nullptr;
    ctx->device_bytes -= ctx->hbuf_len * 4;
    ctx->hbuf_len = 0;
  }
}

extern "C" vmat_status vmat_set_master_budget(vmat_ctx *ctx, int32_t max_ctas) {
  if (!ctx) return VMAT_EINVAL;
  if (max_ctas < 0) return vmat_fail(ctx, VMAT_EINVAL, "max_ctas must be >= 0");
  if (ctx->n_slots != 0) return vmat_fail(ctx, VMAT_EINVAL, "the plan has columns: call vmat_reset first");
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int old_budget = ctx->sm_budget;
  ctx->sm_budget = max_ctas;
  vmat_status s = vmat_configure_master(ctx);
  if (s != VMAT_OK) {
    ctx->sm_budget = old_budget;
    vmat_configure_master(ctx);
    return s;
  }
  free_tiled(ctx);
  s = alloc_tiled(ctx);
  if (s != VMAT_OK) return s;
  return vmat_reset(ctx);
}

extern "C" vmat_status vmat_set_master_method(vmat_ctx *ctx, int32_t method) {
  if (!ctx) return VMAT_EINVAL;
  if (method != VMAT_MASTER_PROJECTED_GRADIENT && method != VMAT_MASTER_PROJECTED_NEWTON)
    return vmat_fail(ctx, VMAT_EINVAL, "unknown master method %d", method);
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int old = ctx->master_method;
  ctx->master_method = method;
  vmat_status s = vmat_configure_master(ctx);  // same tiling; checks the variant fits an SM
  if (s != VMAT_OK) {
    ctx->master_method = old;
    vmat_configure_master(ctx);
    return s;
  }
  if (method == VMAT_MASTER_PROJECTED_NEWTON && !ctx->hbuf) {
    ctx->hbuf_len = (int64_t)(ctx->master_grid + 1) * vmat_hessian_len(ctx->N);
    VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->hbuf, ctx->hbuf_len));
  }
  return VMAT_OK;
}

extern "C" vmat_status vmat_set_master_precision(vmat_ctx *ctx, int32_t extended) {
  if (!ctx) return VMAT_EINVAL;
  if (extended != 0 && extended != 1)
    return vmat_fail(ctx, VMAT_EINVAL, "master precision must be 0 (FP32) or 1 (extended)");
  if (extended == ctx->master_xp) return VMAT_OK;
  if (ctx->n_slots != 0)
    return vmat_fail(ctx, VMAT_EINVAL, "the plan has columns: call vmat_reset first");
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int old = ctx->master_xp;
  ctx->master_xp = extended;
  vmat_status s = vmat_configure_master(ctx);  // same tiling; checks the variant fits an SM
  if (s == VMAT_OK && extended) s = alloc_xp(ctx);
  if (s != VMAT_OK) {
    ctx->master_xp = old;
    vmat_configure_master(ctx);
    return s;
  }
  if (!extended) free_xp(ctx);
  return vmat_reset(ctx);  // F' of the empty plan in the new form
}

extern "C" vmat_status vmat_set_price_smoothing(vmat_ctx *ctx, int32_t on) {
  if (!ctx) return VMAT_EINVAL;
  if (on != 0 && on != 1) return vmat_fail(ctx, VMAT_EINVAL, "price_smoothing must be 0 or 1");
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->price_smoothing = on;
  return VMAT_OK;
}

extern "C" vmat_status vmat_set_price_path(vmat_ctx *ctx, int32_t path) {
  if (!ctx) return VMAT_EINVAL;
  if (path != VMAT_PRICE_AUTO && path != VMAT_PRICE_ROWS && path != VMAT_PRICE_LIVE)
    return vmat_fail(ctx, VMAT_EINVAL, "price path must be 0 (auto), 1 (rows) or 2 (live voxels)");
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->price_path = path;
  return VMAT_OK;
}

static vmat_status create_impl(const vmat_problem *P, vmat_dtype dt, cudaStream_t st,
                               vmat_ctx *ctx) {
  Tmp tmp;
  ctx->stream = st;
  VMAT_CUDA(ctx, cudaGetDevice(&ctx->device));
  VMAT_CUDA(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  ctx->V = P->n_vox;
  ctx->N = P->n_angles;
  ctx->R = P->n_rows;
  ctx->C = P->n_cols;
  ctx->B = (int64_t)ctx->N * ctx->R * ctx->C;
  ctx->nnz = P->nnz;
  ctx->dt = dt;
  ctx->gamma = P->gamma;
  ctx->cyclic = P->cyclic ? 1 : 0;
  ctx->step = P->max_leaf_step < P->n_cols + 1 ? P->max_leaf_step : P->n_cols + 1;
  ctx->n_struct = P->n_struct;
  const int64_t B = ctx->B, nnz = ctx->nnz;
  const int32_t V = ctx->V;

  // small tables
  std::vector<double> tab(3 * 256, 0.0);
  std::vector<float> tabf(3 * 256, 0.0f);
  for (int q = 0; q < P->n_struct; ++q) {
    tab[q] = P->T[q];
    tab[256 + q] = P->alpha[q];
    tab[512 + q] = P->beta[q];
  }
  for (int q = 0; q < 3 * 256; ++q) tabf[q] = (float)tab[q];
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->tabd, 3 * 256));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->tabf, 3 * 256));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->theta, ctx->N));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->tabd, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, st));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->tabf, tabf.data(), tabf.size() * 4, cudaMemcpyHostToDevice, st));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->theta, P->theta_deg, ctx->N * 8, cudaMemcpyHostToDevice, st));
  ctx->theta_h.assign(P->theta_deg, P->theta_deg + ctx->N);
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->sid_full, V));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->sid_full, P->struct_id, V, cudaMemcpyHostToDevice, st));

  // D upload
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->bm_ptr, B + 1));
  VMAT_CUDA(ctx, cudaMemcpyAsync(ctx->bm_ptr, P->row_ptr, (B + 1) * 8, cudaMemcpyHostToDevice, st));
  int32_t *colv;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &colv, nnz));
  ctx->bm_col = colv;
  VMAT_CUDA(ctx, cudaMemcpyAsync(colv, P->vox_idx, nnz * 4, cudaMemcpyHostToDevice, st));
  size_t vbytes = P->val_dtype == VMAT_F64 ? 8 : 4;
  void *val_in;
  VMAT_CUDA(ctx, tmp.alloc((char **)&val_in, nnz * vbytes));
  VMAT_CUDA(ctx, cudaMemcpyAsync(val_in, P->val, nnz * vbytes, cudaMemcpyHostToDevice, st));

  int *bad;
  VMAT_CUDA(ctx, tmp.alloc(&bad, 1));
  VMAT_CUDA(ctx, cudaMemsetAsync(bad, 0, 4, st));
  unsigned nb = (unsigned)((B + 7) / 8);
  if (P->val_dtype == VMAT_F64)
    k_validate_rows<double><<<nb, 256, 0, st>>>(ctx->bm_ptr, colv, (const double *)val_in, B, V, bad);
  else
    k_validate_rows<float><<<nb, 256, 0, st>>>(ctx->bm_ptr, colv, (const float *)val_in, B, V, bad);
  VMAT_CUDA(ctx, cudaGetLastError());
  int hbad = 0;
  VMAT_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  if (hbad)
    return vmat_fail(ctx, VMAT_EINVAL,
                     "D rows must hold strictly ascending voxels in [0, n_vox) with finite values > 0");

  // active voxels
  int32_t *flag, *excl;
  VMAT_CUDA(ctx, tmp.alloc(&flag, V));
  VMAT_CUDA(ctx, tmp.alloc(&excl, V));
  VMAT_CUDA(ctx, cudaMemsetAsync(flag, 0, (size_t)V * 4, st));
  if (nnz > 0) k_mark_active<<<4 * ctx->num_sms, 256, 0, st>>>(colv, nnz, flag);
  size_t tbytes = 0;
  VMAT_CUDA(ctx, cub::DeviceScan::ExclusiveSum(nullptr, tbytes, flag, excl, V, st));
  void *tst;
  VMAT_CUDA(ctx, tmp.alloc((char **)&tst, tbytes));
  VMAT_CUDA(ctx, cub::DeviceScan::ExclusiveSum(tst, tbytes, flag, excl, V, st));
  int32_t last[2];
  VMAT_CUDA(ctx, cudaMemcpyAsync(&last[0], excl + V - 1, 4, cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaMemcpyAsync(&last[1], flag + V - 1, 4, cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  ctx->Va = last[0] + last[1];
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->vox2act, V));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->act_vox, ctx->Va > 0 ? ctx->Va : 1));
  k_compact<<<(V + 255) / 256, 256, 0, st>>>(flag, excl, V, ctx->vox2act, ctx->act_vox);
  if (nnz > 0) k_remap_cols<<<4 * ctx->num_sms, 256, 0, st>>>(colv, nnz, ctx->vox2act);
  VMAT_CUDA(ctx, cudaGetLastError());

  vmat_status s2;
  if (dt == VMAT_F32) s2 = build_storage<float>(ctx, tmp, colv, val_in, P->val_dtype);
  else if (dt == VMAT_F16) s2 = build_storage<__half>(ctx, tmp, colv, val_in, P->val_dtype);
  else s2 = build_storage<__nv_bfloat16>(ctx, tmp, colv, val_in, P->val_dtype);
  if (s2 != VMAT_OK) return s2;

  // master launch shape fixes the padded voxel count
  vmat_status s3 = vmat_configure_master(ctx);
  if (s3 != VMAT_OK) return s3;

  // constant cost of the voxels D never reaches
  double *part, *sum;
  VMAT_CUDA(ctx, tmp.alloc(&part, 256));
  VMAT_CUDA(ctx, tmp.alloc(&sum, 1));
  k_inactive_cost<<<256, 256, 0, st>>>(ctx->sid_full, ctx->vox2act, V, ctx->tabd, part);
  k_sum_fixed<<<1, 32, 0, st>>>(part, 256, sum);
  VMAT_CUDA(ctx, cudaGetLastError());
  VMAT_CUDA(ctx, cudaMemcpyAsync(&ctx->inactive_cost, sum, 8, cudaMemcpyDeviceToHost, st));

  // plan state and workspaces
  const int N = ctx->N, R = ctx->R;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->occ, N));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->lleaf, (size_t)N * R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->rleaf, (size_t)N * R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->slot_beam, N));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->y, N));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->rho_plan, 1));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->g, B));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->pacc, B));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->pacc, 0, (size_t)B * 8, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->pstat, 6));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->pstat, 0, 48, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->plive, ctx->Va > 0 ? ctx->Va : 1));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->rowsum_max, 1));
  {
    vmat_status sr = vmat_row_sum_max(ctx);
    if (sr != VMAT_OK) return sr;
    sr = vmat_build_beam_offsets(ctx);
    if (sr != VMAT_OK) return sr;
  }
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->xs, B));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->ap_price, N));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->ap_l, (size_t)N * R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->ap_r, (size_t)N * R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->sel, 1));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->sel_l, R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->sel_r, R));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->mout, 1));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->bar, 2));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->mstats, 8));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->mstats, 0, 64, st));
  VMAT_CUDA(ctx, vmat_alloc(ctx, &ctx->dstatus, 1));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->dstatus, 0, 4, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->bar, 0, 8, st));
  vmat_status s4 = alloc_tiled(ctx);
  if (s4 != VMAT_OK) return s4;
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  return vmat_reset(ctx);
}

extern "C" vmat_status vmat_create(const vmat_problem *P, vmat_dtype dt, void *stream,
                                   vmat_ctx **out) {
  if (!out) return vmat_fail(nullptr, VMAT_EINVAL, "out is NULL");
  *out = nullptr;
  if (dt != VMAT_F32 && dt != VMAT_F16 && dt != VMAT_BF16)
    return vmat_fail(nullptr, VMAT_EINVAL, "d_dtype must be VMAT_F32, VMAT_F16 or VMAT_BF16");
  vmat_status s = validate_host(P);
  if (s != VMAT_OK) return s;
  vmat_ctx *ctx = new vmat_ctx();
  s = create_impl(P, dt, (cudaStream_t)stream, ctx);
  if (s != VMAT_OK) {
    g_create_error = ctx->err;
    vmat_destroy(ctx);
    return s;
  }
  *out = ctx;
  return VMAT_OK;
}

extern "C" void vmat_destroy(vmat_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  vmat_free_row_tiles(ctx, ctx->vtiles);
  vmat_free_row_tiles(ctx, ctx->btiles);
  free_xp(ctx);
  void *ptrs[] = {ctx->fa32, ctx->act_vox, ctx->vox2act, ctx->sid_full, ctx->sid, ctx->tabf, ctx->tabd,
                  ctx->theta, ctx->scale, ctx->bm_ptr, ctx->bm_col, ctx->bm_val, ctx->vm_ptr,
                  ctx->vm_col, ctx->vm_val, ctx->M, ctx->tflag, ctx->occ, ctx->lleaf, ctx->rleaf,
                  ctx->slot_beam, ctx->y, ctx->zact, ctx->fpact, ctx->rho_plan, ctx->g,
                  ctx->fgather, ctx->xs, ctx->ap_price, ctx->ap_l, ctx->ap_r, ctx->sel, ctx->sel_l,
                  ctx->sel_r, ctx->red, ctx->mout, ctx->bar, ctx->dstatus, ctx->mstats,
                  ctx->hbuf, ctx->pacc, ctx->pstat, ctx->rowsum_max, ctx->plive, ctx->vm_boff};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete ctx;
}

extern "C" vmat_status vmat_get_info(const vmat_ctx *ctx, vmat_info *out) {
  if (!ctx || !out) return VMAT_EINVAL;
  out->n_vox = ctx->V;
  out->n_active = ctx->Va;
  out->n_angles = ctx->N;
  out->n_rows = ctx->R;
  out->n_cols = ctx->C;
  out->n_beamlets = ctx->B;
  out->nnz = ctx->nnz;
  out->n_columns = ctx->n_slots;
  out->device_bytes = ctx->device_bytes;
  out->d_dtype = ctx->dt;
  out->master_grid = ctx->master_grid;
  out->master_block = ctx->master_block;
  out->n_launches = ctx->n_launches;
  double ms[8] = {0};
  if (ctx->mstats) {
    cudaStreamSynchronize(ctx->stream);
    cudaMemcpy(ms, ctx->mstats, sizeof ms, cudaMemcpyDeviceToHost);
  }
  unsigned long long pc[5] = {0, 0, 0, 0, 0};
  if (ctx->pstat) cudaMemcpy(pc, ctx->pstat, sizeof pc, cudaMemcpyDeviceToHost);
  out->price_calls[0] = (int64_t)pc[2];
  out->price_calls[1] = (int64_t)pc[3];
  out->price_live_entries = (int64_t)pc[4];
  for (int q = 0; q < 4; ++q) out->master_ms[q] = ms[q] * 1e-6;
  out->master_syncs = (int64_t)ms[4];
  out->master_wait_ms = ms[6] * 1e-6;
  out->master_pg_iters = (int64_t)ms[5];
  out->master_rejected = (int64_t)ms[7];
  out->tile_entries[0] = ctx->vtiles.n_union;
  out->tile_entries[1] = ctx->btiles.n_union;
  out->subtile_voxels = ctx->master_block * 4;
  out->n_subtiles = ctx->master_grid * (ctx->master_vpt / 4);
  return VMAT_OK;
}

__global__ void k_init_fprime(const uint8_t *sid, const float *tab, const double *tabd, int32_t Vpad,
                              float *z, float *fp, float *fplo) {
  int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Vpad) return;
  int q = sid[a];
  z[a] = 0.f;
  if (fplo) {  // extended precision: F'(0) = -2 alpha T in FP64, as a float pair
    const double f = -2.0 * tabd[256 + q] * tabd[q];
    fp[a] = (float)f;
    fplo[a] = (float)(f - (double)(float)f);
  } else {
    fp[a] = vmat_dF(0.f, tab[q], tab[256 + q], tab[512 + q]);
  }
}

// Clear the plan state on the context's stream without waiting (usable while
// the stream is being captured into a graph).
vmat_status vmat_enqueue_reset(vmat_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  const int N = ctx->N, R = ctx->R;
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->occ, 0, N, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->tflag, 0, (size_t)N * ctx->master_grid * (ctx->master_vpt / 4) * 4, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->lleaf, 0, (size_t)N * R * 2, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->rleaf, 0, (size_t)N * R * 2, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->slot_beam, 0xff, (size_t)N * 4, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->y, 0, (size_t)N * 8, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->rho_plan, 0, 8, st));
  VMAT_CUDA(ctx, cudaMemsetAsync(ctx->dstatus, 0, 4, st));
  k_init_fprime<<<(ctx->Vpad + 255) / 256, 256, 0, st>>>(ctx->sid, ctx->tabf, ctx->tabd, ctx->Vpad,
                                                          ctx->zact, ctx->fpact,
                                                          ctx->master_xp ? ctx->fplo : nullptr);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  ctx->n_slots = 0;
  return VMAT_OK;
}

extern "C" vmat_status vmat_reset(vmat_ctx *ctx) {
  if (!ctx) return VMAT_EINVAL;
  vmat_status s = vmat_enqueue_reset(ctx);
  if (s != VMAT_OK) return s;
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return VMAT_OK;
}


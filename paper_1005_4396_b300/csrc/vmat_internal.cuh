// Internal declarations of libvmat: device context layout, error handling and
// the bounded grid barrier used by the persistent master kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vmat.h"

#define VMAT_MAX_ANGLES 360
#define VMAT_MAX_ROWS 128
#define VMAT_MAX_COLS 128
#define VMAT_NULL_STRUCT 255  // parameter slot with T = alpha = beta = 0 (padding voxels)

// Per-selection record kept on the device between kernels.
struct SelRec {
  int32_t k;       // chosen beam (-1: none)
  int32_t status;  // 0 ok, VMAT_ESTATE on failure
  double p, p2;    // chosen price, least price of the other free beams
};

// Per-master-solve outputs written by the master kernel.
struct MasterOut {
  double cost_active;  // sum_j F(z_j) over active voxels (FP64)
  double smooth;       // G(y)
  double rho, rho0;
  int32_t iters, status;
};

// Rows [8 t, 8 t + 8) of a CSR as the sorted union of their column indices
// and a dense [|U|][8] value block (0 where a row has no entry); built on
// the first batched product that needs it (tiles.cu).
struct RowTiles {
  int64_t n_tiles = 0, n_union = 0;
  int64_t *uptr = nullptr;  // [n_tiles + 1] first union entry of each tile
  int32_t *ucol = nullptr;  // [n_union] column index
  void *uval = nullptr;     // [n_union][8] values in the storage type of D
};

struct vmat_ctx {
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;

  // sizes
  int32_t V = 0, Va = 0, Vpad = 0, N = 0, R = 0, C = 0, n_struct = 0;
  int64_t B = 0, nnz = 0;
  vmat_dtype dt = VMAT_F32;
  double gamma = 0.0;
  int32_t cyclic = 1, step = 1;
  int32_t price_smoothing = 0;  // 1: pricing adds gamma dG/dy_k (exact reduced cost)
  double inactive_cost = 0.0;  // sum of F(0) over voxels D never reaches

  // problem on the device
  int32_t *act_vox = nullptr;  // [Va] grid index of active voxel a
  int32_t *vox2act = nullptr;  // [V] active index or -1
  uint8_t *sid_full = nullptr; // [V] structure of grid voxel
  uint8_t *sid = nullptr;      // [Vpad] structure of active voxel (padding: VMAT_NULL_STRUCT)
  float *tabf = nullptr;       // [3*256] T, alpha, beta (float)
  double *tabd = nullptr;      // [3*256] T, alpha, beta (double)
  double *theta = nullptr;     // [N]
  std::vector<double> theta_h; // [N] host copy (dose-rate limits between neighbours)
  float *scale = nullptr;      // [B] per-beamlet scale of reduced-precision D (1 for F32)
  int64_t *bm_ptr = nullptr;   // [B+1] beamlet-major CSR over active voxels
  int32_t *bm_col = nullptr;
  void *bm_val = nullptr;
  int64_t *vm_ptr = nullptr;   // [Va+1] voxel-major CSR, rows sorted by beamlet
  uint16_t *vm_boff = nullptr; // [Va][N+1] offset of each beam's entries in its row (or NULL)
  int32_t *vm_col = nullptr;
  void *vm_val = nullptr;

  // plan state
  float *M = nullptr;          // [N][Vpad] aperture-dose columns in order of addition
  float *Mlo = nullptr;        // [N][Vpad] extended precision: each entry minus its FP32 value
  int32_t *tflag = nullptr;    // [N][master_grid*vpt/4] 1 if column s is nonzero in master subtile
  uint8_t *occ = nullptr;      // [N]
  int16_t *lleaf = nullptr, *rleaf = nullptr;  // [N*R]
  int32_t *slot_beam = nullptr;                // [N]
  int32_t n_slots = 0;                         // host mirror of the column count
  double *y = nullptr;         // [N]
  float *zact = nullptr;       // [Vpad] plan dose on active voxels
  float *fpact = nullptr;      // [Vpad] F'(z) of the plan dose
  float *fplo = nullptr;       // [Vpad] extended precision: F' minus its FP32 value
  double *rho_plan = nullptr;  // [1] residual at the start of the plan's first master solve

  // workspaces
  float *g = nullptr;          // [B] beamlet prices
  float *fgather = nullptr;    // [Vpad] caller vector gathered onto active voxels
  float *xs = nullptr;         // [B] scaled fluence for reduced-precision dose
  float *fa32 = nullptr;       // [Va*32] batched adjoint input on active voxels (lazy)
  RowTiles vtiles, btiles;     // row tiles of the voxel-major and beamlet-major CSR (lazy)
  double *ap_price = nullptr;  // [N] best aperture price per beam
  int16_t *ap_l = nullptr, *ap_r = nullptr;  // [N*R] best leaves per beam
  SelRec *sel = nullptr;       // [1]
  int16_t *sel_l = nullptr, *sel_r = nullptr;  // [R]
  double *red = nullptr;       // reduction scratch [red_len]
  int64_t red_len = 0;
  MasterOut *mout = nullptr;   // [1]
  unsigned *bar = nullptr;     // [2] grid barrier word (+ spare)
  double *mstats = nullptr;    // [8] cumulative master-kernel phase ns, grid syncs, iterations
  int *dstatus = nullptr;      // [1] sticky device error (VMAT_ETIMEOUT, ...)

  // master launch shape
  int master_grid = 0, master_block = 0, master_vpt = 0;
  size_t master_smem = 0;
  int64_t device_bytes = 0;
  int64_t n_launches = 0;      // kernels launched by this context
  int profiling = 0;
  int sm_budget = 0;           // master kernel CTA budget (0: every SM)
  int master_method = 0;       // VMAT_MASTER_PROJECTED_GRADIENT or _NEWTON
  int master_xp = 0;           // 1: extended-precision master (float-pair dose excess and F')
  size_t master_smem_pn = 0;   // shared memory of the projected-Newton variant
  float *hbuf = nullptr;       // projected Newton: [grid + 1][(N+1)(N+2)/2] Gram partials + sum
  int64_t hbuf_len = 0;
  // live-voxel prices (spmv.cu)
  int price_path = VMAT_PRICE_AUTO;
  unsigned long long *pacc = nullptr;  // [B] fixed-point price accumulators, zero between calls
  unsigned long long *pstat = nullptr; // [6] max|f| bits, live entries (per call); live-form
                                       // calls, calls, live entries read (cumulative); live rows
  int32_t *plive = nullptr;            // [Va] live rows of the current call
  double *rowsum_max = nullptr;        // [1] largest row sum of Dhat
};

// ---------------------------------------------------------------- helpers
vmat_status vmat_fail(vmat_ctx *ctx, vmat_status st, const char *fmt, ...);
vmat_status vmat_cuda_fail(vmat_ctx *ctx, cudaError_t e, const char *what);

#define VMAT_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return vmat_cuda_fail(ctx, e_, #call); \
  } while (0)

template <typename T>
inline cudaError_t vmat_alloc(vmat_ctx *ctx, T **p, size_t n) {
  size_t bytes = n * sizeof(T) > 0 ? n * sizeof(T) : 16;
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e == cudaSuccess) ctx->device_bytes += (int64_t)bytes;
  return e;
}

__device__ __forceinline__ unsigned long long vmat_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Voxel cost pieces of Eq. 1 in single precision (derivative) and double (cost).
__device__ __forceinline__ float vmat_dF(float z, float T, float a, float b) {
  float e = z - T;
  return e > 0.f ? 2.f * b * e : (e < 0.f ? 2.f * a * e : 0.f);
}
__device__ __forceinline__ double vmat_F(double z, double T, double a, double b) {
  double e = z - T;
  return e > 0.0 ? b * e * e : a * e * e;
}

// Value loads of D in its storage type, as float.
__device__ __forceinline__ float vmat_ld(const float *p, int64_t e) { return __ldg(p + e); }
__device__ __forceinline__ float vmat_ld(const __half *p, int64_t e) { return __half2float(p[e]); }
__device__ __forceinline__ float vmat_ld(const __nv_bfloat16 *p, int64_t e) {
  return __bfloat162float(p[e]);
}

// Launchers implemented in the .cu files.
vmat_status vmat_launch_price(vmat_ctx *ctx, const float *f_act, const uint8_t *mask, int mode,
                              float *g, const float *f_lo = nullptr);
vmat_status vmat_gather_active(vmat_ctx *ctx, const float *full, float *act);
vmat_status vmat_row_sum_max(vmat_ctx *ctx);
vmat_status vmat_build_beam_offsets(vmat_ctx *ctx);
vmat_status vmat_launch_dose(vmat_ctx *ctx, const float *x, float *z_full, float *fp_full,
                             double *cost_dev);
vmat_status vmat_launch_pricing(vmat_ctx *ctx, const float *g);
vmat_status vmat_launch_add_column(vmat_ctx *ctx, int slot, int32_t *rec_subtiles = nullptr);
vmat_status vmat_launch_master(vmat_ctx *ctx, int max_iters, double kkt_tol, double rho_ref,
                               int set_rho_plan, double *rec_cost, double *rec_rho,
                               int32_t *rec_iters, int32_t *rec_status);
vmat_status vmat_launch_dose_batch32(vmat_ctx *ctx, const float *X, float *Z, float *Fp,
                                     double *cost_dev);
vmat_status vmat_launch_price_batch32(vmat_ctx *ctx, const float *Fp, const float *colw, float *G);
vmat_status vmat_configure_master(vmat_ctx *ctx);
vmat_status vmat_ensure_row_tiles(vmat_ctx *ctx, bool voxel_major);
void vmat_free_row_tiles(vmat_ctx *ctx, RowTiles &t);
int64_t vmat_master_scratch(int grid, int N);
int64_t vmat_hessian_len(int N);
vmat_status vmat_enqueue_reset(vmat_ctx *ctx);

// Device-resident per-iteration records of a column-generation run.
struct Records {
  int32_t *k, *iters, *status, *tiles;
  double *p, *p2, *cost, *rho;
};
// Enqueue n column-generation iterations on ctx->stream without any host
// synchronisation or allocation (safe inside a stream capture).
vmat_status vmat_enqueue_colgen(vmat_ctx *ctx, int n, int master_max_iters, double kkt_tol,
                                const Records &rec, bool fresh);

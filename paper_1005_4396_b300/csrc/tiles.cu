// Row-tiled copies of the two CSR forms of D for the batched products over 32
// vectors (the differentiable forward and its adjoint, Eq. 1-3).
//
// Every nonzero of a CSR row gathers a whole 128-byte row of the dense
// operand (32 vectors).  Neighbouring rows share most of their column
// indices: consecutive active voxels are crossed by the same beamlets, and
// neighbouring beamlets of a leaf row pass through the same voxels.  A tile
// holds 8 consecutive rows as the sorted union U of their column indices and
// a dense [|U|][8] block of values (0 where a row has no entry), so one
// gathered row of the dense operand serves all 8 rows of the tile.  A row
// visits its own columns in the same ascending order as in the CSR, and
// a zero entry adds exactly 0, so each row's FP32 sum is the CSR kernel's
// sum term for term.
//
// Built on the device by one pass that counts |U| per tile, a scan, and one
// pass that writes U and the values: 8 lanes of a warp walk the 8 rows of a
// tile together, and each step emits the least column index at the heads
// of the rows.
#include <climits>

#include <cub/cub.cuh>

#include "vmat_internal.cuh"

#define TILE_ROWS 8

template <typename TV>
__device__ __forceinline__ TV tv_zero();
template <>
__device__ __forceinline__ float tv_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ __half tv_zero<__half>() { return __float2half(0.f); }
template <>
__device__ __forceinline__ __nv_bfloat16 tv_zero<__nv_bfloat16>() { return __float2bfloat16(0.f); }

// One warp walks 4 tiles (lanes 8g..8g+7 are the rows of tile g).  fill = 0:
// count[t] = |U| of tile t; fill = 1: write U and the value block from uptr.
template <typename TV>
__global__ void __launch_bounds__(256) k_tile_union(const int64_t *__restrict__ ptr,
                                                    const int32_t *__restrict__ col,
                                                    const TV *__restrict__ val, int64_t n_rows,
                                                    int64_t n_tiles, int fill, int64_t *count,
                                                    const int64_t *__restrict__ uptr,
                                                    int32_t *__restrict__ ucol, TV *__restrict__ uval) {
  const int lane = threadIdx.x & 31, g = lane >> 3, r = lane & 7;
  const int64_t tile = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4 + g;
  const int64_t row = tile * TILE_ROWS + r;
  int64_t p = 0, end = 0;
  if (tile < n_tiles && row < n_rows) {
    p = ptr[row];
    end = ptr[row + 1];
  }
  int64_t pos = (fill && tile < n_tiles) ? uptr[tile] : 0;
  int64_t cnt = 0;
  for (;;) {
    const int head = p < end ? col[p] : INT_MAX;
    int m = head;
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 1));
    const bool active = m != INT_MAX;  // the same in the 8 lanes of a tile
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      if (fill) {
        if (r == 0) ucol[pos] = m;
        uval[pos * TILE_ROWS + r] = head == m ? val[p] : tv_zero<TV>();
        ++pos;
      }
      ++cnt;
      if (head == m) ++p;
    }
  }
  if (!fill && r == 0 && tile < n_tiles) count[tile] = cnt;
}

template <typename TV>
static vmat_status build_one(vmat_ctx *ctx, const int64_t *ptr, const int32_t *col, const void *val,
                             int64_t n_rows, RowTiles &t) {
  cudaStream_t st = ctx->stream;
  const int64_t nt = (n_rows + TILE_ROWS - 1) / TILE_ROWS;
  t.n_tiles = nt;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &t.uptr, (size_t)nt + 1));
  const unsigned nb = (unsigned)((nt + 31) / 32 > 0 ? (nt + 31) / 32 : 1);  // 8 warps x 4 tiles
  k_tile_union<TV><<<nb, 256, 0, st>>>(ptr, col, (const TV *)val, n_rows, nt, 0, t.uptr, nullptr,
                                       nullptr, nullptr);
  VMAT_CUDA(ctx, cudaGetLastError());
  size_t tbytes = 0;
  VMAT_CUDA(ctx, cub::DeviceScan::ExclusiveSum(nullptr, tbytes, t.uptr, t.uptr, (int)(nt + 1), st));
  void *tmp = nullptr;
  VMAT_CUDA(ctx, cudaMallocAsync(&tmp, tbytes > 0 ? tbytes : 16, st));
  // the count of the last (phantom) entry is zeroed so the scan's last value is the total
  VMAT_CUDA(ctx, cudaMemsetAsync(t.uptr + nt, 0, 8, st));
  VMAT_CUDA(ctx, cub::DeviceScan::ExclusiveSum(tmp, tbytes, t.uptr, t.uptr, (int)(nt + 1), st));
  cudaFreeAsync(tmp, st);
  int64_t total = 0;
  VMAT_CUDA(ctx, cudaMemcpyAsync(&total, t.uptr + nt, 8, cudaMemcpyDeviceToHost, st));
  VMAT_CUDA(ctx, cudaStreamSynchronize(st));
  t.n_union = total;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &t.ucol, (size_t)(total > 0 ? total : 1)));
  TV *uv = nullptr;
  VMAT_CUDA(ctx, vmat_alloc(ctx, &uv, (size_t)(total > 0 ? total : 1) * TILE_ROWS));
  t.uval = uv;
  k_tile_union<TV><<<nb, 256, 0, st>>>(ptr, col, (const TV *)val, n_rows, nt, 1, nullptr, t.uptr,
                                       t.ucol, uv);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 2;
  return VMAT_OK;
}

// Builds the voxel-major (dose) or beamlet-major (price) tiles if missing.
vmat_status vmat_ensure_row_tiles(vmat_ctx *ctx, bool voxel_major) {
  RowTiles &t = voxel_major ? ctx->vtiles : ctx->btiles;
  if (t.uptr) return VMAT_OK;
  const int64_t *ptr = voxel_major ? ctx->vm_ptr : ctx->bm_ptr;
  const int32_t *col = voxel_major ? ctx->vm_col : ctx->bm_col;
  const void *val = voxel_major ? ctx->vm_val : ctx->bm_val;
  const int64_t rows = voxel_major ? ctx->Va : ctx->B;
  vmat_status s;
  if (ctx->dt == VMAT_F32) s = build_one<float>(ctx, ptr, col, val, rows, t);
  else if (ctx->dt == VMAT_F16) s = build_one<__half>(ctx, ptr, col, val, rows, t);
  else s = build_one<__nv_bfloat16>(ctx, ptr, col, val, rows, t);
  if (s != VMAT_OK) vmat_free_row_tiles(ctx, t);
  return s;
}

void vmat_free_row_tiles(vmat_ctx *ctx, RowTiles &t) {
  const size_t vb = ctx->dt == VMAT_F32 ? 4 : 2;
  if (t.uptr) ctx->device_bytes -= (int64_t)((t.n_tiles + 1) * 8);
  if (t.ucol) ctx->device_bytes -= (int64_t)((t.n_union > 0 ? t.n_union : 1) * 4);
  if (t.uval) ctx->device_bytes -= (int64_t)((t.n_union > 0 ? t.n_union : 1) * TILE_ROWS * vb);
  cudaFree(t.uptr);
  cudaFree(t.ucol);
  cudaFree(t.uval);
  t = RowTiles();
}

// Plan quality on the GPU: dose-volume histograms per structure (the
// evaluation behind the paper's Fig. 2), not part of the optimisation.
//
// k_dvh: one pass over the V voxels of a dose vector; each CTA counts into a
// shared-memory histogram [n_struct][n_bins] (32-bit integer atomics), then
// adds its counts to the global 64-bit histogram.  Integer sums do not
// depend on their order, so the counts are exact and reproducible.  A
// voxel's bin is floor(z * s) in FP32 with s = n_bins / dose_max (rounded to
// FP32 once), clamped to [0, n_bins - 1]: the last bin also holds doses at
// or above dose_max.
#include "vmat_internal.cuh"

__global__ void __launch_bounds__(256) k_dvh(const float *__restrict__ z, const uint8_t *__restrict__ sid,
                                             int32_t V, int n_struct, int n_bins, float scale,
                                             unsigned long long *__restrict__ hist) {
  extern __shared__ unsigned s_h[];  // [n_struct * n_bins]
  const int nh = n_struct * n_bins;
  for (int q = threadIdx.x; q < nh; q += blockDim.x) s_h[q] = 0u;
  __syncthreads();
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < V; j += gridDim.x * blockDim.x) {
    const float v = __fmul_rn(z[j], scale);
    int b = v > 0.f ? (int)v : 0;  // truncation = floor for non-negative values
    if (b > n_bins - 1) b = n_bins - 1;
    atomicAdd(&s_h[sid[j] * n_bins + b], 1u);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nh; q += blockDim.x)
    if (s_h[q]) atomicAdd(hist + q, (unsigned long long)s_h[q]);
}

extern "C" vmat_status vmat_dvh(vmat_ctx *ctx, const float *z_dev, double dose_max, int32_t n_bins,
                                int64_t *counts_host) {
  if (!ctx) return VMAT_EINVAL;
  if (!z_dev || !counts_host || !(dose_max > 0.0) || !isfinite(dose_max) || n_bins < 1 || n_bins > 4096)
    return vmat_fail(ctx, VMAT_EINVAL, "z and counts required, dose_max > 0, 1 <= n_bins <= 4096");
  const int ns = ctx->n_struct;
  const size_t nh = (size_t)ns * n_bins, smem = nh * 4;
  if (smem > 96 * 1024)
    return vmat_fail(ctx, VMAT_EINVAL, "n_struct x n_bins = %zu exceeds the shared-memory histogram", nh);
  unsigned long long *h = nullptr;
  VMAT_CUDA(ctx, cudaMallocAsync((void **)&h, nh * 8, ctx->stream));
  VMAT_CUDA(ctx, cudaMemsetAsync(h, 0, nh * 8, ctx->stream));
  VMAT_CUDA(ctx, cudaFuncSetAttribute(k_dvh, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = ctx->num_sms * 4;
  k_dvh<<<grid, 256, smem, ctx->stream>>>(z_dev, ctx->sid_full, ctx->V, ns, n_bins,
                                          (float)(n_bins / dose_max), h);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts_host, h, nh * 8, cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(h, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return vmat_cuda_fail(ctx, e, "dvh");
  ctx->n_launches += 1;
  return VMAT_OK;
}

// Aperture maps and the smoothing term for 32 intensity vectors at once: the
// pieces of the differentiable forward z = D^T (A y) with cost
// sum_j F(z_j) + gamma G(y) (Eq. 1-3) that sit around the sparse products.
//
//   fluence   X[i][b] = Y[k(i)][b] if column c(i) of row r(i) is open in beam
//             k(i) (l <= c < r), else 0                         (x = A y)
//   adjoint   GY[k][b] = sum over open beamlets i of beam k of GX[i][b]  (A^T)
//   smoothing G_b = sum_pairs (Y[k+1][b] - Y[k][b])^2 / gap, and dG/dY (Eq. 2)
// Vectors are row-major [rows][32]: lane b of a warp owns vector b.
#include "vmat_internal.cuh"

__global__ void k_fluence32(const int16_t *__restrict__ l, const int16_t *__restrict__ r,
                            const float *__restrict__ Y, int R, int C, int64_t B,
                            float *__restrict__ X) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 32) return;
  const int64_t i = t >> 5;
  const int b = (int)(t & 31);
  const int64_t RC = (int64_t)R * C;
  const int k = (int)(i / RC), row = (int)((i % RC) / C), c = (int)(i % C);
  const int kr = k * R + row;
  X[t] = (c >= l[kr] && c < r[kr]) ? Y[(int64_t)k * 32 + b] : 0.f;
}

// one warp per beam; lanes = vectors; rows then columns in order.  With Y,
// adds gamma * w_b * dG/dY[k][b] (the smoothing term's gradient, Eq. 2).
__global__ void k_adjoint32(const int16_t *__restrict__ l, const int16_t *__restrict__ r,
                            const float *__restrict__ GX, int N, int R, int C,
                            const float *__restrict__ Y, const float *__restrict__ w,
                            const double *__restrict__ theta, int cyclic, double gamma,
                            float *__restrict__ GY) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int b = threadIdx.x & 31;
  if (k >= N) return;
  float acc = 0.f;
  for (int row = 0; row < R; ++row) {
    const int kr = k * R + row;
    const int64_t base = ((int64_t)k * R + row) * C;
    for (int c = l[kr]; c < r[kr]; ++c) acc += GX[(base + c) * 32 + b];
  }
  if (Y) {
    double v = 0.0;
    const double yk = Y[(int64_t)k * 32 + b];
    if (k > 0 || cyclic) {
      const int km = k > 0 ? k - 1 : N - 1;
      const double gap = k > 0 ? theta[k] - theta[km] : theta[0] + 360.0 - theta[N - 1];
      v += 2.0 * (yk - (double)Y[(int64_t)km * 32 + b]) / gap;
    }
    if (k < N - 1 || cyclic) {
      const int kp = k < N - 1 ? k + 1 : 0;
      const double gap = k < N - 1 ? theta[kp] - theta[k] : theta[0] + 360.0 - theta[N - 1];
      v -= 2.0 * ((double)Y[(int64_t)kp * 32 + b] - yk) / gap;
    }
    acc += (float)(gamma * v * (w ? (double)w[b] : 1.0));
  }
  GY[(int64_t)k * 32 + b] = acc;
}

// one warp: lane b computes G of vector b (FP64) and dG/dY[k][b]
__global__ void k_smooth32(const float *__restrict__ Y, const double *__restrict__ theta, int N,
                           int cyclic, double *__restrict__ Gout, float *__restrict__ dG) {
  const int b = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double g = 0.0;
  const int npair = cyclic ? N : N - 1;
  for (int k = 0; k < npair; ++k) {
    const int kp = k + 1 < N ? k + 1 : 0;
    const double gap = k + 1 < N ? theta[kp] - theta[k] : theta[0] + 360.0 - theta[N - 1];
    const double d = (double)Y[(int64_t)kp * 32 + b] - (double)Y[(int64_t)k * 32 + b];
    g += d * d / gap;
  }
  Gout[b] = g;
  if (dG)
    for (int k = 0; k < N; ++k) {
      double v = 0.0;
      const double yk = Y[(int64_t)k * 32 + b];
      if (k > 0 || cyclic) {
        const int km = k > 0 ? k - 1 : N - 1;
        const double gap = k > 0 ? theta[k] - theta[km] : theta[0] + 360.0 - theta[N - 1];
        v += 2.0 * (yk - (double)Y[(int64_t)km * 32 + b]) / gap;
      }
      if (k < N - 1 || cyclic) {
        const int kp = k < N - 1 ? k + 1 : 0;
        const double gap = k < N - 1 ? theta[kp] - theta[k] : theta[0] + 360.0 - theta[N - 1];
        v -= 2.0 * ((double)Y[(int64_t)kp * 32 + b] - yk) / gap;
      }
      dG[(int64_t)k * 32 + b] = (float)v;
    }
}

static vmat_status check_leaves(vmat_ctx *ctx, const int16_t *l, const int16_t *r) {
  if (!l || !r) return vmat_fail(ctx, VMAT_EINVAL, "leaves are NULL");
  return VMAT_OK;
}

static vmat_status finish(vmat_ctx *ctx, int launches) {
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += launches;
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return VMAT_OK;
}

extern "C" vmat_status vmat_aperture_fluence_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                     const int16_t *r_dev, const float *Y_dev,
                                                     float *X_dev) {
  if (!ctx || !Y_dev || !X_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = check_leaves(ctx, l_dev, r_dev);
  if (s != VMAT_OK) return s;
  const int64_t n = ctx->B * 32;
  k_fluence32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(l_dev, r_dev, Y_dev, ctx->R,
                                                                     ctx->C, ctx->B, X_dev);
  return finish(ctx, 1);
}

extern "C" vmat_status vmat_aperture_adjoint_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                     const int16_t *r_dev, const float *GX_dev,
                                                     const float *Y_dev, const float *w_dev,
                                                     float *GY_dev) {
  if (!ctx || !GX_dev || !GY_dev) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = check_leaves(ctx, l_dev, r_dev);
  if (s != VMAT_OK) return s;
  k_adjoint32<<<(ctx->N + 7) / 8, 256, 0, ctx->stream>>>(l_dev, r_dev, GX_dev, ctx->N, ctx->R,
                                                         ctx->C, Y_dev, w_dev, ctx->theta,
                                                         ctx->cyclic, ctx->gamma, GY_dev);
  return finish(ctx, 1);
}

extern "C" vmat_status vmat_smoothing_batch32(vmat_ctx *ctx, const float *Y_dev, double *G_host,
                                              float *dG_dev) {
  if (!ctx || !Y_dev || !G_host) return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  double *gdev = ctx->red + ctx->red_len - 32;
  k_smooth32<<<1, 32, 0, ctx->stream>>>(Y_dev, ctx->theta, ctx->N, ctx->cyclic, gdev, dG_dev);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  VMAT_CUDA(ctx, cudaMemcpyAsync(G_host, gdev, 32 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return VMAT_OK;
}

// Eq. 3 for 32 intensity vectors on fixed apertures: X = A Y, Z = D^T X with
// F'(Z), and cost_b = sum_j F(Z_jb) (FP64) + gamma * G(Y_b) (FP64, Eq. 2),
// the two parts added here in FP64.
extern "C" vmat_status vmat_aperture_dose_cost_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                       const int16_t *r_dev, const float *Y_dev,
                                                       float *X_dev, float *Z_dev,
                                                       float *fprime_dev, double *cost_host) {
  if (!ctx || !Y_dev || !X_dev || !Z_dev || !cost_host)
    return ctx ? vmat_fail(ctx, VMAT_EINVAL, "NULL argument") : VMAT_EINVAL;
  vmat_status s = check_leaves(ctx, l_dev, r_dev);
  if (s != VMAT_OK) return s;
  const int64_t n = ctx->B * 32;
  k_fluence32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(l_dev, r_dev, Y_dev, ctx->R,
                                                                     ctx->C, ctx->B, X_dev);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  double *cdev = ctx->red + ctx->red_len - 64;  // [0, 32): voxel cost, [32, 64): G
  s = vmat_launch_dose_batch32(ctx, X_dev, Z_dev, fprime_dev, cdev);
  if (s != VMAT_OK) return s;
  k_smooth32<<<1, 32, 0, ctx->stream>>>(Y_dev, ctx->theta, ctx->N, ctx->cyclic, cdev + 32, nullptr);
  VMAT_CUDA(ctx, cudaGetLastError());
  ctx->n_launches += 1;
  double h[64];
  VMAT_CUDA(ctx, cudaMemcpyAsync(h, cdev, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  VMAT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int b = 0; b < 32; ++b) cost_host[b] = h[b] + ctx->inactive_cost + ctx->gamma * h[32 + b];
  return VMAT_OK;
}

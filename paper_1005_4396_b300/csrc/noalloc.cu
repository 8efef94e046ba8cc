// Dose and voxel cost for callers that may not allocate device memory.
//
// Some hosts cannot let a library call cudaMalloc: a framework that owns a
// fixed device-memory pool and forbids driver allocations behind its back, a
// planning service that must not allocate while serving requests, or an
// embedded/real-time integration that sizes all memory up front.  For them
// this file offers one dose + cost entry point that needs no context and no
// allocation: the caller passes the voxel-major D, the fluence and the
// outputs; the only scratch (one FP64 partial cost per thread block, reduced
// in a fixed order) lives in a file-scope __device__ array that every GPU
// loading the library holds until the process exits.
#include <mutex>

#include "vmat_internal.cuh"

#define NOALLOC_ROWS_PER_BLOCK 8
#define NOALLOC_MAX_BLOCKS 65536  // 512 KiB of FP64 partials
#define NOALLOC_MAX_ROWS (NOALLOC_ROWS_PER_BLOCK * NOALLOC_MAX_BLOCKS)
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

// Device address of the scratch array, looked up once per device (with that
// device current) and cached; the host-side name of the array is only a
// stand-in and must never be passed to a kernel.  The cache lives as long as
// the process: a cudaDeviceReset gives the device a new context in which the
// cached address is no longer valid, so a process that resets a device must
// not call this entry point on it afterwards.
static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

static vmat_status noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vmat_cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return vmat_fail(nullptr, VMAT_EINVAL, "device index %d beyond %d", dev, NOALLOC_MAX_DEVICES);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
    if (e != cudaSuccess) return vmat_cuda_fail(nullptr, e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return VMAT_OK;
}

// One warp per voxel row: z_j = sum_e val[e] x[col[e]], then F'(z_j) and the
// block's FP64 partial of sum_j F(z_j) (Eq. 1) into partials[blockIdx.x].
__global__ void __launch_bounds__(256) k_dose_noalloc(
    int32_t n_vox, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, const uint8_t *__restrict__ sid,
    const double *__restrict__ prm, int32_t n_struct, float *__restrict__ z,
    float *__restrict__ fp, double *__restrict__ partials) {
  __shared__ double s_cost[NOALLOC_ROWS_PER_BLOCK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t j = blockIdx.x * NOALLOC_ROWS_PER_BLOCK + warp;
  double c = 0.0;
  if (j < n_vox) {
    const int64_t e0 = ptr[j], e1 = ptr[j + 1];
    float acc = 0.f;
    for (int64_t e = e0 + lane; e < e1; e += 32) acc = fmaf(val[e], __ldg(x + col[e]), acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int q = sid[j];
      if (z) z[j] = acc;
      if (q < n_struct) {
        const double T = prm[q], al = prm[n_struct + q], be = prm[2 * n_struct + q];
        if (fp) fp[j] = vmat_dF(acc, (float)T, (float)al, (float)be);
        c = vmat_F((double)acc, T, al, be);
      } else {  // structure id beyond params: flag the voxel, read nothing
        if (fp) fp[j] = __int_as_float(0x7fc00000);
        c = __longlong_as_double(0x7ff8000000000000ll);
      }
    }
  }
  if (lane == 0) s_cost[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < NOALLOC_ROWS_PER_BLOCK; ++q) s += s_cost[q];
    partials[blockIdx.x] = s;  // every block writes its own slot: nothing to clear
  }
}

__global__ void k_sum_noalloc(const double *__restrict__ partials, int n, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += partials[q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

extern "C" vmat_status vmat_dose_cost_noalloc(int32_t n_vox, const int64_t *row_ptr_dev,
                                              const int32_t *beamlet_dev, const float *val_dev,
                                              const float *x_dev, const uint8_t *struct_id_dev,
                                              const double *params_dev, int32_t n_struct,
                                              float *z_dev, float *fprime_dev, double *cost_dev,
                                              void *cuda_stream) {
  if (n_vox <= 0 || n_vox > NOALLOC_MAX_ROWS)
    return vmat_fail(nullptr, VMAT_EINVAL,
                     "vmat_dose_cost_noalloc: n_vox must be in [1, %d] (static scratch of %d "
                     "partial sums); use vmat_dose for larger grids",
                     NOALLOC_MAX_ROWS, NOALLOC_MAX_BLOCKS);
  if (n_struct <= 0 || n_struct > 256)
    return vmat_fail(nullptr, VMAT_EINVAL, "vmat_dose_cost_noalloc: n_struct must be in [1, 256]");
  if (!row_ptr_dev || !beamlet_dev || !val_dev || !x_dev || !struct_id_dev || !params_dev ||
      !cost_dev)
    return vmat_fail(nullptr, VMAT_EINVAL, "vmat_dose_cost_noalloc: NULL argument");
  double *partials = nullptr;
  vmat_status s = noalloc_scratch(&partials);
  if (s != VMAT_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = (n_vox + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK;
  k_dose_noalloc<<<nb, 32 * NOALLOC_ROWS_PER_BLOCK, 0, st>>>(n_vox, row_ptr_dev, beamlet_dev,
                                                             val_dev, x_dev, struct_id_dev,
                                                             params_dev, n_struct, z_dev,
                                                             fprime_dev, partials);
  k_sum_noalloc<<<1, 256, 0, st>>>(partials, nb, cost_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vmat_cuda_fail(nullptr, e, "vmat_dose_cost_noalloc launch");
  return VMAT_OK;
}

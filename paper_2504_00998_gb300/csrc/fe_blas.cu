// Deterministic double-precision vector kernels used by the Lanczos and CG loops.
// Reductions use a fixed grid and a fixed two-stage order, so repeated runs give
// bitwise-identical results.
#include "fe_internal.h"
#include "fe_blas.cuh"

namespace fe {

__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y,
                              int64_t n, int64_t incx, double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)RED_BLOCKS * RED_THREADS)
    s = fma(x[i * incx], y[i * incx], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_partial(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double sh[RED_BLOCKS];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

fe_status dot_async(const double* x, const double* y, int64_t n, int64_t inc, double* part,
                    double* out, cudaStream_t st) {
  k_dot_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(x, y, n, inc, part); fe_count_launch();
  k_sum_partial<<<1, RED_BLOCKS, 0, st>>>(part, RED_BLOCKS, out); fe_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "dot: %s", cudaGetErrorString(e));
  return FE_OK;
}

fe_status sum_async(const double* part, int n, double* out, cudaStream_t st) {
  k_sum_partial<<<1, RED_BLOCKS, 0, st>>>(part, n, out); fe_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "sum: %s", cudaGetErrorString(e));
  return FE_OK;
}

}  // namespace fe

fe_status fe_dot(fe_mesh* m, const double* x, const double* y, int64_t n, double* out_dev) {
  void* part;
  FE_TRY(fe_ws(m, WS_RED, sizeof(double) * fe::RED_BLOCKS * 4, &part));
  return fe::dot_async(x, y, n, 1, (double*)part, out_dev, m->stream);
}

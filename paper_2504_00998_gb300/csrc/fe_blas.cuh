// Small deterministic vector helpers shared by the iterative drivers.
#pragma once

#include "fe_internal.h"

namespace fe {

constexpr int RED_BLOCKS = 512;
constexpr int RED_THREADS = 256;

// out_dev = sum_i x[i*inc] y[i*inc]; part holds RED_BLOCKS doubles
fe_status dot_async(const double* x, const double* y, int64_t n, int64_t inc, double* part,
                    double* out, cudaStream_t st);

// out_dev = sum of n (<= RED_BLOCKS) block partials
fe_status sum_async(const double* part, int n, double* out, cudaStream_t st);

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace fe

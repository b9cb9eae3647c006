// Instantiations of the tensor-product operator kernel: float storage, 1-element chunks,
// 1 chunk(s) per node in a tile (single-vector operator of the mixed-precision Poisson solve).
#include "fe_kron.cuh"

namespace fe {

fe_status kron_k1f(const KronCoef& cf, const KronGeom& g, const KronIO<float>& io, cudaStream_t st) {
  return kron_dispatch<float, 1, 1>(cf, g, io, st);
}

}  // namespace fe

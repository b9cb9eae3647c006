// Instantiations of the tensor-product operator kernel: double storage, 1-element chunks,
// 1 chunk(s) per node in a tile.
#include "fe_kron.cuh"

namespace fe {

fe_status kron_k1(const KronCoef& cf, const KronGeom& g, const KronIO<double>& io, cudaStream_t st) {
  return kron_dispatch<double, 1, 1>(cf, g, io, st);
}

}  // namespace fe

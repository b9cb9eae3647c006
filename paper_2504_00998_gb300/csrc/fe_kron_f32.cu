// Instantiations of the tensor-product operator kernel: float storage, 4-element chunks,
// 2 chunk(s) per node in a tile.
#include "fe_kron.cuh"

namespace fe {

fe_status kron_f32(const KronCoef& cf, const KronGeom& g, const KronIO<float>& io, cudaStream_t st) {
  return kron_dispatch<float, 4, 2>(cf, g, io, st);
}

int64_t kron_batch_plan_f32(int p, KronInst<float>* inst, int n, int zseg_req) {
  return kron_batch_plan_dispatch<float, 4, 2>(p, inst, n, zseg_req);
}

fe_status kron_batch_f32(const KronCoef& cf, int p, const KronInst<float>* d_inst, int n,
                         int64_t total_ctas, bool use_z, bool full, cudaStream_t st, unsigned long long* counter) {
  return kron_batch_dispatch<float, 4, 2>(cf, p, d_inst, n, total_ctas, use_z, full, st, counter);
}

}  // namespace fe

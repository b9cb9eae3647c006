// Instantiations of the tensor-product operator kernel: double storage, 2-element chunks,
// 2 chunk(s) per node in a tile.
#include "fe_kron.cuh"

namespace fe {

fe_status kron_f64(const KronCoef& cf, const KronGeom& g, const KronIO<double>& io, cudaStream_t st) {
  return kron_dispatch<double, 2, 2>(cf, g, io, st);
}

int64_t kron_batch_plan_f64(int p, KronInst<double>* inst, int n, int zseg_req) {
  return kron_batch_plan_dispatch<double, 2, 2>(p, inst, n, zseg_req);
}

fe_status kron_batch_f64(const KronCoef& cf, int p, const KronInst<double>* d_inst, int n,
                         int64_t total_ctas, bool use_z, bool full, cudaStream_t st, unsigned long long* counter) {
  return kron_batch_dispatch<double, 2, 2>(cf, p, d_inst, n, total_ctas, use_z, full, st, counter);
}

}  // namespace fe

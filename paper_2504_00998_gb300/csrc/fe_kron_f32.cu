// Instantiations of the tensor-product operator kernel: float storage, 4-element chunks.
#include "fe_kron.cuh"

namespace fe {

fe_status kron_f32(const KronCoef& cf, const KronGeom& g, const KronIO<float>& io, int nch,
                  cudaStream_t st) {
  const int nitems = g.bx * g.p * g.by * g.p * nch;
  const int ipt = nitems <= 512 ? 1 : (nitems <= 1024 ? 2 : 4);  // at most 512 threads
  if (nitems > 2048) return fe_fail(FE_EINVAL, "tile of %d items exceeds one CTA", nitems);
#define FE_K(P_)                                                         \
  case P_:                                                               \
    if (ipt == 1) return kron_launch_t<float, P_, 4, 1>(cf, g, io, nch, st); \
    if (ipt == 2) return kron_launch_t<float, P_, 4, 2>(cf, g, io, nch, st); \
    return kron_launch_t<float, P_, 4, 4>(cf, g, io, nch, st);
  switch (g.p) {
    FE_K(1) FE_K(2) FE_K(3) FE_K(4) FE_K(5) FE_K(6)
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", g.p);
  }
#undef FE_K
}

}  // namespace fe

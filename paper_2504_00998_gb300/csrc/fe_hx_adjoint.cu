// Adjoint of the Hamiltonian application with respect to the potential.
//
// Eq. Veff and Hloc with Section 2.3: Ht = 1/2 M^-1/2 K M^-1/2 + diag(V_eff) on psi nodes,
// the potential collocated at the nodes.  For Y = Ht(V) X and a loss L(Y) with
// Ybar = dL/dY, V enters only through the diagonal term, so
//   dL/dV_I = sum_v Ybar_Iv X_Iv,
// and the adjoint with respect to X is Ht^T Ybar = Ht Ybar (Ht is symmetric), i.e.
// fe_apply_H itself.  One warp per node row: the lanes stride over the row's vector
// entries (coalesced), accumulate in double, and the warp sums them in a fixed order, so
// the result is deterministic.
#include <cstdint>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

template <typename T>
__global__ void k_potential_vjp(const T* __restrict__ X, const T* __restrict__ Yb, int64_t ld,
                                int64_t nl, int64_t n, double* __restrict__ g) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
       row += warps) {
    const T* x = X + row * ld;
    const T* y = Yb + row * ld;
    double s = 0.0;
    for (int64_t v = lane; v < nl; v += 32) s = fma((double)y[v], (double)x[v], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[row] = s;
  }
}

}  // namespace

extern "C" fe_status fe_potential_vjp(fe_mesh* m, const void* X, const void* Ybar, int64_t nvec,
                                      int64_t ld, double* gV, fe_precision prec) {
  if (!m || !X || !Ybar || !gV) return fe_fail(FE_EINVAL, "fe_potential_vjp: null argument");
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_BF16_F32ACC && prec != FE_F32_F32ACC)
    return fe_fail(FE_EINVAL, "fe_potential_vjp: bad precision");
  if (nvec < 1 || ld < nvec) return fe_fail(FE_EINVAL, "fe_potential_vjp: need 1 <= nvec <= ld");
  if (m->has_quad)
    return fe_fail(FE_EUNSUPPORTED, "fe_potential_vjp: the potential is collocated only (the "
                   "Gauss-quadrature potential is in effect)");
  FE_TRY(fe_activate(m));
  // complex (Bloch) blocks: the diagonal term acts on both (re, im) lanes alike
  const int64_t lanes = m->has_k ? 2 : 1;
  const int64_t nl = nvec * lanes, ldl = ld * lanes;
  const int blocks = fe::grid_for(m->n_psi * 32, 256);
  if (prec == FE_F64)
    k_potential_vjp<double><<<blocks, 256, 0, m->stream>>>((const double*)X, (const double*)Ybar,
                                                           ldl, nl, m->n_psi, gV);
  else
    k_potential_vjp<float><<<blocks, 256, 0, m->stream>>>((const float*)X, (const float*)Ybar,
                                                          ldl, nl, m->n_psi, gV);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

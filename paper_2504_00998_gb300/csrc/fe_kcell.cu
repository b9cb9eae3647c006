// Single-vector stiffness product y = K x (float) for the Poisson iterations of Section 2.3,
// cell by cell (the cell products and the node sums are in fe_kcell.cuh).  With one vector
// the plane sweep of the block operator leaves most of a CTA idle between its per-plane
// barriers, so this path has two short passes instead:
//   1. k_cell_apply: a CTA takes a strip of CX cells along x and forms y_e = K_e x_e of every
//      cell into the discontinuous node grid;
//   2. k_cell_gather: every node sums its one to eight cell copies, lower cells first.
#include <cstdint>

#include "fe_internal.h"
#include "fe_kcell.cuh"

namespace {

using fe_kc::CellCoef;
using fe_kc::CellStrip;

template <int P>
__global__ void __launch_bounds__(CellStrip<P>::NTHR)
k_cell_apply(const CellCoef cf, const float* __restrict__ x, float* __restrict__ ycell, int nx,
             int ny, int NX, int NY) {
  fe_pdl_enter();
  using S = CellStrip<P>;
  __shared__ float U[S::U_FLOATS];
  __shared__ float A[S::A_FLOATS];
  __shared__ float B[S::A_FLOATS];
  auto load = [x](int64_t gid) { return x[gid]; };
  fe_kc::cell_strip<P>(cf, load, ycell, blockIdx.x * S::CX, blockIdx.y, blockIdx.z, nx, ny, NX,
                       NY, U, A, B);
}

// y at node (gx, gy, gz) = sum of its copies in the discontinuous grid; blocks of 32 x 8
// nodes of one plane (blockIdx.z strides over the planes)
template <int P>
__global__ void __launch_bounds__(256)
k_cell_gather(const float* __restrict__ ycell, float* __restrict__ y, int nx, int ny, int nz,
              int NX, int NY) {
  fe_pdl_enter();
  const int gx = blockIdx.x * 32 + threadIdx.x;
  const int gy = blockIdx.y * 8 + threadIdx.y;
  if (gx >= NX || gy >= NY) return;
  int dx[2], dy[2];
  const int nxc = fe_kc::cell_copies_periodic<P>(gx, nx, dx);
  const int nyc = fe_kc::cell_copies_periodic<P>(gy, ny, dy);
  for (int gz = blockIdx.z; gz <= nz * P; gz += gridDim.z)
    y[((int64_t)gz * NY + gy) * NX + gx] =
        fe_kc::cell_gather_node<P>(ycell, dx, nxc, dy, nyc, gz, nx, ny, nz);
}

template <int P>
fe_status cell_apply_p(const CellCoef& cf, const fe_mesh* m, const float* x, float* y,
                       float* ycell) {
  using S = CellStrip<P>;
  const int nstrip = (m->nx + S::CX - 1) / S::CX;
  if (m->ny > 65535 || m->nz > 65535) return fe_fail(FE_EINVAL, "cell operator: mesh too large");
  // programmatic dependent launches (each kernel waits for its predecessor at entry)
  FE_CUDA(fe_launch_pdl(k_cell_apply<P>, dim3(nstrip, m->ny, m->nz), dim3(S::NTHR), 0, m->stream,
                        cf, x, ycell, m->nx, m->ny, m->NX, m->NY));
  fe_count_launch();
  const int planes = m->NZ < 65535 ? m->NZ : 65535;
  const float* yc = ycell;
  FE_CUDA(fe_launch_pdl(k_cell_gather<P>, dim3((m->NX + 31) / 32, (m->NY + 7) / 8, planes),
                        dim3(32, 8), 0, m->stream, yc, y, m->nx, m->ny, m->nz, m->NX, m->NY));
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // namespace

// scratch of the discontinuous grid: (p+1)^3 floats per cell
size_t fe_kcell_scratch_bytes(const fe_mesh* m) {
  const size_t n1 = (size_t)m->p + 1;
  return sizeof(float) * n1 * n1 * n1 * (size_t)m->nx * m->ny * m->nz;
}

fe_status fe_kcell_apply_f32(fe_mesh* m, const float* x, float* y) {
  void* ws = nullptr;
  FE_TRY(fe_ws(m, WS_KCELL, fe_kcell_scratch_bytes(m), &ws));
  const CellCoef cf = fe_kc::cell_coef(m);
  float* yc = static_cast<float*>(ws);
  switch (m->p) {
    case 1: return cell_apply_p<1>(cf, m, x, y, yc);
    case 2: return cell_apply_p<2>(cf, m, x, y, yc);
    case 3: return cell_apply_p<3>(cf, m, x, y, yc);
    case 4: return cell_apply_p<4>(cf, m, x, y, yc);
    case 5: return cell_apply_p<5>(cf, m, x, y, yc);
    case 6: return cell_apply_p<6>(cf, m, x, y, yc);
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", m->p);
  }
}

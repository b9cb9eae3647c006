// Analysis outputs of a slab solution (Section 3): the dipole moment about the domain
// centre, mu_z = int (b + rho)(z - Lz/2) (Section 3.1), and the planar integral / average of
// a phi-node field per phi plane (Section 3.3: rho0(z) = int_{S_z} rho dx dy and
// V0_bare(z) = (1/A_z) int_{S_z} V_bare dx dy), all with the lumped (GLL) quadrature.
#include <cmath>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

// one block per phi plane: S1 = sum M f, S0 = sum M over the plane, deterministic order
__global__ void k_plane_moments(const double* __restrict__ f, const double* __restrict__ mass,
                                int64_t plane, double* __restrict__ s1, double* __restrict__ s0) {
  __shared__ double a[fe::RED_THREADS], c[fe::RED_THREADS];
  const int64_t base = (int64_t)blockIdx.x * plane;
  double x = 0.0, y = 0.0;
  for (int64_t i = threadIdx.x; i < plane; i += fe::RED_THREADS) {
    const double mi = mass[base + i];
    x += mi * f[base + i];
    y += mi;
  }
  a[threadIdx.x] = x;
  c[threadIdx.x] = y;
  __syncthreads();
  for (int o = fe::RED_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { a[threadIdx.x] += a[threadIdx.x + o]; c[threadIdx.x] += c[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { s1[blockIdx.x] = a[0]; s0[blockIdx.x] = c[0]; }
}

__global__ void k_plane_finish(const double* __restrict__ s1, const double* __restrict__ s0,
                               const double* __restrict__ zw, int nz, int average,
                               double* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz; k += gridDim.x * blockDim.x)
    out[k] = average ? s1[k] / s0[k] : s1[k] / zw[k];
}

struct ZGeom {
  int NX, NY, p, nz;
  double hz, Lz;
  double xi[FE_MAXN1];
};

// partial sums of M (rho + b)(z - Lz/2), one per block
__global__ void k_dipole_partial(const double* __restrict__ rho, const double* __restrict__ b,
                                 const double* __restrict__ mass, ZGeom g, int64_t n,
                                 double* __restrict__ part) {
  __shared__ double sh[fe::RED_THREADS];
  const int64_t plane = (int64_t)g.NX * g.NY;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS) {
    const int gz = (int)(i / plane);
    const double z = (gz / g.p) * g.hz + (g.xi[gz % g.p] + 1.0) * 0.5 * g.hz;
    s += mass[i] * (rho[i] + b[i]) * (z - 0.5 * g.Lz);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = fe::RED_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

}  // namespace

extern "C" fe_status fe_planar(fe_mesh* m, const double* f, int mode, double* out) {
  if (!m || !f || !out) return fe_fail(FE_EINVAL, "fe_planar: null argument");
  if (mode != FE_PLANAR_INTEGRAL && mode != FE_PLANAR_AVERAGE)
    return fe_fail(FE_EINVAL, "fe_planar: bad mode");
  FE_TRY(fe_activate(m));
  cudaStream_t st = m->stream;
  const int nz = m->NZ;
  const int64_t plane = (int64_t)m->NX * m->NY;
  // the z factor (h_z / 2) mz of every phi plane
  std::vector<double> zw(nz);
  for (int gz = 0; gz < nz; ++gz) {
    const int l = gz % m->p;
    const double mz = l ? m->w[l] : ((gz == 0 || gz == nz - 1) ? m->w[0] : 2.0 * m->w[0]);
    zw[gz] = 0.5 * m->h[2] * mz;
  }
  void* wsp;
  FE_TRY(fe_ws(m, WS_RED, sizeof(double) * 3 * (size_t)nz + 64, &wsp));
  double* s1 = (double*)wsp;
  double* s0 = s1 + nz;
  double* dz = s0 + nz;
  FE_CUDA(cudaMemcpyAsync(dz, zw.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st));
  k_plane_moments<<<nz, fe::RED_THREADS, 0, st>>>(f, m->d_mass, plane, s1, s0); fe_count_launch();
  k_plane_finish<<<(nz + 255) / 256, 256, 0, st>>>(s1, s0, dz, nz, mode == FE_PLANAR_AVERAGE, out);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  // the host copy of zw must outlive the asynchronous copy
  FE_CUDA(cudaStreamSynchronize(st));
  return FE_OK;
}

extern "C" fe_status fe_dipole(fe_mesh* m, const double* rho, double* mu_z) {
  if (!m || !mu_z) return fe_fail(FE_EINVAL, "fe_dipole: null argument");
  if (!m->d_b) return fe_fail(FE_EINVAL, "fe_dipole: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  cudaStream_t st = m->stream;
  ZGeom g{};
  g.NX = m->NX;
  g.NY = m->NY;
  g.p = m->p;
  g.nz = m->nz;
  g.hz = m->h[2];
  g.Lz = m->desc.L[2];
  for (int k = 0; k < FE_MAXN1; ++k) g.xi[k] = k <= m->p ? m->xi[k] : 0.0;
  void* wsp;
  FE_TRY(fe_ws(m, WS_RED, sizeof(double) * (fe::RED_BLOCKS + 8), &wsp));
  double* part = (double*)wsp;
  double* res = part + fe::RED_BLOCKS;
  k_dipole_partial<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(rho ? rho : m->d_rho, m->d_b,
                                                               m->d_mass, g, m->n_phi, part);
  fe_count_launch();
  FE_TRY(fe::sum_async(part, fe::RED_BLOCKS, res, st));
  FE_CUDA(cudaMemcpyAsync(mu_z, res, sizeof(double), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  return FE_OK;
}

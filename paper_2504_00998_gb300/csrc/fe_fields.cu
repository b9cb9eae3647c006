// Atom-centred fields at the phi nodes (Eq. Governing equations / Governing equations1).
//
//   V_loc^a - V_sm^a = Z [erf(r / (sqrt2 sigma_b)) - erf(r / rc_loc)] / r   (limit at r = 0)
//   b^a  = -Z_a s_a g_{sigma_b},  s_a chosen so that sum_I M_I b^a(x_I) = -Z_a
//   rho  = t * sum_a Z_a g_{sigma_rho}, t chosen so that sum_I M_I rho(x_I) = sum_a Z_a
// with g_s the normalised Gaussian of standard deviation s; every function is summed over
// the periodic x/y images within 10 bohr of the node and cut there.
#include <cmath>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

constexpr double RCUT = 10.0;

struct FieldGeom {
  int NX, NY, NZ, p;
  double hx, hy, hz, Lx, Ly;
  double xi[FE_MAXN1];
};

__device__ __forceinline__ void node_xyz(const FieldGeom& g, int64_t id, double* x, double* y,
                                         double* z) {
  int gx = (int)(id % g.NX);
  int gy = (int)((id / g.NX) % g.NY);
  int gz = (int)(id / ((int64_t)g.NX * g.NY));
  *x = (gx / g.p) * g.hx + (g.xi[gx % g.p] + 1.0) * 0.5 * g.hx;
  *y = (gy / g.p) * g.hy + (g.xi[gy % g.p] + 1.0) * 0.5 * g.hy;
  *z = (gz / g.p) * g.hz + (g.xi[gz % g.p] + 1.0) * 0.5 * g.hz;
}

// image offsets k with |d + k L| <= rc for the wrapped displacement d
__device__ __forceinline__ void image_range(double d, double L, int* k0, int* k1) {
  *k0 = (int)ceil((-RCUT - d) / L);
  *k1 = (int)floor((RCUT - d) / L);
}

__device__ __forceinline__ double gauss(double r, double s) {
  const double c = 0.06349363593424097;  // (2 pi)^-3/2
  return c / (s * s * s) * exp(-r * r / (2.0 * s * s));
}

__device__ __forceinline__ double vlms_radial(double r, double Z, double sigma_b, double rc_loc) {
  const double a = 1.0 / (sqrt(2.0) * sigma_b), b = 1.0 / rc_loc;
  if (r < 1e-8) return Z * 1.1283791670955126 * (a - b);  // 2/sqrt(pi) (a - b)
  return Z * (erf(a * r) - erf(b * r)) / r;
}

// per-atom lumped integral of the unnormalised smeared charge, partial sums per block
__global__ void k_atom_norm(FieldGeom g, const double* __restrict__ atoms, int natoms,
                            double sigma_b, const double* __restrict__ mass,
                            double* __restrict__ part, int nblk) {
  const int a = blockIdx.y;
  const double X = atoms[4 * a], Y = atoms[4 * a + 1], Zc = atoms[4 * a + 2];
  int gz0 = max(0, (int)floor((Zc - RCUT) / g.hz)) * g.p;
  int gz1 = min(g.NZ - 1, ((int)floor((Zc + RCUT) / g.hz) + 1) * g.p);
  int64_t plane = (int64_t)g.NX * g.NY;
  int64_t i0 = gz0 * plane, i1 = (gz1 + 1) * plane;
  double s = 0.0;
  for (int64_t id = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < i1;
       id += (int64_t)nblk * blockDim.x) {
    double x, y, z;
    node_xyz(g, id, &x, &y, &z);
    double dx = x - X, dy = y - Y, dz = z - Zc;
    dx -= g.Lx * rint(dx / g.Lx);
    dy -= g.Ly * rint(dy / g.Ly);
    int kx0, kx1, ky0, ky1;
    image_range(dx, g.Lx, &kx0, &kx1);
    image_range(dy, g.Ly, &ky0, &ky1);
    double acc = 0.0;
    for (int ky = ky0; ky <= ky1; ++ky)
      for (int kx = kx0; kx <= kx1; ++kx) {
        double ex = dx + kx * g.Lx, ey = dy + ky * g.Ly;
        double r = sqrt(ex * ex + ey * ey + dz * dz);
        if (r <= RCUT) acc += gauss(r, sigma_b);
      }
    s = fma(mass[id], acc, s);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)a * nblk + blockIdx.x] = sh[0];
}

__global__ void k_rowsum(const double* __restrict__ part, int nblk, int nrows,
                         double* __restrict__ out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nrows) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)a * nblk + b];
  out[a] = s;
}

__global__ void k_fields(FieldGeom g, const double* __restrict__ atoms, int natoms,
                         const double* __restrict__ bnorm, double sigma_b, double rc_loc,
                         double sigma_rho, double* __restrict__ vlms, double* __restrict__ rho,
                         double* __restrict__ b, int64_t n) {
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n;
       id += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    node_xyz(g, id, &x, &y, &z);
    double sv = 0.0, sr = 0.0, sb = 0.0;
    for (int a = 0; a < natoms; ++a) {
      const double X = atoms[4 * a], Y = atoms[4 * a + 1], Zc = atoms[4 * a + 2];
      const double Za = atoms[4 * a + 3];
      double dz = z - Zc;
      if (fabs(dz) > RCUT) continue;
      double dx = x - X, dy = y - Y;
      dx -= g.Lx * rint(dx / g.Lx);
      dy -= g.Ly * rint(dy / g.Ly);
      int kx0, kx1, ky0, ky1;
      image_range(dx, g.Lx, &kx0, &kx1);
      image_range(dy, g.Ly, &ky0, &ky1);
      double bscale = -Za / bnorm[a];
      for (int ky = ky0; ky <= ky1; ++ky)
        for (int kx = kx0; kx <= kx1; ++kx) {
          double ex = dx + kx * g.Lx, ey = dy + ky * g.Ly;
          double r = sqrt(ex * ex + ey * ey + dz * dz);
          if (r > RCUT) continue;
          sv += vlms_radial(r, Za, sigma_b, rc_loc);
          sr += Za * gauss(r, sigma_rho);
          sb += bscale * gauss(r, sigma_b);
        }
    }
    vlms[id] = sv;
    rho[id] = sr;
    b[id] = sb;
  }
}

__global__ void k_scale_by_ratio(double* __restrict__ x, int64_t n, double num,
                                 const double* __restrict__ den) {
  double s = num / *den;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

}  // namespace

fe_status fe_fields_build(fe_mesh* m) {
  const int64_t n = m->n_phi;
  cudaStream_t st = m->stream;
  if (!m->d_vlms) {
    FE_CUDA(cudaMalloc(&m->d_vlms, n * sizeof(double)));
    FE_CUDA(cudaMalloc(&m->d_rho, n * sizeof(double)));
    FE_CUDA(cudaMalloc(&m->d_b, n * sizeof(double)));
  }
  if (m->natoms == 0) {
    FE_CUDA(cudaMemsetAsync(m->d_vlms, 0, n * sizeof(double), st));
    FE_CUDA(cudaMemsetAsync(m->d_rho, 0, n * sizeof(double), st));
    FE_CUDA(cudaMemsetAsync(m->d_b, 0, n * sizeof(double), st));
    return FE_OK;
  }
  FieldGeom g;
  g.NX = m->NX; g.NY = m->NY; g.NZ = m->NZ; g.p = m->p;
  g.hx = m->h[0]; g.hy = m->h[1]; g.hz = m->h[2];
  g.Lx = m->desc.L[0]; g.Ly = m->desc.L[1];
  for (int k = 0; k < FE_MAXN1; ++k) g.xi[k] = k <= m->p ? m->xi[k] : 0.0;
  const int nblk = 64;
  void* wsp;
  FE_TRY(fe_ws(m, WS_RED, sizeof(double) * ((size_t)m->natoms * (nblk + 1) + fe::RED_BLOCKS + 8),
               &wsp));
  double* part = (double*)wsp;
  double* bnorm = part + (size_t)m->natoms * nblk;
  double* red = bnorm + m->natoms;
  double* tot = red + fe::RED_BLOCKS;
  k_atom_norm<<<dim3(nblk, m->natoms), 256, 0, st>>>(g, m->d_atoms, m->natoms, m->sigma_b,
                                                     m->d_mass, part, nblk); fe_count_launch();
  k_rowsum<<<(m->natoms + 127) / 128, 128, 0, st>>>(part, nblk, m->natoms, bnorm); fe_count_launch();
  k_fields<<<fe::grid_for(n), 256, 0, st>>>(g, m->d_atoms, m->natoms, bnorm, m->sigma_b,
                                            m->rc_loc, m->sigma_rho, m->d_vlms, m->d_rho,
                                            m->d_b, n); fe_count_launch();
  FE_TRY(fe::dot_async(m->d_mass, m->d_rho, n, 1, red, tot, st));
  double ne = 0.0;
  for (int a = 0; a < m->natoms; ++a) ne += m->h_atoms[4 * a + 3];
  k_scale_by_ratio<<<fe::grid_for(n), 256, 0, st>>>(m->d_rho, n, ne, tot); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  double tot_h = 0.0;
  FE_CUDA(cudaMemcpyAsync(&tot_h, tot, sizeof(double), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  m->rho_scale = ne / tot_h;
  m->n_electrons = ne;
  return FE_OK;
}

// Electrostatic energy of the biased slab and its derivatives, for differentiation through
// the Poisson solve.
//
// Energy at fixed electron density (Eq. electrostatics Energy, Eq. local pseudopotential and,
// for CEF, the V_app term of Eq. KS DFT variational problem cef), with lumped quadrature:
//   E = c . phi - phi^T K phi / (8 pi) + sum_I M_I (V_loc - V_sm)_I rho_I
//       + sum_I M_I (rho + b)_I V_app,I,            c = M (rho + b).
// phi maximises E over the free nodes (Eq. electrostatics Energy), so dE/dphi_free = 0 and the
// derivatives follow from the explicit dependences (envelope theorem):
//   dE/d rho_I  = M_I (phi_I + (V_loc - V_sm)_I + V_app,I)
//   dE/d b_I    = M_I (phi_I + V_app,I)
//   dE/d vlms_I = M_I rho_I - r_I [I constrained]   (CPD values depend on -(V_loc - V_sm))
//   dE/d E_field = sum_I M_I (rho + b)_I dV_app/dE
//   dE/d dV      = sum_{I in Omega_1} r_I,           r = c - K phi / (4 pi)
// (the reaction charge on the conductor; Section 2.2.2).  The smeared-charge self energy
// is constant in the bias and the positions and is left out.
//
// Atom-position derivatives: fe_atom_fields_vjp contracts node weights with the analytic
// derivatives of the atom-centred fields of fe_set_atoms, including the per-atom and global
// renormalisations.
#include <cmath>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

constexpr double FOUR_PI = 12.566370614359172;
constexpr double RCUT = 10.0;

struct AGeom {
  int NX, NY, NZ, p;
  double hx, hy, hz, Lx, Ly, Lz;
  double xi[FE_MAXN1];
};

AGeom ageom(const fe_mesh* m) {
  AGeom g;
  g.NX = m->NX; g.NY = m->NY; g.NZ = m->NZ; g.p = m->p;
  g.hx = m->h[0]; g.hy = m->h[1]; g.hz = m->h[2];
  g.Lx = m->desc.L[0]; g.Ly = m->desc.L[1]; g.Lz = m->desc.L[2];
  for (int k = 0; k < FE_MAXN1; ++k) g.xi[k] = k <= m->p ? m->xi[k] : 0.0;
  return g;
}

__device__ __forceinline__ void xyz(const AGeom& g, int64_t id, double* x, double* y, double* z) {
  int gx = (int)(id % g.NX);
  int gy = (int)((id / g.NX) % g.NY);
  int gz = (int)(id / ((int64_t)g.NX * g.NY));
  *x = (gx / g.p) * g.hx + (g.xi[gx % g.p] + 1.0) * 0.5 * g.hx;
  *y = (gy / g.p) * g.hy + (g.xi[gy % g.p] + 1.0) * 0.5 * g.hy;
  *z = (gz / g.p) * g.hz + (g.xi[gz % g.p] + 1.0) * 0.5 * g.hz;
}

__device__ __forceinline__ double vapp(double z, double E, double Lz) {
  const double z1 = 0.1 * Lz, z2 = 0.9 * Lz;
  if (z < z1) return -E * (z1 - 0.5 * Lz) * z / z1;
  if (z > z2) return -E * (z2 - 0.5 * Lz) * (Lz - z) / (Lz - z2);
  return -E * (z - 0.5 * Lz);
}

constexpr int NE_TERMS = 6;  // c.phi, phi.Kphi, M vlms rho, M (rho+b) vapp, dE/dfield, dE/ddV

__global__ void k_energy(AGeom g, fe_poisson_bc bc, const double* __restrict__ mass,
                         const double* __restrict__ rho, const double* __restrict__ b,
                         const double* __restrict__ vlms, const double* __restrict__ phi,
                         const double* __restrict__ kphi, double* __restrict__ g_rho,
                         double* __restrict__ g_b, double* __restrict__ g_vlms,
                         double* __restrict__ part, int64_t n) {
  __shared__ double sh[NE_TERMS][fe::RED_THREADS];
  double acc[NE_TERMS] = {0, 0, 0, 0, 0, 0};
  const bool cef = bc.kind == FE_BIAS_CEF;
  for (int64_t id = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; id < n;
       id += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS) {
    double x, y, z;
    xyz(g, id, &x, &y, &z);
    const double M = mass[id], r_ = rho[id], b_ = b[id], v_ = vlms[id], p_ = phi[id];
    const double c = M * (r_ + b_);
    const double va = cef ? vapp(z, bc.field, g.Lz) : 0.0;
    const double dva = cef ? vapp(z, 1.0, g.Lz) : 0.0;
    acc[0] += c * p_;
    acc[1] += p_ * kphi[id];
    acc[2] += M * v_ * r_;
    acc[3] += c * va;
    acc[4] += c * dva;
    double react = 0.0;
    bool om1 = false, constrained = false;
    if (!cef) {
      const double tol = 1e-12;
      bool om0 = z <= bc.zA + tol;
      om1 = z >= bc.zB - tol;
      if (bc.has_patch)
        om1 = om1 && x >= bc.patch_lo[0] - tol && x <= bc.patch_hi[0] + tol &&
              y >= bc.patch_lo[1] - tol && y <= bc.patch_hi[1] + tol;
      constrained = om0 || om1;
      if (constrained) react = c - kphi[id] / FOUR_PI;
    }
    if (om1) acc[5] += react;
    g_rho[id] = M * (p_ + v_ + va);
    g_b[id] = M * (p_ + va);
    g_vlms[id] = M * r_ - (constrained ? react : 0.0);
  }
  for (int t = 0; t < NE_TERMS; ++t) sh[t][threadIdx.x] = acc[t];
  __syncthreads();
  for (int w = fe::RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int t = 0; t < NE_TERMS; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NE_TERMS) part[threadIdx.x * fe::RED_BLOCKS + blockIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_sum_rows(const double* __restrict__ part, int rows, int cols,
                           double* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double s = 0.0;
  for (int c = 0; c < cols; ++c) s += part[(int64_t)r * cols + c];
  out[r] = s;
}

constexpr int NV = 17;  // per-atom accumulators of the VJP

// per atom a, over the nodes within reach:
//  [0] s = sum M g_b        [1..3] sum M dg_b/dR     [4..6] sum w dg_b/dR   [7] sum w g_b
//  [8..10] sum u dg_r/dR    [11..13] sum M dg_r/dR   [14..16] sum q dv_a/dR
__global__ void k_vjp_atoms(AGeom g, const double* __restrict__ atoms, double sigma_b,
                            double sigma_rho, double rc_loc, const double* __restrict__ mass,
                            const double* __restrict__ w, const double* __restrict__ u,
                            const double* __restrict__ q, double* __restrict__ part, int nblk) {
  const int a = blockIdx.y;
  const double X = atoms[4 * a], Y = atoms[4 * a + 1], Zc = atoms[4 * a + 2], Za = atoms[4 * a + 3];
  int gz0 = max(0, (int)floor((Zc - RCUT) / g.hz)) * g.p;
  int gz1 = min(g.NZ - 1, ((int)floor((Zc + RCUT) / g.hz) + 1) * g.p);
  const int64_t plane = (int64_t)g.NX * g.NY;
  const int64_t i0 = gz0 * plane, i1 = (gz1 + 1) * plane;
  const double cb = 0.06349363593424097 / (sigma_b * sigma_b * sigma_b);
  const double cr = 0.06349363593424097 / (sigma_rho * sigma_rho * sigma_rho);
  const double al = 1.0 / (sqrt(2.0) * sigma_b), be = 1.0 / rc_loc;
  const double tsp = 1.1283791670955126;  // 2 / sqrt(pi)
  double acc[NV];
  for (int t = 0; t < NV; ++t) acc[t] = 0.0;
  for (int64_t id = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < i1;
       id += (int64_t)nblk * blockDim.x) {
    double x, y, z;
    xyz(g, id, &x, &y, &z);
    double dx = x - X, dy = y - Y, dz = z - Zc;
    dx -= g.Lx * rint(dx / g.Lx);
    dy -= g.Ly * rint(dy / g.Ly);
    int kx0 = (int)ceil((-RCUT - dx) / g.Lx), kx1 = (int)floor((RCUT - dx) / g.Lx);
    int ky0 = (int)ceil((-RCUT - dy) / g.Ly), ky1 = (int)floor((RCUT - dy) / g.Ly);
    const double M = mass[id], wi = w[id], ui = u[id], qi = q[id];
    for (int ky = ky0; ky <= ky1; ++ky)
      for (int kx = kx0; kx <= kx1; ++kx) {
        const double ex = dx + kx * g.Lx, ey = dy + ky * g.Ly;
        const double r2 = ex * ex + ey * ey + dz * dz;
        const double r = sqrt(r2);
        if (r > RCUT) continue;
        // Gaussians: dG/dR = (d / s^2) G with d = x - R
        const double gb = cb * exp(-r2 / (2.0 * sigma_b * sigma_b));
        const double gr = cr * exp(-r2 / (2.0 * sigma_rho * sigma_rho));
        const double fb = gb / (sigma_b * sigma_b), fr = gr / (sigma_rho * sigma_rho);
        acc[0] += M * gb;
        acc[1] += M * fb * ex; acc[2] += M * fb * ey; acc[3] += M * fb * dz;
        acc[4] += wi * fb * ex; acc[5] += wi * fb * ey; acc[6] += wi * fb * dz;
        acc[7] += wi * gb;
        acc[8] += ui * fr * ex; acc[9] += ui * fr * ey; acc[10] += ui * fr * dz;
        acc[11] += M * fr * ex; acc[12] += M * fr * ey; acc[13] += M * fr * dz;
        // v(r) = Z [erf(al r) - erf(be r)] / r; dv/dR = -v'(r) d / r
        double vp_over_r;
        if (r < 1e-3) {
          // series of erf: v'(r)/r = Z (2/sqrt pi) [-(2/3)(al^3 - be^3) + (2/5)(al^5 - be^5) r^2
          //                                         - (1/7)(al^7 - be^7) r^4 + ...]
          vp_over_r = Za * tsp * (-(2.0 / 3.0) * (pow(al, 3) - pow(be, 3)) +
                                  0.4 * (pow(al, 5) - pow(be, 5)) * r2 -
                                  (1.0 / 7.0) * (pow(al, 7) - pow(be, 7)) * r2 * r2);
        } else {
          const double num = tsp * (al * exp(-al * al * r2) - be * exp(-be * be * r2)) / r -
                             (erf(al * r) - erf(be * r)) / r2;
          vp_over_r = Za * num / r;
        }
        acc[14] -= qi * vp_over_r * ex;
        acc[15] -= qi * vp_over_r * ey;
        acc[16] -= qi * vp_over_r * dz;
      }
  }
  __shared__ double sh[NV][256];
  for (int t = 0; t < NV; ++t) sh[t][threadIdx.x] = acc[t];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int t = 0; t < NV; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < NV)
    part[((int64_t)a * NV + threadIdx.x) * nblk + blockIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

extern "C" fe_status fe_atom_fields(fe_mesh* m, double* rho, double* b, double* vlms) {
  if (!m) return fe_fail(FE_EINVAL, "fe_atom_fields: null mesh");
  if (!m->d_rho) return fe_fail(FE_EINVAL, "fe_atom_fields: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  const size_t bytes = sizeof(double) * m->n_phi;
  if (rho) FE_CUDA(cudaMemcpyAsync(rho, m->d_rho, bytes, cudaMemcpyDeviceToDevice, m->stream));
  if (b) FE_CUDA(cudaMemcpyAsync(b, m->d_b, bytes, cudaMemcpyDeviceToDevice, m->stream));
  if (vlms) FE_CUDA(cudaMemcpyAsync(vlms, m->d_vlms, bytes, cudaMemcpyDeviceToDevice, m->stream));
  return FE_OK;
}

extern "C" fe_status fe_energy(fe_mesh* m, const fe_poisson_bc* bc, const double* phi,
                               double* E, double* dE_dfield, double* dE_ddV, double* g_rho,
                               double* g_b, double* g_vlms) {
  if (!m || !bc || !phi || !E || !g_rho || !g_b || !g_vlms)
    return fe_fail(FE_EINVAL, "fe_energy: null argument");
  if (!m->d_rho) return fe_fail(FE_EINVAL, "fe_energy: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_phi;
  void* wsp;
  FE_TRY(fe_ws(m, WS_LANCZOS, sizeof(double) * ((size_t)n + NE_TERMS * fe::RED_BLOCKS + 16), &wsp));
  double* kphi = (double*)wsp;
  double* part = kphi + n;
  double* tot = part + NE_TERMS * fe::RED_BLOCKS;
  FE_TRY(fe_poisson_apply_K(m, phi, kphi));
  k_energy<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, m->stream>>>(ageom(m), *bc, m->d_mass, m->d_rho,
                                                              m->d_b, m->d_vlms, phi, kphi, g_rho,
                                                              g_b, g_vlms, part, n); fe_count_launch();
  k_sum_rows<<<1, 32, 0, m->stream>>>(part, NE_TERMS, fe::RED_BLOCKS, tot); fe_count_launch();
  double h[NE_TERMS];
  FE_CUDA(cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  *E = h[0] - h[1] / (2.0 * FOUR_PI) + h[2] + h[3];
  if (dE_dfield) *dE_dfield = h[4];
  if (dE_ddV) *dE_ddV = h[5];
  return FE_OK;
}

extern "C" fe_status fe_atom_fields_vjp(fe_mesh* m, const double* g_rho, const double* g_b,
                                        const double* g_vlms, double* dR) {
  if (!m || !g_rho || !g_b || !g_vlms || !dR)
    return fe_fail(FE_EINVAL, "fe_atom_fields_vjp: null argument");
  if (!m->d_rho || m->natoms == 0) return fe_fail(FE_EINVAL, "fe_atom_fields_vjp: no atoms");
  FE_TRY(fe_activate(m));
  const int nblk = 32, na = m->natoms;
  void* wsp;
  FE_TRY(fe_ws(m, WS_RED, sizeof(double) * ((size_t)na * NV * (nblk + 1) + fe::RED_BLOCKS + 8),
               &wsp));
  double* part = (double*)wsp;
  double* per_atom = part + (size_t)na * NV * nblk;
  double* red = per_atom + (size_t)na * NV;
  double* U = red + fe::RED_BLOCKS;
  k_vjp_atoms<<<dim3(nblk, na), 256, 0, m->stream>>>(ageom(m), m->d_atoms, m->sigma_b,
                                                     m->sigma_rho, m->rc_loc, m->d_mass, g_b,
                                                     g_rho, g_vlms, part, nblk); fe_count_launch();
  k_sum_rows<<<(na * NV + 127) / 128, 128, 0, m->stream>>>(part, na * NV, nblk, per_atom); fe_count_launch();
  FE_TRY(fe::dot_async(g_rho, m->d_rho, m->n_phi, 1, red, U, m->stream));
  std::vector<double> h((size_t)na * NV + 1);
  FE_CUDA(cudaMemcpyAsync(h.data(), per_atom, sizeof(double) * na * NV, cudaMemcpyDeviceToHost,
                          m->stream));
  FE_CUDA(cudaMemcpyAsync(h.data() + (size_t)na * NV, U, sizeof(double), cudaMemcpyDeviceToHost,
                          m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  const double Uv = h[(size_t)na * NV];
  const double ne = m->n_electrons, t = m->rho_scale;
  for (int a = 0; a < na; ++a) {
    const double* v = &h[(size_t)a * NV];
    const double Za = m->h_atoms[4 * a + 3];
    const double s = v[0];
    for (int k = 0; k < 3; ++k) {
      // b = -Z g / s:   d/dR = -Z/s (dg - g ds/s)
      double db = -Za / s * (v[4 + k] - (v[7] / s) * v[1 + k]);
      // rho = t Z g_r (global renormalisation): d/dR = t Z (dg_r - (rho/N_e) dT/(t Z)...)
      double drho = t * Za * (v[8 + k] - (Uv / ne) * v[11 + k]);
      dR[3 * a + k] = db + drho + v[14 + k];
    }
  }
  return FE_OK;
}

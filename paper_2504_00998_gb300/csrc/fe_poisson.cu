// Poisson problem with the paper's two bias setups, solved by Jacobi-preconditioned CG on
// the matrix-free stiffness operator.
//
// Eq. Poissons equation, FE form (Section 2.3): K phi = 4 pi c, c_I = M_II (rho + b)(x_I).
// CEF (Eq. governing_equations CEF): zero-Neumann z faces (natural), int phi = 0.  The load
//   is projected onto range(K) (f <- f - (sum f / sum M) M), the CG residual is re-projected
//   onto the complement of the constants every iteration, and phi is shifted to
//   sum_I M_I phi_I = 0 at the end.  V_app is the sawtooth of Section 2.2.1 with slope -E on
//   [0.1 Lz, 0.9 Lz] (extrema 0.1 fractional units from the boundaries, Section 3.1) and
//   linear return ramps to zero at z = 0 and z = Lz.
// CPD / L-CPD (Eq. governing_equations APD): phi = -(V_loc - V_sm) on Omega_0 = {z <= zA}
//   and dV - (V_loc - V_sm) on Omega_1 = {z >= zB} (intersected with the patch for L-CPD);
//   CG runs on the free nodes with the constrained rows and columns masked; V_app = 0.
//
// Every CG iteration is a fixed sequence of stream-ordered launches with all scalars on the
// device; a block of iterations is captured once into a CUDA graph and replayed, and the
// host reads the convergence flag between replays.  The iteration cap bounds the loop.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <vector>

#include "fe_blas.cuh"
#include "fe_cg.cuh"
#include "fe_internal.h"

namespace {

constexpr double FOUR_PI = 12.566370614359172;

using fe_cg::CgState;

struct PGeom {
  int NX, NY, NZ, p;
  double hx, hy, hz, Lz;
  double xi[FE_MAXN1];
  double K1d0, K1dp;            // K1[0][0], K1[p][p]
  double K1diag[FE_MAXN1], M1diag[FE_MAXN1];
  double ax, ay, az;
};

__device__ __forceinline__ void pnode(const PGeom& g, int64_t id, int* gx, int* gy, int* gz) {
  *gx = (int)(id % g.NX);
  *gy = (int)((id / g.NX) % g.NY);
  *gz = (int)(id / ((int64_t)g.NX * g.NY));
}

__device__ __forceinline__ double zcoord(const PGeom& g, int gz) {
  return (gz / g.p) * g.hz + (g.xi[gz % g.p] + 1.0) * 0.5 * g.hz;
}

// diagonal of an assembled 1D element matrix at global index gi (periodic or bounded)
__device__ __forceinline__ double diag1(const double* d, int p, int gi, bool periodic, int nmax) {
  int l = gi % p;
  if (l != 0) return d[l];
  if (periodic) return d[0] + d[p];
  if (gi == 0) return d[0];
  if (gi == nmax) return d[p];
  return d[0] + d[p];
}

__device__ __forceinline__ double vapp(double z, double E, double Lz) {
  const double z1 = 0.1 * Lz, z2 = 0.9 * Lz;
  if (z < z1) return -E * (z1 - 0.5 * Lz) * z / z1;
  if (z > z2) return -E * (z2 - 0.5 * Lz) * (Lz - z) / (Lz - z2);
  return -E * (z - 0.5 * Lz);
}

// f = 4 pi M (rho + b); Jacobi inverse; constraint mask and values; phi initialisation
// (f_ext: a given load instead of 4 pi M (rho + b); phic_ext: given constrained values)
__global__ void k_setup(PGeom g, fe_poisson_bc bc, const double* __restrict__ mass,
                        const double* __restrict__ rho, const double* __restrict__ b,
                        const double* __restrict__ vlms, const double* __restrict__ f_ext,
                        const double* __restrict__ phic_ext, double* __restrict__ f,
                        double* __restrict__ dinv, unsigned char* __restrict__ mask,
                        double* __restrict__ phi, int64_t n) {
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n;
       id += (int64_t)gridDim.x * blockDim.x) {
    int gx, gy, gz;
    pnode(g, id, &gx, &gy, &gz);
    f[id] = f_ext ? f_ext[id] : FOUR_PI * mass[id] * (rho[id] + b[id]);
    int nz = g.NZ - 1;
    double kx = diag1(g.K1diag, g.p, gx, true, 0), mx = diag1(g.M1diag, g.p, gx, true, 0);
    double ky = diag1(g.K1diag, g.p, gy, true, 0), my = diag1(g.M1diag, g.p, gy, true, 0);
    double kz = diag1(g.K1diag, g.p, gz, false, nz), mz = diag1(g.M1diag, g.p, gz, false, nz);
    double d = g.ax * kx * my * mz + g.ay * mx * ky * mz + g.az * mx * my * kz;
    dinv[id] = 1.0 / d;
    unsigned char c = 0;
    double val = 0.0;
    if (bc.kind == FE_BIAS_CPD) {
      double x = (gx / g.p) * g.hx + (g.xi[gx % g.p] + 1.0) * 0.5 * g.hx;
      double y = (gy / g.p) * g.hy + (g.xi[gy % g.p] + 1.0) * 0.5 * g.hy;
      double z = zcoord(g, gz);
      const double tol = 1e-12;
      bool om0 = z <= bc.zA + tol;
      bool om1 = z >= bc.zB - tol;
      if (bc.has_patch)
        om1 = om1 && x >= bc.patch_lo[0] - tol && x <= bc.patch_hi[0] + tol &&
              y >= bc.patch_lo[1] - tol && y <= bc.patch_hi[1] + tol;
      if (om0) { c = 1; val = phic_ext ? phic_ext[id] : -vlms[id]; }
      if (om1) { c = 1; val = phic_ext ? phic_ext[id] : bc.dV - vlms[id]; }
    }
    mask[id] = c;
    phi[id] = val;
  }
}

// Block sums in a fixed order (so every reduction is reproducible): a shuffle tree inside
// each warp, then every warp reduces the per-warp sums the same way.  blockDim.x is a multiple
// of 32 (at most 1024); every thread receives the total; one barrier per call (two with the
// barrier that lets a later call reuse the staging array).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31;
  if (lane == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
  t = __shfl_sync(0xffffffffu, warp_sum(t), 0);
  __syncthreads();
  return t;
}
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double wa[32], wb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31;
  if (lane == 0) { wa[threadIdx.x >> 5] = a; wb[threadIdx.x >> 5] = b; }
  __syncthreads();
  const bool in = lane < (int)(blockDim.x >> 5);
  a = __shfl_sync(0xffffffffu, warp_sum(in ? wa[lane] : 0.0), 0);
  b = __shfl_sync(0xffffffffu, warp_sum(in ? wb[lane] : 0.0), 0);
  __syncthreads();
}

// partial sums of x (y == nullptr) or x.y, accumulated in double; one partial per block
template <typename V>
__global__ void k_psum(const V* __restrict__ x, const V* __restrict__ y, int64_t n,
                       double* __restrict__ part) {
  V s = V(0);   // a thread's few terms in the vector precision, the block sum in double
  for (int64_t i = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS)
    s += y ? x[i] * y[i] : x[i];
  const double t = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__device__ double block_sum_partials(const double* part) {
  double s = 0.0;
  for (int i = threadIdx.x; i < fe::RED_BLOCKS; i += blockDim.x) s += part[i];
  return block_sum(s);
}

// CEF load projection: f <- f - (sum f / sum M) M
__global__ void k_fin_project_load(const double* part_f, const double* part_m, CgState* s) {
  double sf = block_sum_partials(part_f);
  double sm = block_sum_partials(part_m);
  if (threadIdx.x == 0) s->mean = sf / sm;
}
__global__ void k_project_load(double* __restrict__ f, const double* __restrict__ mass,
                               const CgState* s, int64_t n) {
  double c = s->mean;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    f[i] -= c * mass[i];
}

// r = (f - K phi) on free rows, 0 on constrained rows
__global__ void k_resid0(const double* __restrict__ f, const double* __restrict__ kphi,
                         const unsigned char* __restrict__ mask, double* __restrict__ r,
                         int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = mask[i] ? 0.0 : f[i] - kphi[i];
}

__global__ void k_fin_mean(const double* part, CgState* s, double inv_n) {
  double v = block_sum_partials(part);
  if (threadIdx.x == 0) s->mean = v * inv_n;
}

// r -= mean (CEF only); z = Dinv r (+ the coarse correction of the node's plane) on free
// rows; one partial of r.z and r.r per block (of the stored, possibly rounded, values)
// (mean_part: the block partials of sum r, reduced here by every block instead of a separate
// finishing kernel; nullptr: the mean already in the state)
template <typename V>
__global__ void k_precond(V* __restrict__ r, V* __restrict__ z, const V* __restrict__ dinv,
                          const unsigned char* __restrict__ mask, const CgState* s, int project,
                          int64_t n, double* __restrict__ part_rz, double* __restrict__ part_rr,
                          const double* __restrict__ cy, int64_t plane,
                          const double* __restrict__ mean_part) {
  double mean_d = 0.0;
  if (project) mean_d = mean_part ? block_sum_partials(mean_part) * (1.0 / (double)n) : s->mean;
  const V mean = (V)mean_d;
  const uint32_t pl = (uint32_t)plane;
  V a1 = V(0), a2 = V(0);
  for (int64_t i = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS) {
    V ri = r[i];
    if (project) { ri -= mean; r[i] = ri; }
    const V zi = mask[i] ? V(0) : dinv[i] * ri + (cy ? (V)cy[(uint32_t)i / pl] : V(0));
    z[i] = zi;
    a1 += ri * zi;
    a2 += ri * ri;
  }
  double t1 = (double)a1, t2 = (double)a2;
  block_sum2(t1, t2);
  if (threadIdx.x == 0) { part_rz[blockIdx.x] = t1; part_rr[blockIdx.x] = t2; }
}

// first iteration: p = z, rz, rr, |b|^2
// (tol2_abs > 0: that absolute bound on |r|^2, else rtol relative to this initial residual)
__global__ void k_fin_init(const double* part_rz, const double* part_rr, CgState* s, double rtol,
                           double tol2_abs) {
  double rz = block_sum_partials(part_rz);
  double rr = block_sum_partials(part_rr);
  if (threadIdx.x == 0) {
    s->rz = rz;
    s->rr = rr;
    s->bnorm2 = rr;
    s->tol2 = tol2_abs > 0.0 ? tol2_abs : rtol * rtol * rr;
    s->done = (rr <= s->tol2) || rr == 0.0;
    s->iters = 0;
  }
}

template <typename V>
__global__ void k_copy(const V* __restrict__ a, V* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// alpha = rz / p.q
__global__ void k_fin_alpha(const double* part, CgState* s) {
  double pq = block_sum_partials(part);
  if (threadIdx.x == 0) {
    s->pq = pq;
    s->alpha = (s->done || pq == 0.0) ? 0.0 : s->rz / pq;
  }
}

// x += alpha p; r -= alpha q (free rows); partial sums of r for the projection
// (pq_part: the block partials of p.q; every block forms alpha = r.z / p.q itself and block 0
// records it in the state, so no separate finishing kernel runs)
template <typename V>
__global__ void k_update_xr(V* __restrict__ x, V* __restrict__ r, const V* __restrict__ p,
                            const V* __restrict__ q, const unsigned char* __restrict__ mask,
                            CgState* s, int64_t n, double* __restrict__ part,
                            const double* __restrict__ pq_part) {
  const double pq = block_sum_partials(pq_part);
  const double al = (s->done || pq == 0.0) ? 0.0 : s->rz / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->pq = pq;
    s->alpha = al;
  }
  const V a = (V)al;
  V acc = V(0);
  for (int64_t i = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS) {
    V ri = r[i];
    if (!mask[i]) {
      x[i] += a * p[i];
      ri -= a * q[i];
      r[i] = ri;
    }
    acc += ri;
  }
  const double t = block_sum((double)acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// beta = rz_new / rz; convergence test on |r|^2; iteration count
__global__ void k_fin_beta(const double* part_rz, const double* part_rr, CgState* s) {
  double rz = block_sum_partials(part_rz);
  double rr = block_sum_partials(part_rr);
  if (threadIdx.x == 0) {
    if (!s->done) {
      s->beta = s->rz == 0.0 ? 0.0 : rz / s->rz;
      s->rz = rz;
      s->rr = rr;
      s->iters += 1;
      if (rr <= s->tol2 || s->iters >= s->maxit) s->done = 1;
    } else {
      s->beta = 0.0;
    }
  }
}

// p = z + beta p (skipped once converged so p, x stay fixed)
template <typename V>
__global__ void k_update_p(V* __restrict__ p, const V* __restrict__ z, const CgState* s,
                           int64_t n) {
  if (s->done && s->alpha == 0.0) return;
  const V b = (V)s->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + b * p[i];
}

// mixed-precision refinement: the float copy of the double residual, and phi += delta
__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_add_delta(double* __restrict__ phi, const float* __restrict__ d,
                            const unsigned char* __restrict__ mask, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!mask[i]) phi[i] += (double)d[i];
}
// r -= mean (after k_fin_mean); |r|^2 goes through k_psum
__global__ void k_sub_mean(double* __restrict__ r, const CgState* s, int64_t n) {
  const double c = s->mean;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] -= c;
}
__global__ void k_fin_rr(const double* part, CgState* s) {
  double v = block_sum_partials(part);
  if (threadIdx.x == 0) s->rr = v;
}
// residual replacement in a running CG: new r.z and |r|^2, the search direction is kept
__global__ void k_fin_replace(const double* part_rz, const double* part_rr, CgState* s) {
  double rz = block_sum_partials(part_rz);
  double rr = block_sum_partials(part_rr);
  if (threadIdx.x == 0) {
    s->rz = rz;
    s->rr = rr;
    s->done = (rr == 0.0 || s->iters >= s->maxit) ? 1 : 0;
  }
}

// CEF: phi -= (M . phi) / sum M
__global__ void k_shift_mean(double* __restrict__ phi, const double* part_mphi,
                             const double* part_m, int64_t n) {
  __shared__ double c;
  double a = block_sum_partials(part_mphi);
  double b = block_sum_partials(part_m);
  if (threadIdx.x == 0) c = a / b;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    phi[i] -= c;
}

// V_eff at psi nodes: phi + (V_loc - V_sm) + V_app
__global__ void k_vbare(PGeom g, const double* __restrict__ phi, const double* __restrict__ vlms,
                        double field, int cef, int gz_lo, double* __restrict__ out, int64_t npsi) {
  int64_t off = (int64_t)gz_lo * g.NX * g.NY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npsi;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t id = i + off;
    int gz = (int)(id / ((int64_t)g.NX * g.NY));
    double v = phi[id] + vlms[id];
    if (cef) v += vapp(zcoord(g, gz), field, g.Lz);
    out[i] = v;
  }
}

// ---- z-plane coarse space ---------------------------------------------------------------
// Basis: one function per phi plane, the indicator of the plane's free nodes.  R x = plane
// sums over free nodes; the coarse matrix Ac = R K R^T couples planes that share a cell layer.

// out[gz] = sum of x over the free nodes of plane gz (x == nullptr: the free-node count);
// ---- float vectors, four nodes per access --------------------------------------------------
// Used when a z plane holds a multiple of four nodes (a group of four never straddles a plane)
// and the arrays are 16-byte (vectors) and 4-byte (mask) aligned.  A thread issues the loads of
// up to V4B groups before using any of them, so that one round trip to L2 covers its share;
// the sums keep the scalar kernels' structure (a thread's terms in float, the block sum in
// double, one partial per block).
constexpr int V4B = 4;
constexpr int64_t V4S = (int64_t)fe::RED_BLOCKS * fe::RED_THREADS;

__device__ __forceinline__ void block_partial(float v, double* __restrict__ part) {
  const double t = block_sum((double)v);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__device__ __forceinline__ float sum4(const float4& a) { return a.x + a.y + a.z + a.w; }

// partial sums of x (y == nullptr) or x.y over n4 groups
__global__ void k_psum4(const float* __restrict__ x, const float* __restrict__ y, int64_t n4,
                        double* __restrict__ part) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  const int64_t g = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x;
  float s = 0.f;
  for (int64_t q0 = g; q0 < n4; q0 += V4B * V4S) {
    float4 a[V4B], b[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t q = q0 + u * V4S;
      if (q < n4) {
        a[u] = x4[q];
        if (y) b[u] = y4[q];
      }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      if (q0 + u * V4S >= n4) continue;
      s += y ? a[u].x * b[u].x + a[u].y * b[u].y + a[u].z * b[u].z + a[u].w * b[u].w : sum4(a[u]);
    }
  }
  block_partial(s, part);
}

// alpha from the p.q partials (every block; block 0 records it); x += alpha p, r -= alpha q
// on free nodes; partials of sum r
__global__ void k_update_xr4(float* __restrict__ x, float* __restrict__ r,
                             const float* __restrict__ p, const float* __restrict__ q,
                             const unsigned char* __restrict__ mask, CgState* s, int64_t n4,
                             double* __restrict__ part, const double* __restrict__ pq_part) {
  const double pq = block_sum_partials(pq_part);
  const double al = (s->done || pq == 0.0) ? 0.0 : s->rz / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->pq = pq;
    s->alpha = al;
  }
  const float a = (float)al;
  float4* x4 = reinterpret_cast<float4*>(x);
  float4* r4 = reinterpret_cast<float4*>(r);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(mask);
  const int64_t g = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x;
  float acc = 0.f;
  for (int64_t q0 = g; q0 < n4; q0 += V4B * V4S) {
    float4 xv[V4B], rv[V4B], pv[V4B], qv[V4B];
    uchar4 mv[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = q0 + u * V4S;
      if (k < n4) { xv[u] = x4[k]; rv[u] = r4[k]; pv[u] = p4[k]; qv[u] = q4[k]; mv[u] = m4[k]; }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = q0 + u * V4S;
      if (k >= n4) continue;
      if (!mv[u].x) { xv[u].x += a * pv[u].x; rv[u].x -= a * qv[u].x; }
      if (!mv[u].y) { xv[u].y += a * pv[u].y; rv[u].y -= a * qv[u].y; }
      if (!mv[u].z) { xv[u].z += a * pv[u].z; rv[u].z -= a * qv[u].z; }
      if (!mv[u].w) { xv[u].w += a * pv[u].w; rv[u].w -= a * qv[u].w; }
      x4[k] = xv[u];
      r4[k] = rv[u];
      acc += sum4(rv[u]);
    }
  }
  block_partial(acc, part);
}

// r -= mean (CEF); z = Dinv r + coarse correction of the node's plane on free nodes; partials
// of r.z and r.r (mean_part: the partials of sum r, or nullptr for the mean in the state)
__global__ void k_precond4(float* __restrict__ r, float* __restrict__ z,
                           const float* __restrict__ dinv, const unsigned char* __restrict__ mask,
                           const CgState* s, int project, int64_t n4, double* __restrict__ part_rz,
                           double* __restrict__ part_rr, const double* __restrict__ cy,
                           uint32_t plane4, const double* __restrict__ mean_part, int64_t n) {
  double mean_d = 0.0;
  if (project) mean_d = mean_part ? block_sum_partials(mean_part) * (1.0 / (double)n) : s->mean;
  const float mean = (float)mean_d;
  float4* r4 = reinterpret_cast<float4*>(r);
  float4* z4 = reinterpret_cast<float4*>(z);
  const float4* d4 = reinterpret_cast<const float4*>(dinv);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(mask);
  const int64_t g = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x;
  float a1 = 0.f, a2 = 0.f;
  for (int64_t q0 = g; q0 < n4; q0 += V4B * V4S) {
    float4 rv[V4B], dv[V4B];
    uchar4 mv[V4B];
    float cv[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = q0 + u * V4S;
      if (k < n4) {
        rv[u] = r4[k];
        dv[u] = d4[k];
        mv[u] = m4[k];
        cv[u] = cy ? (float)cy[(uint32_t)k / plane4] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = q0 + u * V4S;
      if (k >= n4) continue;
      float4 ri = rv[u], zi;
      if (project) {
        ri.x -= mean; ri.y -= mean; ri.z -= mean; ri.w -= mean;
        r4[k] = ri;
      }
      zi.x = mv[u].x ? 0.f : dv[u].x * ri.x + cv[u];
      zi.y = mv[u].y ? 0.f : dv[u].y * ri.y + cv[u];
      zi.z = mv[u].z ? 0.f : dv[u].z * ri.z + cv[u];
      zi.w = mv[u].w ? 0.f : dv[u].w * ri.w + cv[u];
      z4[k] = zi;
      a1 += ri.x * zi.x + ri.y * zi.y + ri.z * zi.z + ri.w * zi.w;
      a2 += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
    }
  }
  double t1 = (double)a1, t2 = (double)a2;
  block_sum2(t1, t2);
  if (threadIdx.x == 0) { part_rz[blockIdx.x] = t1; part_rr[blockIdx.x] = t2; }
}

// p = z + beta p (skipped once converged)
__global__ void k_update_p4(float* __restrict__ p, const float* __restrict__ z, const CgState* s,
                            int64_t n4) {
  fe_pdl_enter();
  if (s->done && s->alpha == 0.0) return;
  const float b = (float)s->beta;
  float4* p4 = reinterpret_cast<float4*>(p);
  const float4* z4 = reinterpret_cast<const float4*>(z);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n4;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float4 zv = z4[k];
    float4 pv = p4[k];
    pv.x = zv.x + b * pv.x; pv.y = zv.y + b * pv.y; pv.z = zv.z + b * pv.z; pv.w = zv.w + b * pv.w;
    p4[k] = pv;
  }
}

// sum of x over the free nodes of plane blockIdx.x (plane4 groups per plane)
__global__ void k_plane_sum4(const float* __restrict__ x, const unsigned char* __restrict__ mask,
                             int64_t plane4, double* __restrict__ out) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(mask);
  const int64_t base = (int64_t)blockIdx.x * plane4;
  float a = 0.f;
  for (int64_t i0 = threadIdx.x; i0 < plane4; i0 += V4B * fe::RED_THREADS) {
    float4 xv[V4B];
    uchar4 mv[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t i = i0 + u * fe::RED_THREADS;
      if (i < plane4) { xv[u] = x4[base + i]; mv[u] = m4[base + i]; }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      if (i0 + u * fe::RED_THREADS >= plane4) continue;
      a += (mv[u].x ? 0.f : xv[u].x) + (mv[u].y ? 0.f : xv[u].y) + (mv[u].z ? 0.f : xv[u].z) +
           (mv[u].w ? 0.f : xv[u].w);
    }
  }
  block_partial(a, out);
}

// ---- float iteration with the plane coarse space: seven launches per iteration ----------------
// The grid-wide scalars (alpha, the mean, beta and the convergence test) are finished by the
// last block of the kernel that produces their partials (a ticket taken after each block's
// partial is visible), so no single-block finishing launch sits between the vector kernels.
// The last block sums the partials in index order, as a separate finishing kernel would.

// returns true in every thread of the block that finished last (ticket reset for the next use)
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}
__device__ __forceinline__ double sum_partials_cg(const double* part, int np) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += __ldcg(part + i);
  return block_sum(s);
}

// p.q partials; the last block sets pq and alpha = r.z / p.q
__global__ void k_psum4_alpha(const float* __restrict__ p, const float* __restrict__ q, int64_t n4,
                              double* __restrict__ part, CgState* s) {
  fe_pdl_enter();
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.f;
  for (int64_t q0 = g; q0 < n4; q0 += V4B * stride) {
    float4 a[V4B], b[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = q0 + u * stride;
      if (k < n4) { a[u] = p4[k]; b[u] = q4[k]; }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u)
      if (q0 + u * stride < n4)
        acc += a[u].x * b[u].x + a[u].y * b[u].y + a[u].z * b[u].z + a[u].w * b[u].w;
  }
  const double t = block_sum((double)acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (last_block(&s->ticket[0])) {
    const double pq = sum_partials_cg(part, gridDim.x);
    if (threadIdx.x == 0) {
      s->pq = pq;
      s->alpha = (s->done || pq == 0.0) ? 0.0 : s->rz / pq;
      s->ticket[0] = 0;
    }
  }
}

// x += alpha p, r -= alpha q on free nodes, by plane segments: block b takes segment b % nseg of
// plane b / nseg (seglen groups of four nodes) and writes the segment's sum of r to seg[b]
__global__ void k_update_xr4s(float* __restrict__ x, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q,
                              const unsigned char* __restrict__ mask, const CgState* s,
                              int64_t plane4, int nseg, int seglen, double* __restrict__ seg) {
  fe_pdl_enter();
  const float a = (float)s->alpha;
  const int pl = blockIdx.x / nseg, sg = blockIdx.x - pl * nseg;
  const int64_t lo = (int64_t)pl * plane4 + (int64_t)sg * seglen;
  const int64_t hi = min((int64_t)pl * plane4 + plane4, lo + seglen);
  float4* x4 = reinterpret_cast<float4*>(x);
  float4* r4 = reinterpret_cast<float4*>(r);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(mask);
  float acc = 0.f;
  for (int64_t k0 = lo + threadIdx.x; k0 < hi; k0 += V4B * (int64_t)blockDim.x) {
    float4 xv[V4B], rv[V4B], pv[V4B], qv[V4B];
    uchar4 mv[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = k0 + u * (int64_t)blockDim.x;
      if (k < hi) { xv[u] = x4[k]; rv[u] = r4[k]; pv[u] = p4[k]; qv[u] = q4[k]; mv[u] = m4[k]; }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = k0 + u * (int64_t)blockDim.x;
      if (k >= hi) continue;
      if (!mv[u].x) { xv[u].x += a * pv[u].x; rv[u].x -= a * qv[u].x; }
      if (!mv[u].y) { xv[u].y += a * pv[u].y; rv[u].y -= a * qv[u].y; }
      if (!mv[u].z) { xv[u].z += a * pv[u].z; rv[u].z -= a * qv[u].z; }
      if (!mv[u].w) { xv[u].w += a * pv[u].w; rv[u].w -= a * qv[u].w; }
      x4[k] = xv[u];
      r4[k] = rv[u];
      acc += sum4(rv[u]);
    }
  }
  const double t = block_sum((double)acc);
  if (threadIdx.x == 0) seg[blockIdx.x] = t;
}

// The coarse correction from the plane-segment sums: b_k = (sum of plane k's segments) -
// mean cnt_k, mean = (sum of all segments) / n under the CEF projection (block 0 records it),
// then one warp per coarse unknown j: y_j = sum_k Ainv[j][k] b_k (Ainv symmetric), in float.
__global__ void k_coarse_apply4(const double* __restrict__ seg, int nseg,
                                const double* __restrict__ cnt, const double* __restrict__ Ainv,
                                CgState* st, int project, int nz, double inv_n,
                                float* __restrict__ yf) {
  fe_pdl_enter();
  extern __shared__ double cb[];   // b[nz]
  double loc = 0.0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    double sk = 0.0;
    for (int t = 0; t < nseg; ++t) sk += seg[(int64_t)k * nseg + t];
    cb[k] = sk;
    loc += sk;
  }
  const double total = block_sum(loc);
  const double mean = project ? total * inv_n : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->mean = mean;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) cb[k] -= mean * cnt[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j < nz) {
    const double* row = Ainv + (int64_t)j * nz;
    double a = 0.0;
    for (int k = lane; k < nz; k += 32) a += row[k] * cb[k];
    a = warp_sum(a);
    if (lane == 0) yf[j] = (float)a;
  }
}

// r -= mean (the state's, CEF); z = Dinv r + yf[plane] on free nodes; r.z and r.r partials
// per plane segment (block b: segment b % nseg of plane b / nseg, so the coarse correction of
// the block's plane is one value); the last block finishes beta, r.z, |r|^2, the iteration
// count and the convergence test
__global__ void k_precond4s_beta(float* __restrict__ r, float* __restrict__ z,
                                 const float* __restrict__ dinv,
                                 const unsigned char* __restrict__ mask, CgState* s, int project,
                                 int64_t plane4, int nseg, int seglen,
                                 double* __restrict__ part_rz, double* __restrict__ part_rr,
                                 const float* __restrict__ yf) {
  fe_pdl_enter();
  const float mean = project ? (float)s->mean : 0.f;
  const int pl = blockIdx.x / nseg, sg = blockIdx.x - pl * nseg;
  const int64_t lo = (int64_t)pl * plane4 + (int64_t)sg * seglen;
  const int64_t hi = min((int64_t)pl * plane4 + plane4, lo + seglen);
  const float cv = yf[pl];
  float4* r4 = reinterpret_cast<float4*>(r);
  float4* z4 = reinterpret_cast<float4*>(z);
  const float4* d4 = reinterpret_cast<const float4*>(dinv);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(mask);
  float a1 = 0.f, a2 = 0.f;
  for (int64_t k0 = lo + threadIdx.x; k0 < hi; k0 += V4B * (int64_t)blockDim.x) {
    float4 rv[V4B], dv[V4B];
    uchar4 mv[V4B];
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = k0 + u * (int64_t)blockDim.x;
      if (k < hi) { rv[u] = r4[k]; dv[u] = d4[k]; mv[u] = m4[k]; }
    }
#pragma unroll
    for (int u = 0; u < V4B; ++u) {
      const int64_t k = k0 + u * (int64_t)blockDim.x;
      if (k >= hi) continue;
      float4 ri = rv[u], zi;
      if (project) {
        ri.x -= mean; ri.y -= mean; ri.z -= mean; ri.w -= mean;
        r4[k] = ri;
      }
      zi.x = mv[u].x ? 0.f : dv[u].x * ri.x + cv;
      zi.y = mv[u].y ? 0.f : dv[u].y * ri.y + cv;
      zi.z = mv[u].z ? 0.f : dv[u].z * ri.z + cv;
      zi.w = mv[u].w ? 0.f : dv[u].w * ri.w + cv;
      z4[k] = zi;
      a1 += ri.x * zi.x + ri.y * zi.y + ri.z * zi.z + ri.w * zi.w;
      a2 += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
    }
  }
  double t1 = (double)a1, t2 = (double)a2;
  block_sum2(t1, t2);
  if (threadIdx.x == 0) { part_rz[blockIdx.x] = t1; part_rr[blockIdx.x] = t2; }
  if (last_block(&s->ticket[1])) {
    double rz = 0.0, rr = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      rz += __ldcg(part_rz + i);
      rr += __ldcg(part_rr + i);
    }
    block_sum2(rz, rr);
    if (threadIdx.x == 0) {
      if (!s->done) {
        s->beta = s->rz == 0.0 ? 0.0 : rz / s->rz;
        s->rz = rz;
        s->rr = rr;
        s->iters += 1;
        if (rr <= s->tol2 || s->iters >= s->maxit) s->done = 1;
      } else {
        s->beta = 0.0;
      }
      s->ticket[1] = 0;
    }
  }
}

// one block of RED_THREADS per plane, deterministic order
template <typename V>
__global__ void k_plane_sum(const V* __restrict__ x, const unsigned char* __restrict__ mask,
                            int64_t plane, double* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * plane;
  V a = V(0);
  for (int64_t i = threadIdx.x; i < plane; i += fe::RED_THREADS) {
    const int64_t id = base + i;
    if (!mask[id]) a += x ? x[id] : V(1);
  }
  const double t = block_sum((double)a);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// v = sum of the coarse basis functions of the planes gz = color (mod period)
__global__ void k_plane_color(const unsigned char* __restrict__ mask, int64_t plane, int period,
                              int color, double* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (!mask[i] && (int)((i / plane) % period) == color) ? 1.0 : 0.0;
}

// v = the coarse basis functions of in-plane mode (tx, ty) on the planes gz = color (mod
// period): tx[gx] ty[gy] on their free nodes, 0 elsewhere
__global__ void k_mode_color(const unsigned char* __restrict__ mask, int64_t plane, int NX,
                             const double* __restrict__ tx, const double* __restrict__ ty,
                             int period, int color, double* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gz = i / plane, r = i - gz * plane;
    const int gy = (int)(r / NX), gx = (int)(r - (int64_t)gy * NX);
    v[i] = (!mask[i] && (int)(gz % period) == color) ? tx[gx] * ty[gy] : 0.0;
  }
}

// out[j] = sum over the free nodes of plane j of tx[gx] ty[gy] x (one block per plane,
// deterministic order)
__global__ void k_mode_plane_sum(const double* __restrict__ x, const unsigned char* __restrict__ mask,
                                 int64_t plane, int NX, const double* __restrict__ tx,
                                 const double* __restrict__ ty, double* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * plane;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < plane; i += fe::RED_THREADS) {
    const int gy = (int)(i / NX), gx = (int)(i - (int64_t)gy * NX);
    if (!mask[base + i]) a += tx[gx] * ty[gy] * x[base + i];
  }
  const double t = block_sum(a);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

constexpr int COARSE_COLS = 64;   // coarse unknowns per block of k_coarse_apply

// y = Ainv (s - mean cnt): Ainv is the symmetric (pseudo-)inverse of the coarse matrix,
// dense [nz][nz]; block b computes y[64 b, 64 b + 64) with four k-slices per column
__global__ void k_coarse_apply(const double* __restrict__ sums, const double* __restrict__ cnt,
                               const double* __restrict__ Ainv, const CgState* st, int project,
                               int nz, double* __restrict__ y, const double* __restrict__ mean_part,
                               double inv_n) {
  extern __shared__ double cb[];                    // b[nz], then partials [4][64]
  double* part = cb + nz;
  double mean = 0.0;
  if (project) mean = mean_part ? block_sum_partials(mean_part) * inv_n : st->mean;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) cb[k] = sums[k] - mean * cnt[k];
  __syncthreads();
  const int jl = threadIdx.x % COARSE_COLS, ks = threadIdx.x / COARSE_COLS;
  const int j = blockIdx.x * COARSE_COLS + jl;
  double a = 0.0;
  if (j < nz)
    for (int k = ks; k < nz; k += 4) a += Ainv[(int64_t)k * nz + j] * cb[k];
  part[ks * COARSE_COLS + jl] = a;
  __syncthreads();
  if (ks == 0 && j < nz)
    y[j] = (part[jl] + part[COARSE_COLS + jl]) + (part[2 * COARSE_COLS + jl] + part[3 * COARSE_COLS + jl]);
}

// In-place inverse of the SPD matrix A [m][m] (row-major) by Cholesky; false if not SPD.
bool spd_inverse(std::vector<double>& A, int m) {
  std::vector<double> L((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    double d = A[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double v = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = v / ljj;
    }
  }
  // W = L^-1 (lower triangular), then A^-1 = W^T W
  std::vector<double> W((size_t)m * m, 0.0);
  for (int c = 0; c < m; ++c) {
    W[(size_t)c * m + c] = 1.0 / L[(size_t)c * m + c];
    for (int i = c + 1; i < m; ++i) {
      double v = 0.0;
      for (int k = c; k < i; ++k) v -= L[(size_t)i * m + k] * W[(size_t)k * m + c];
      W[(size_t)i * m + c] = v / L[(size_t)i * m + i];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = 0.0;
      for (int k = i; k < m; ++k) v += W[(size_t)k * m + i] * W[(size_t)k * m + j];
      A[(size_t)i * m + j] = v;
      A[(size_t)j * m + i] = v;
    }
  return true;
}

PGeom make_geom(const fe_mesh* m) {
  PGeom g;
  g.NX = m->NX; g.NY = m->NY; g.NZ = m->NZ; g.p = m->p;
  g.hx = m->h[0]; g.hy = m->h[1]; g.hz = m->h[2];
  g.Lz = m->desc.L[2];
  for (int k = 0; k < FE_MAXN1; ++k) {
    g.xi[k] = k <= m->p ? m->xi[k] : 0.0;
    g.K1diag[k] = k <= m->p ? m->K1[k][k] : 0.0;
    g.M1diag[k] = k <= m->p ? m->M1[k][k] : 0.0;
  }
  g.ax = m->h[1] * m->h[2] / (2.0 * m->h[0]);
  g.ay = m->h[0] * m->h[2] / (2.0 * m->h[1]);
  g.az = m->h[0] * m->h[1] / (2.0 * m->h[2]);
  return g;
}

}  // namespace

extern "C" fe_status fe_poisson_rhs(fe_mesh* m, const double* rho, double* f, double* rho_out,
                                    double* b_out) {
  if (!m || !f) return fe_fail(FE_EINVAL, "fe_poisson_rhs: null argument");
  if (!m->d_rho) return fe_fail(FE_EINVAL, "fe_poisson_rhs: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_phi;
  const double* r = rho ? rho : m->d_rho;
  // reuse the setup kernel's load computation through a scratch mask / dinv
  void* wsp;
  FE_TRY(fe_ws(m, WS_CG, n * (sizeof(double) * 2 + 1) + 64, &wsp));
  double* dinv = (double*)wsp;
  double* phi = dinv + n;
  unsigned char* mask = (unsigned char*)(phi + n);
  fe_poisson_bc bc = {};
  bc.kind = FE_BIAS_CEF;
  k_setup<<<fe::grid_for(n), 256, 0, m->stream>>>(make_geom(m), bc, m->d_mass, r, m->d_b,
                                                   m->d_vlms, nullptr, nullptr, f, dinv, mask,
                                                   phi, n); fe_count_launch();
  if (rho_out) FE_CUDA(cudaMemcpyAsync(rho_out, r, n * 8, cudaMemcpyDeviceToDevice, m->stream));
  if (b_out) FE_CUDA(cudaMemcpyAsync(b_out, m->d_b, n * 8, cudaMemcpyDeviceToDevice, m->stream));
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

static fe_status poisson_solve_on(fe_mesh* m, const double* rho, const fe_poisson_bc* bc,
                                  double* phi, double* vbare, fe_solve_info* info,
                                  bool use_graph, const double* f_ext, const double* phic_ext);

static bool same_constraints(const fe_poisson_bc& a, const fe_poisson_bc& b) {
  if (a.kind != b.kind) return false;
  if (a.kind == FE_BIAS_CEF) return true;
  if (a.zA != b.zA || a.zB != b.zB || a.has_patch != b.has_patch) return false;
  if (!a.has_patch) return true;
  return std::memcmp(a.patch_lo, b.patch_lo, sizeof a.patch_lo) == 0 &&
         std::memcmp(a.patch_hi, b.patch_hi, sizeof a.patch_hi) == 0;
}

// The coarse-space inverse for the constraint set of bc (cached on the mesh): the plane
// matrix Ac[j][i] = e_j^T K e_i from 2p + 1 operator applications (planes of one colour are
// 2p + 1 apart, so each plane meets at most one of them), then its inverse on the active
// planes (planes with free nodes; CEF: the last one is dropped to fix the constant), zero
// elsewhere.  v and w are n-double scratch vectors.  *Ainv is nullptr when the coarse
// space is off or its matrix is not numerically SPD.
constexpr int MODES_MIN_CELLS = 8;

// The in-plane modes of wavenumber one added to every plane's coarse function by
// FE_PRECOND_JACOBI_PLANES_MODES: cos and sin of 2 pi x / Lx, of 2 pi y / Ly, and the four
// products (cos x cos y, cos x sin y, sin x cos y, sin x sin y).  On a mesh without
// constrained phi nodes the cell-translation invariance of K (and its reflection symmetry in
// x and in y) decouples them from one another and from the plane indicator, so each has its
// own nz x nz coarse matrix R_m K R_m^T (built, like the plane matrix, from K applied to
// colourings of its basis functions).  Workspace WS_PMODES: the NM - 1 inverses (float),
// then the tables as float (cos x, sin x [NX]; cos y, sin y [NY]) and as double (the same and
// the two ones tables).
static fe_status modes_setup(fe_mesh* m, const unsigned char* mask, double* v, double* w,
                             const double* hcnt, const float** Amodes, const float** mtab) {
  const int nz = m->NZ, NX = m->NX, NY = m->NY;
  const int64_t plane = (int64_t)NX * NY, n = m->n_phi;
  for (int j = 0; j < nz; ++j)
    if (hcnt[j] < (double)plane - 0.5) return FE_OK;   // constrained nodes: planes only
  if (NX % 4 != 0) return FE_OK;
  constexpr int NMOD = fe_cg::MODES_NM - 1;
  const size_t nzz = (size_t)nz * nz;
  const size_t bytes = sizeof(float) * NMOD * nzz + sizeof(float) * 2 * ((size_t)NX + NY) + 64 +
                       sizeof(double) * 3 * ((size_t)NX + NY);
  void* wsp;
  FE_TRY(fe_ws(m, WS_PMODES, bytes, &wsp));
  float* dAm = (float*)wsp;   // the mode inverses in float (enough for a coarse correction)
  float* dtab = dAm + NMOD * nzz;
  double* dtd = (double*)(((uintptr_t)(dtab + 2 * (NX + NY)) + 63) & ~(uintptr_t)63);
  // node coordinates along x and y (GLL points of each cell)
  const double two_pi = 2.0 * 3.14159265358979323846;
  std::vector<double> htd(3 * ((size_t)NX + NY));
  std::vector<float> htab(2 * ((size_t)NX + NY));
  const double Lx = m->nx * m->h[0], Ly = m->ny * m->h[1];
  for (int g = 0; g < NX; ++g) {
    const double x = (g / m->p) * m->h[0] + 0.5 * (m->xi[g % m->p] + 1.0) * m->h[0];
    htd[g] = std::cos(two_pi * x / Lx);
    htd[NX + g] = std::sin(two_pi * x / Lx);
    htd[2 * NX + 2 * NY + g] = 1.0;
  }
  for (int g = 0; g < NY; ++g) {
    const double y = (g / m->p) * m->h[1] + 0.5 * (m->xi[g % m->p] + 1.0) * m->h[1];
    htd[2 * NX + g] = std::cos(two_pi * y / Ly);
    htd[2 * NX + NY + g] = std::sin(two_pi * y / Ly);
    htd[3 * NX + 2 * NY + g] = 1.0;
  }
  for (size_t i = 0; i < htab.size(); ++i) htab[i] = (float)htd[i];
  cudaStream_t st = m->stream;
  FE_CUDA(cudaMemcpyAsync(dtd, htd.data(), sizeof(double) * htd.size(), cudaMemcpyHostToDevice, st));
  FE_CUDA(cudaMemcpyAsync(dtab, htab.data(), sizeof(float) * htab.size(), cudaMemcpyHostToDevice, st));
  const double* ones_x = dtd + 2 * NX + 2 * NY;
  const double* ones_y = ones_x + NX;
  const double* cxd = dtd;
  const double* sxd = dtd + NX;
  const double* cyd = dtd + 2 * NX;
  const double* syd = dtd + 2 * NX + NY;
  const double* tx[8] = {cxd, sxd, ones_x, ones_x, cxd, cxd, sxd, sxd};
  const double* ty[8] = {ones_y, ones_y, cyd, syd, cyd, syd, cyd, syd};
  static_assert(NMOD <= 8, "mode tables");
  const int period = 2 * m->p + 1;
  std::vector<double> wsum((size_t)period * nz);
  void* sws;
  FE_TRY(fe_ws(m, WS_PCOARSE, sizeof(double) * (nzz + 2 * (size_t)nz) + 64, &sws));
  double* dsum = (double*)sws + nzz + nz;
  for (int md = 0; md < NMOD; ++md) {
    for (int c = 0; c < period; ++c) {
      k_mode_color<<<fe::grid_for(n), 256, 0, st>>>(mask, plane, NX, tx[md], ty[md], period, c,
                                                    v, n);
      fe_count_launch();
      FE_TRY(fe_poisson_apply_K(m, v, w));
      k_mode_plane_sum<<<nz, fe::RED_THREADS, 0, st>>>(w, mask, plane, NX, tx[md], ty[md], dsum);
      fe_count_launch();
      FE_CUDA(cudaMemcpyAsync(wsum.data() + (size_t)c * nz, dsum, sizeof(double) * nz,
                              cudaMemcpyDeviceToHost, st));
    }
    FE_CUDA(cudaStreamSynchronize(st));
    std::vector<double> A(nzz, 0.0);
    for (int j = 0; j < nz; ++j)
      for (int i = j - m->p; i <= j + m->p; ++i)
        if (i >= 0 && i < nz) A[(size_t)j * nz + i] = wsum[(size_t)(i % period) * nz + j];
    for (int a = 0; a < nz; ++a)
      for (int b = 0; b < a; ++b) {
        const double s2 = 0.5 * (A[(size_t)a * nz + b] + A[(size_t)b * nz + a]);
        A[(size_t)a * nz + b] = A[(size_t)b * nz + a] = s2;
      }
    if (!spd_inverse(A, nz)) return FE_OK;   // (not expected: planes only)
    std::vector<float> Af(A.begin(), A.end());
    FE_CUDA(cudaMemcpyAsync(dAm + md * nzz, Af.data(), sizeof(float) * nzz,
                            cudaMemcpyHostToDevice, st));
    FE_CUDA(cudaStreamSynchronize(st));
  }
  *Amodes = dAm;
  *mtab = dtab;
  return FE_OK;
}

static fe_status coarse_setup(fe_mesh* m, const fe_poisson_bc* bc, const unsigned char* mask,
                              double* v, double* w, const double** Ainv, const double** cnt,
                              const float** Amodes, const float** mtab) {
  *Ainv = nullptr;
  *cnt = nullptr;
  *Amodes = nullptr;
  *mtab = nullptr;
  const int nz = m->NZ;
  if ((m->poisson_precond != FE_PRECOND_JACOBI_PLANES &&
       m->poisson_precond != FE_PRECOND_JACOBI_PLANES_MODES) || nz > 2048)
    return FE_OK;
  // (the wavenumber-one modes are slow modes of the Jacobi-preconditioned operator only when
  // the slab spans many cells in x and y; on narrow slabs they would only add to the top of
  // the preconditioned spectrum)
  const bool want_modes = m->poisson_precond == FE_PRECOND_JACOBI_PLANES_MODES &&
                          m->nx >= MODES_MIN_CELLS && m->ny >= MODES_MIN_CELLS;
  const int64_t plane = (int64_t)m->NX * m->NY, n = m->n_phi;
  void* wsp;
  FE_TRY(fe_ws(m, WS_PCOARSE, sizeof(double) * ((size_t)nz * nz + 2 * (size_t)nz) + 64, &wsp));
  double* dA = (double*)wsp;
  double* dcnt = dA + (size_t)nz * nz;
  double* dsum = dcnt + nz;
  if (m->pc_state != 0 && m->pc_nz == nz && same_constraints(m->pc_key, *bc) &&
      (!want_modes || m->pc_modes != 0)) {
    if (m->pc_state == 1) { *Ainv = dA; *cnt = dcnt; }
    if (m->pc_state == 1 && want_modes && m->pc_modes == 1) {
      const float* mw = static_cast<const float*>(m->ws[WS_PMODES]);
      *Amodes = mw;
      *mtab = mw + (fe_cg::MODES_NM - 1) * (size_t)nz * nz;
    }
    return FE_OK;
  }
  m->pc_modes = 0;
  cudaStream_t st = m->stream;
  const int period = 2 * m->p + 1;
  std::vector<double> wsum((size_t)period * nz), hcnt(nz);
  k_plane_sum<double><<<nz, fe::RED_THREADS, 0, st>>>(nullptr, mask, plane, dcnt); fe_count_launch();
  FE_CUDA(cudaMemcpyAsync(hcnt.data(), dcnt, sizeof(double) * nz, cudaMemcpyDeviceToHost, st));
  for (int c = 0; c < period; ++c) {
    k_plane_color<<<fe::grid_for(n), 256, 0, st>>>(mask, plane, period, c, v, n); fe_count_launch();
    FE_TRY(fe_poisson_apply_K(m, v, w));
    k_plane_sum<<<nz, fe::RED_THREADS, 0, st>>>(w, mask, plane, dsum); fe_count_launch();
    FE_CUDA(cudaMemcpyAsync(wsum.data() + (size_t)c * nz, dsum, sizeof(double) * nz,
                            cudaMemcpyDeviceToHost, st));
  }
  FE_CUDA(cudaStreamSynchronize(st));
  // active planes and the dense coarse matrix on them
  std::vector<int> act;
  for (int j = 0; j < nz; ++j) if (hcnt[j] > 0.5) act.push_back(j);
  if (bc->kind == FE_BIAS_CEF && !act.empty()) act.pop_back();
  const int na = (int)act.size();
  std::vector<int> pos(nz, -1);
  for (int a = 0; a < na; ++a) pos[act[a]] = a;
  std::vector<double> A((size_t)na * na, 0.0);
  for (int a = 0; a < na; ++a) {
    const int j = act[a];
    for (int i = j - m->p; i <= j + m->p; ++i) {
      if (i < 0 || i >= nz || pos[i] < 0) continue;
      A[(size_t)a * na + pos[i]] = wsum[(size_t)(i % period) * nz + j];
    }
  }
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < a; ++b) {
      const double s2 = 0.5 * (A[(size_t)a * na + b] + A[(size_t)b * na + a]);
      A[(size_t)a * na + b] = A[(size_t)b * na + a] = s2;
    }
  m->pc_key = *bc;
  m->pc_nz = nz;
  if (na == 0 || !spd_inverse(A, na)) {
    m->pc_state = 2;
    m->pc_modes = 2;
    return FE_OK;
  }
  std::vector<double> full((size_t)nz * nz, 0.0);
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < na; ++b) full[(size_t)act[a] * nz + act[b]] = A[(size_t)a * na + b];
  FE_CUDA(cudaMemcpyAsync(dA, full.data(), sizeof(double) * full.size(), cudaMemcpyHostToDevice, st));
  FE_CUDA(cudaStreamSynchronize(st));
  m->pc_state = 1;
  *Ainv = dA;
  *cnt = dcnt;
  if (want_modes) {
    FE_TRY(modes_setup(m, mask, v, w, hcnt.data(), Amodes, mtab));
    m->pc_modes = *Amodes ? 1 : 2;
  }
  return FE_OK;
}

// The solve runs on the mesh's private non-blocking stream (ordered after the caller's stream
// with an event, and the caller's stream ordered after it), because CUDA graphs cannot be
// captured on the legacy default stream.  When the caller's stream is itself being captured,
// the iterations are issued directly instead (the host convergence test still synchronises,
// so the solve as a whole cannot be part of a caller's graph).
static fe_status poisson_solve_forked(fe_mesh* m, const double* rho, const fe_poisson_bc* bc,
                                     double* phi, double* vbare, fe_solve_info* info,
                                     const double* f_ext, const double* phic_ext) {
  FE_TRY(fe_activate(m));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FE_CUDA(cudaStreamIsCapturing(m->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return poisson_solve_on(m, rho, bc, phi, vbare, info, false, f_ext, phic_ext);
  cudaStream_t user = m->stream;
  FE_CUDA(cudaEventRecord(m->ev_fork, user));
  FE_CUDA(cudaStreamWaitEvent(m->aux_stream, m->ev_fork, 0));
  m->stream = m->aux_stream;
  fe_status st = poisson_solve_on(m, rho, bc, phi, vbare, info, true, f_ext, phic_ext);
  m->stream = user;
  cudaError_t e1 = cudaEventRecord(m->ev_join, m->aux_stream);
  cudaError_t e2 = cudaStreamWaitEvent(user, m->ev_join, 0);
  if (st == FE_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) {
    cudaGetLastError();
    return fe_fail(FE_ECUDA, "Poisson stream join failed");
  }
  return st;
}

extern "C" fe_status fe_poisson_constraints(fe_mesh* m, const fe_poisson_bc* bc,
                                            unsigned char* mask, double* values) {
  if (!m || !bc || !mask || !values) return fe_fail(FE_EINVAL, "fe_poisson_constraints: null argument");
  if (!m->d_rho) return fe_fail(FE_EINVAL, "fe_poisson_constraints: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_phi;
  void* wsp;
  FE_TRY(fe_ws(m, WS_CG, n * sizeof(double) * 2 + 64, &wsp));
  double* f = (double*)wsp;
  double* dinv = f + n;
  k_setup<<<fe::grid_for(n), 256, 0, m->stream>>>(make_geom(m), *bc, m->d_mass, m->d_rho, m->d_b,
                                                   m->d_vlms, nullptr, nullptr, f, dinv, mask,
                                                   values, n); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

extern "C" fe_status fe_vbare_phi(fe_mesh* m, const double* phi, const fe_poisson_bc* bc,
                                  double* out) {
  if (!m || !phi || !bc || !out) return fe_fail(FE_EINVAL, "fe_vbare_phi: null argument");
  if (!m->d_vlms) return fe_fail(FE_EINVAL, "fe_vbare_phi: call fe_set_atoms first");
  FE_TRY(fe_activate(m));
  k_vbare<<<fe::grid_for(m->n_phi), 256, 0, m->stream>>>(make_geom(m), phi, m->d_vlms, bc->field,
                                                           bc->kind == FE_BIAS_CEF, 0, out,
                                                           m->n_phi); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

extern "C" fe_status fe_poisson_solve(fe_mesh* m, const double* rho, const fe_poisson_bc* bc,
                                      double* phi, double* vbare, fe_solve_info* info) {
  if (!m || !bc || !phi) return fe_fail(FE_EINVAL, "fe_poisson_solve: null argument");
  return poisson_solve_forked(m, rho, bc, phi, vbare, info, nullptr, nullptr);
}

extern "C" fe_status fe_poisson_solve_load(fe_mesh* m, const double* f, const fe_poisson_bc* bc,
                                           const double* phic, double* phi,
                                           fe_solve_info* info) {
  if (!m || !bc || !phi || !f) return fe_fail(FE_EINVAL, "fe_poisson_solve_load: null argument");
  return poisson_solve_forked(m, nullptr, bc, phi, nullptr, info, f, phic);
}

// ---- preconditioned CG in a given vector precision -------------------------------------------
namespace {

template <typename V>
struct CgBuf {
  V *x, *r, *z, *p, *q;
  const V* dinv;
  const unsigned char* mask;
  double *pa, *pb, *pc, *pd;   // block partials
  CgState* s;
  const double* Ainv;          // coarse space (nullptr: Jacobi only)
  const double* ccnt;
  double* csum;
  double* cy;
  double* seg;                 // float path with the coarse space: plane-segment sums of r, then
                               // the preconditioner's r.z and r.r partials (3 nz nseg doubles)
  float* cyf;                  // float coarse correction per plane
  int nseg;                    // segments per plane
  // in-plane mode coarse space (persistent float iteration only; nullptr: planes only):
  // the mode inverses [MODES_NM - 1][nz][nz] (float) and the float mode tables (cos x,
  // sin x, cos y, sin y)
  const float* Amodes;
  const float* mtab;
};

fe_status apply_K_v(fe_mesh* m, const double* x, double* y) { return fe_poisson_apply_K(m, x, y); }
fe_status apply_K_v(fe_mesh* m, const float* x, float* y) { return fe_kcell_apply_f32(m, x, y); }

// CG on K_ff x = r0 from the iterate in b.x, whose masked residual is in b.r (projected by
// the first preconditioner call for CEF).  Stops at |r|^2 <= tol2_abs, or (tol2_abs <= 0)
// |r|^2 <= rtol^2 |r0|^2, or after maxit iterations.  Blocks of iterations replay a CUDA graph
// captured on first use (*exec, kept by the caller for the rest of the solve).
// Between blocks of iterations the optional hook sees the state and chooses: CG_CONTINUE,
// CG_STOP, CG_REPLACED (it has written a new residual into b.r: the run recomputes its
// preconditioned form and r.z and continues with the same search direction) or
// CG_RESTARTED (the same, and the search direction restarts from the new preconditioned
// residual).
enum { CG_CONTINUE = 0, CG_STOP = 1, CG_REPLACED = 2, CG_RESTARTED = 3 };
constexpr int PERSIST_ITERS = 4096;

template <typename V, typename Hook>
fe_status cg_run(fe_mesh* m, const CgBuf<V>& b, int project, double rtol, double tol2_abs,
                 int maxit, bool use_graph, cudaGraphExec_t* exec, int64_t* graph_kernels,
                 CgState* out, const fe_cg::FusedStop* stop, Hook&& hook) {
  if constexpr (std::is_same<V, float>::value) {
    // the float operator's scratch exists before any graph capture
    void* w = nullptr;
    FE_TRY(fe_ws(m, WS_KCELL, fe_kcell_scratch_bytes(m), &w));
  }
  const int64_t n = m->n_phi;
  const int64_t plane = (int64_t)m->NX * m->NY;
  const int nzp = m->NZ;
  cudaStream_t st = m->stream;
  const int gb = fe::grid_for(n);
  const int cblocks = (nzp + COARSE_COLS - 1) / COARSE_COLS;
  const size_t csmem = sizeof(double) * ((size_t)nzp + 4 * COARSE_COLS);
  const double* cy = b.Ainv ? b.cy : nullptr;
  // four nodes per access for float vectors whose planes hold a multiple of four nodes
  auto al16 = [](const void* q) { return ((uintptr_t)q % 16) == 0; };
  bool v4 = false;
  if constexpr (std::is_same<V, float>::value)
    v4 = plane % 4 == 0 && al16(b.x) && al16(b.r) && al16(b.z) && al16(b.p) && al16(b.q) &&
         al16(b.dinv) && ((uintptr_t)b.mask % 4) == 0;
  const int64_t n4 = n / 4;
  auto psum = [&](const V* x, const V* y, double* part) {
    if constexpr (std::is_same<V, float>::value) {
      if (v4) {
        k_psum4<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(x, y, n4, part); fe_count_launch();
        return;
      }
    }
    k_psum<V><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(x, y, n, part); fe_count_launch();
  };
  auto precond = [&](const double* mean_part) {
    if constexpr (std::is_same<V, float>::value) {
      if (v4) {
        k_precond4<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(b.r, b.z, b.dinv, b.mask, b.s,
                                                               project, n4, b.pc, b.pd, cy,
                                                               (uint32_t)(plane / 4), mean_part, n);
        fe_count_launch();
        return;
      }
    }
    k_precond<V><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(b.r, b.z, b.dinv, b.mask, b.s, project,
                                                             n, b.pc, b.pd, cy, plane, mean_part);
    fe_count_launch();
  };
  auto coarse = [&](const double* mean_part) {
    if (!b.Ainv) return;
    bool done4 = false;
    if constexpr (std::is_same<V, float>::value) {
      if (v4) {
        k_plane_sum4<<<nzp, fe::RED_THREADS, 0, st>>>(b.r, b.mask, plane / 4, b.csum);
        fe_count_launch();
        done4 = true;
      }
    }
    if (!done4) {
      k_plane_sum<V><<<nzp, fe::RED_THREADS, 0, st>>>(b.r, b.mask, plane, b.csum); fe_count_launch();
    }
    k_coarse_apply<<<cblocks, 4 * COARSE_COLS, csmem, st>>>(b.csum, b.ccnt, b.Ainv, b.s, project,
                                                            nzp, b.cy, mean_part, 1.0 / (double)n);
    fe_count_launch();
  };
  CgState s0 = {};
  s0.maxit = maxit;
  FE_CUDA(cudaMemcpyAsync(b.s, &s0, sizeof(CgState), cudaMemcpyHostToDevice, st));
  if (project) {
    psum(b.r, nullptr, b.pa);
    k_fin_mean<<<1, fe::RED_BLOCKS, 0, st>>>(b.pa, b.s, 1.0 / (double)n); fe_count_launch();
  }
  coarse(nullptr);
  precond(nullptr);
  k_fin_init<<<1, fe::RED_BLOCKS, 0, st>>>(b.pc, b.pd, b.s, rtol, tol2_abs); fe_count_launch();
  k_copy<V><<<gb, 256, 0, st>>>(b.z, b.p, n); fe_count_launch();
  FE_CUDA(cudaGetLastError());

  // float, four nodes per access, coarse space present: the seven-launch iteration
  const bool fused = v4 && b.Ainv && b.nseg > 0 && b.seg && b.cyf;
  const int seglen = fused ? (int)((plane / 4 + b.nseg - 1) / b.nseg) : 0;
  auto iteration = [&]() -> fe_status {
    FE_TRY(apply_K_v(m, b.p, b.q));
    if constexpr (std::is_same<V, float>::value) {
      if (fused) {
        // (programmatic dependent launches: each kernel waits for its predecessor at entry)
        const float* cp = b.p;
        const float* cq = b.q;
        FE_CUDA(fe_launch_pdl(k_psum4_alpha, dim3(fe::RED_BLOCKS), dim3(fe::RED_THREADS), 0, st,
                              cp, cq, n4, b.pa, b.s));
        fe_count_launch();
        const unsigned char* cmask = b.mask;
        const CgState* cs = b.s;
        const int64_t pl4 = plane / 4;
        FE_CUDA(fe_launch_pdl(k_update_xr4s, dim3(nzp * b.nseg), dim3(256), 0, st, b.x, b.r, cp, cq,
                              cmask, cs, pl4, b.nseg, seglen, b.seg));
        fe_count_launch();
        const double* cseg = b.seg;
        const double* ccnt = b.ccnt;
        const double* cAinv = b.Ainv;
        const double inv_n = 1.0 / (double)n;
        FE_CUDA(fe_launch_pdl(k_coarse_apply4, dim3((nzp + 7) / 8), dim3(256),
                              sizeof(double) * nzp, st, cseg, b.nseg, ccnt, cAinv, b.s, project,
                              nzp, inv_n, b.cyf));
        fe_count_launch();
        const int64_t nsegs = (int64_t)nzp * b.nseg;
        const float* cdinv = b.dinv;
        const float* cyf = b.cyf;
        double* prz = b.seg + nsegs;
        double* prr = b.seg + 2 * nsegs;
        FE_CUDA(fe_launch_pdl(k_precond4s_beta, dim3(nzp * b.nseg), dim3(256), 0, st, b.r, b.z,
                              cdinv, cmask, b.s, project, pl4, b.nseg, seglen, prz, prr, cyf));
        fe_count_launch();
        const float* cz = b.z;
        FE_CUDA(fe_launch_pdl(k_update_p4, dim3(fe::grid_for(n4)), dim3(256), 0, st, b.p, cz, cs,
                              n4));
        fe_count_launch();
        return FE_OK;
      }
    }
    psum(b.p, b.q, b.pa);
    bool xr4 = false;
    if constexpr (std::is_same<V, float>::value) {
      if (v4) {
        k_update_xr4<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(b.x, b.r, b.p, b.q, b.mask, b.s, n4,
                                                                 b.pb, b.pa);
        fe_count_launch();
        xr4 = true;
      }
    }
    if (!xr4) {
      k_update_xr<V><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(b.x, b.r, b.p, b.q, b.mask, b.s, n,
                                                                 b.pb, b.pa);
      fe_count_launch();
    }
    coarse(b.pb);
    precond(b.pb);
    k_fin_beta<<<1, fe::RED_BLOCKS, 0, st>>>(b.pc, b.pd, b.s); fe_count_launch();
    bool p4 = false;
    if constexpr (std::is_same<V, float>::value) {
      if (v4) {
        k_update_p4<<<fe::grid_for(n4), 256, 0, st>>>(b.p, b.z, b.s, n4); fe_count_launch();
        p4 = true;
      }
    }
    if (!p4) { k_update_p<V><<<gb, 256, 0, st>>>(b.p, b.z, b.s, n); fe_count_launch(); }
    return FE_OK;
  };
  // the same iteration in one cooperative kernel per interval between the hook's actions
  bool persist = false;
  if constexpr (std::is_same<V, float>::value)
    persist = fused && use_graph && m->poisson_iter == FE_POISSON_ITER_PERSISTENT &&
              fe_cg::fused_available(m);
  const int per_graph = 16;
  if (use_graph && !persist && !*exec) {
    cudaGraph_t graph = nullptr;
    FE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    fe_status cst = FE_OK;
    const int64_t before = fe_kernel_launches();
    for (int i = 0; i < per_graph && cst == FE_OK; ++i) cst = iteration();
    // captured launches run only when the graph is replayed
    *graph_kernels = fe_kernel_launches() - before;
    fe_count_launch(-*graph_kernels);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (cst != FE_OK) { cudaGetLastError(); if (graph) cudaGraphDestroy(graph); return cst; }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ECUDA, "CG capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *exec = nullptr;
      return fe_fail(FE_ECUDA, "CG graph: %s", cudaGetErrorString(e));
    }
  }
  auto replaced = [&](bool restart) {
    if (project) {
      psum(b.r, nullptr, b.pa);
      k_fin_mean<<<1, fe::RED_BLOCKS, 0, st>>>(b.pa, b.s, 1.0 / (double)n); fe_count_launch();
    }
    coarse(nullptr);
    precond(nullptr);
    k_fin_replace<<<1, fe::RED_BLOCKS, 0, st>>>(b.pc, b.pd, b.s); fe_count_launch();
    if (restart) { k_copy<V><<<gb, 256, 0, st>>>(b.z, b.p, n); fe_count_launch(); }
  };
  int launched = 0;
  while (true) {
    FE_CUDA(cudaMemcpyAsync(out, b.s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    if (persist) {
      if (out->fused_err)
        return fe_fail(FE_ETIMEOUT, "Poisson CG: a grid barrier of the persistent iteration "
                       "gave up after %d iterations", out->iters);
      launched = out->iters;
    }
    int action = out->done ? CG_STOP : CG_CONTINUE;
    FE_TRY(hook(*out, &action));
    if (action == CG_STOP || launched >= maxit) break;
    if (action == CG_REPLACED || action == CG_RESTARTED) {
      replaced(action == CG_RESTARTED);
      FE_CUDA(cudaGetLastError());
    }
    if (persist) {
      if constexpr (std::is_same<V, float>::value) {
        const fe_cg::FusedCg fb{b.x, b.r, b.z, b.p, b.q, b.dinv, b.mask, b.Ainv, b.ccnt, b.s,
                                project, b.Amodes, b.mtab};
        const fe_cg::FusedStop none{-1.0, HUGE_VAL, maxit};
        // at most PERSIST_ITERS iterations per launch, so the host regains control
        FE_TRY(fe_cg::fused_run(m, fb, PERSIST_ITERS, stop ? *stop : none));
      }
    } else if (use_graph) {
      cudaError_t e = cudaGraphLaunch(*exec, st);
      if (e != cudaSuccess) return fe_fail(FE_ECUDA, "CG graph launch: %s", cudaGetErrorString(e));
      fe_count_launch(*graph_kernels);
      launched += per_graph;
    } else {
      FE_TRY(iteration());
      launched += 1;
    }
  }
  return FE_OK;
}

struct GraphExec {
  cudaGraphExec_t e = nullptr;
  ~GraphExec() { if (e) cudaGraphExecDestroy(e); }
};

}  // namespace

static fe_status poisson_solve_on(fe_mesh* m, const double* rho, const fe_poisson_bc* bc,
                                  double* phi, double* vbare, fe_solve_info* info,
                                  bool use_graph, const double* f_ext, const double* phic_ext) {
  if (bc->kind != FE_BIAS_CEF && bc->kind != FE_BIAS_CPD)
    return fe_fail(FE_EINVAL, "fe_poisson_solve: bad bias kind");
  if (!(bc->rtol > 0.0) || bc->max_iter < 1)
    return fe_fail(FE_EINVAL, "fe_poisson_solve: need rtol > 0 and max_iter >= 1");
  if (!m->d_rho && !(f_ext && (phic_ext || bc->kind == FE_BIAS_CEF)))
    return fe_fail(FE_EINVAL, "fe_poisson_solve: call fe_set_atoms first");
  if (bc->kind == FE_BIAS_CPD && !(bc->zA < bc->zB))
    return fe_fail(FE_EINVAL, "fe_poisson_solve: need zA < zB");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_phi;
  if (n >= (int64_t(1) << 32))
    return fe_fail(FE_EUNSUPPORTED, "fe_poisson_solve: 2^32 or more phi nodes");
  const int nzp = m->NZ;
  cudaStream_t st = m->stream;
  const bool mixed = m->poisson_arith == FE_POISSON_MIXED;
  // workspace: double f, dinv, r, z, p, q; float r, z, p, q, delta, dinv (mixed only);
  // partials, coarse correction, two states, mask
  void* wsp;
  const size_t nd = (size_t)n * 6, nf = mixed ? (size_t)n * 6 : 0;
  // float path, planes of a multiple of four nodes: plane segments of at most 1024 groups of
  // four nodes (one batch of loads per thread in the segment kernel)
  const int64_t plane_n = (int64_t)m->NX * m->NY;
  const int nseg = (mixed && plane_n % 4 == 0) ? (int)((plane_n / 4 + 1023) / 1024) : 0;
  size_t bytes = nd * sizeof(double) + nf * sizeof(float) + 64 +
                 (4 * fe::RED_BLOCKS + (size_t)nzp) * sizeof(double) + 2 * sizeof(CgState) + n + 256 +
                 3 * (size_t)nzp * nseg * sizeof(double) + (size_t)nzp * sizeof(float) + 256;
  FE_TRY(fe_ws(m, WS_CG, bytes, &wsp));
  double* f = (double*)wsp;
  double* dinv = f + n;
  double* r = dinv + n;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  float* fl = (float*)(q + n);
  double* pa = (double*)(((uintptr_t)(fl + nf) + 63) & ~(uintptr_t)63);
  double* pb = pa + fe::RED_BLOCKS;
  double* pc = pb + fe::RED_BLOCKS;
  double* pd = pc + fe::RED_BLOCKS;
  double* cyv = pd + fe::RED_BLOCKS;
  CgState* s = (CgState*)(cyv + nzp);
  CgState* sref = s + 1;
  unsigned char* mask = (unsigned char*)(sref + 1);
  double* segp = (double*)(((uintptr_t)(mask + n) + 255) & ~(uintptr_t)255);
  float* cyf = (float*)(segp + 3 * (size_t)nzp * nseg);
  const int project = bc->kind == FE_BIAS_CEF;
  const double* rh = rho ? rho : m->d_rho;
  const int gb = fe::grid_for(n);
  PGeom g = make_geom(m);

  k_setup<<<gb, 256, 0, st>>>(g, *bc, m->d_mass, rh, m->d_b, m->d_vlms, f_ext, phic_ext, f, dinv,
                              mask, phi, n); fe_count_launch();
  if (project) {
    k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(f, nullptr, n, pa); fe_count_launch();
    k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(m->d_mass, nullptr, n, pb); fe_count_launch();
    k_fin_project_load<<<1, fe::RED_BLOCKS, 0, st>>>(pa, pb, s); fe_count_launch();
    k_project_load<<<gb, 256, 0, st>>>(f, m->d_mass, s, n); fe_count_launch();
  }
  // coarse space of z-planes (z and q serve as scratch before the iteration starts)
  const double* Ainv = nullptr;
  const double* ccnt = nullptr;
  const float* Amodes = nullptr;
  const float* mtab = nullptr;
  FE_TRY(coarse_setup(m, bc, mask, z, q, &Ainv, &ccnt, &Amodes, &mtab));
  double* csum = Ainv ? (double*)(ccnt + nzp) : nullptr;

  // double residual r = f - K phi (masked; CEF: minus its mean) and |r|^2 on the host
  auto residual = [&](double* rr) -> fe_status {
    FE_TRY(fe_poisson_apply_K(m, phi, q));
    k_resid0<<<gb, 256, 0, st>>>(f, q, mask, r, n); fe_count_launch();
    if (project) {
      k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(r, nullptr, n, pa); fe_count_launch();
      k_fin_mean<<<1, fe::RED_BLOCKS, 0, st>>>(pa, sref, 1.0 / (double)n); fe_count_launch();
      k_sub_mean<<<gb, 256, 0, st>>>(r, sref, n); fe_count_launch();
    }
    k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(r, r, n, pb); fe_count_launch();
    k_fin_rr<<<1, fe::RED_BLOCKS, 0, st>>>(pb, sref); fe_count_launch();
    CgState h;
    FE_CUDA(cudaMemcpyAsync(&h, sref, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    *rr = h.rr;
    return FE_OK;
  };
  double rr = 0.0;
  FE_TRY(residual(&rr));
  if (!std::isfinite(rr)) {
    // a NaN or infinity in rho, the atoms or the constraint values: no iteration can mean
    // anything, so report it instead of running to the iteration cap
    if (info) { info->iters = 0; info->rel_residual = rr; info->status = FE_EINVAL; }
    return fe_fail(FE_EINVAL, "Poisson: the initial residual is not finite (NaN or infinity "
                   "in the density, the atoms or the constraint values)");
  }
  const double bnorm2 = rr;
  const double tol2 = bc->rtol * bc->rtol * bnorm2;
  int used = 0;
  CgState hs = {};
  GraphExec gexec_f, gexec_d;
  int64_t gk_f = 0, gk_d = 0;

  auto no_hook = [](const CgState&, int*) { return FE_OK; };
  if (mixed && rr > tol2) {
    // One float CG (operator, vectors and preconditioner in float; dot products in double)
    // whose residual is replaced by the double residual f - K phi whenever the float
    // residual has dropped by 1e2 since the last replacement (reliable updates, Sleijpen
    // and van der Vorst 1996): phi accumulates the float iterate in double and the stopping
    // test is on the double residual.  The Krylov direction is kept across a replacement
    // while the float recurrence still tracks the true residual (within 2x in norm) and
    // restarted otherwise.  When a replacement interval stops reducing the double
    // residual, the double CG finishes from the current phi.
    float* rf = fl;
    float* zf = rf + n;
    float* pf = zf + n;
    float* qf = pf + n;
    float* df = qf + n;
    float* dinvf = df + n;
    k_to_float<<<gb, 256, 0, st>>>(dinv, dinvf, n); fe_count_launch();
    k_to_float<<<gb, 256, 0, st>>>(r, rf, n); fe_count_launch();
    FE_CUDA(cudaMemsetAsync(df, 0, sizeof(float) * n, st));
    CgBuf<float> bf{df, rf, zf, pf, qf, dinvf, mask, pa, pb, pc, pd, s, Ainv, ccnt, csum, cyv,
                    segp, cyf, nseg, Amodes, mtab};
    double rr_last = rr;
    int it_last = 0, stalls = 0, breakdowns = 0;
    // the persistent iteration returns as soon as one of the tests below would act
    fe_cg::FusedStop stop{1e-4 * rr_last, 1e2 * rr_last, it_last + 512};
    auto restop = [&]() { stop = fe_cg::FusedStop{1e-4 * rr_last, 1e2 * rr_last, it_last + 512}; };
    auto reliable = [&](const CgState& cs, int* action) -> fe_status {
      used = cs.iters;
      // A kept search direction that no longer matches the replaced residual can make the
      // float recurrence grow without bound (seen far below float resolution of the
      // original load).  Its correction since the last replacement is then discarded (phi
      // and the double residual r are those of that replacement) and the iteration
      // restarts from r; a second breakdown hands the solve to the double CG.
      if (!(cs.rr <= 1e2 * rr_last)) {
        FE_CUDA(cudaMemsetAsync(df, 0, sizeof(float) * n, st));
        if (++breakdowns >= 2 || cs.iters >= bc->max_iter) { *action = CG_STOP; return FE_OK; }
        it_last = cs.iters;
        restop();
        k_to_float<<<gb, 256, 0, st>>>(r, rf, n); fe_count_launch();
        *action = CG_RESTARTED;
        return FE_OK;
      }
      const bool trigger = cs.done || cs.rr <= 1e-4 * rr_last || cs.iters - it_last >= 512;
      if (!trigger) { *action = CG_CONTINUE; return FE_OK; }
      k_add_delta<<<gb, 256, 0, st>>>(phi, df, mask, n); fe_count_launch();
      FE_CUDA(cudaMemsetAsync(df, 0, sizeof(float) * n, st));
      FE_TRY(residual(&rr));
      if (rr <= tol2 || cs.iters >= bc->max_iter) { *action = CG_STOP; return FE_OK; }
      stalls = rr > 0.25 * rr_last ? stalls + 1 : 0;
      if (stalls >= 2) { *action = CG_STOP; return FE_OK; }
      // keep the search direction only while the float recurrence still tracks the true
      // residual; a larger gap would scale the next step by their ratio, so restart
      const bool tracks = rr <= 4.0 * cs.rr;
      rr_last = rr;
      it_last = cs.iters;
      restop();
      k_to_float<<<gb, 256, 0, st>>>(r, rf, n); fe_count_launch();
      *action = tracks ? CG_REPLACED : CG_RESTARTED;
      return FE_OK;
    };
    FE_TRY(cg_run<float>(m, bf, project, 0.0, tol2, bc->max_iter, use_graph, &gexec_f.e, &gk_f,
                         &hs, &stop, reliable));
  }
  if (rr > tol2 && used < bc->max_iter) {
    // double CG from the current phi (the whole solve when the mixed mode is off)
    CgBuf<double> bd{phi, r, z, p, q, dinv, mask, pa, pb, pc, pd, s, Ainv, ccnt, csum, cyv,
                     nullptr, nullptr, 0, nullptr, nullptr};
    FE_TRY(cg_run<double>(m, bd, project, bc->rtol, tol2, bc->max_iter - used, use_graph,
                          &gexec_d.e, &gk_d, &hs, nullptr, no_hook));
    used += hs.iters;
    rr = hs.rr;
  }
  if (project) {
    k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(m->d_mass, phi, n, pa); fe_count_launch();
    k_psum<double><<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(m->d_mass, nullptr, n, pb); fe_count_launch();
    k_shift_mean<<<gb, fe::RED_BLOCKS, 0, st>>>(phi, pa, pb, n); fe_count_launch();
  }
  if (vbare) {
    k_vbare<<<fe::grid_for(m->n_psi), 256, 0, st>>>(g, phi, m->d_vlms, bc->field, project,
                                                      m->gz_lo, vbare, m->n_psi); fe_count_launch();
  }
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaStreamSynchronize(st));
  double rel = bnorm2 > 0 ? std::sqrt(rr / bnorm2) : 0.0;
  bool conv = bnorm2 == 0.0 || rr <= tol2;
  if (info) {
    info->iters = used;
    info->rel_residual = rel;
    info->status = conv ? FE_OK : FE_ENOCONV;
  }
  if (!conv)
    return fe_fail(FE_ENOCONV, "Poisson CG: %d iterations, relative residual %.3e", used, rel);
  return FE_OK;
}

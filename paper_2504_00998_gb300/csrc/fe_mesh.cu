// Mesh construction, 1D element rules and the library's error state.
//
// Section 2.3 (FE discretization): C0 Lagrange polynomials of degree p on GLL nodes.
// The 1D rules are computed here from the Legendre recurrence: GLL nodes are -1, +1 and
// the roots of P_p', with weights 2 / (p (p+1) P_p^2); the element matrices
// K1_ij = int l_i' l_j' and M1_ij = int l_i l_j on [-1, 1] use (p+1)-point Gauss-Legendre
// quadrature, exact for their degree <= 2p integrands.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "fe_internal.h"

// ---- error state --------------------------------------------------------------------------
static thread_local char g_err[512] = "";

fe_status fe_fail(fe_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

extern "C" const char* fe_last_error(void) { return g_err; }

static std::atomic<int64_t> g_launches{0};

void fe_count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t fe_kernel_launches(void) { return g_launches.load(); }

// ---- 1D rules ---------------------------------------------------------------------------------
// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // P_n' = n (x P_n - P_{n-1}) / (x^2 - 1) away from the end points
  *dP = (std::fabs(x * x - 1.0) > 1e-300) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.0;
}

static void gll_rule(int p, double* x, double* w) {
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    // Newton on q = P_p' with q' = (2 x P_p' - p (p+1) P_p) / (1 - x^2) (Legendre's equation)
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, &P, &dP);
      double d2 = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

static void gauss_rule(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre(q, t, &P, &dP);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// Lagrange basis on nodes xn[0..n): value and derivative of l_i at t
static void lagrange(int n, const double* xn, int i, double t, double* l, double* dl) {
  double v = 1.0, d = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double f = (t - xn[j]) / (xn[i] - xn[j]);
    d = d * f + v / (xn[i] - xn[j]);
    v *= f;
  }
  *l = v;
  *dl = d;
}

static void element_matrices(fe_mesh* m) {
  const int n1 = m->p + 1;
  double gq[FE_MAXN1 + 1], gw[FE_MAXN1 + 1];
  gauss_rule(n1, gq, gw);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) { m->K1[i][j] = 0.0; m->M1[i][j] = 0.0; m->G1[i][j] = 0.0; }
  for (int a = 0; a < n1; ++a) {
    double l[FE_MAXN1], dl[FE_MAXN1];
    for (int i = 0; i < n1; ++i) lagrange(n1, m->xi, i, gq[a], &l[i], &dl[i]);
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) {
        m->K1[i][j] += gw[a] * dl[i] * dl[j];
        m->M1[i][j] += gw[a] * l[i] * l[j];
        m->G1[i][j] += gw[a] * l[i] * dl[j];
      }
  }
}

// Coefficient tables of the tensor-product operator (see KronCoef).
static void build_coef(fe_mesh* m, bool hamiltonian, KronCoef* c) {
  const int p = m->p, n1 = p + 1;
  const double hx = m->h[0], hy = m->h[1], hz = m->h[2];
  const double ax = hy * hz / (2.0 * hx), ay = hx * hz / (2.0 * hy), az = hx * hy / (2.0 * hz);
  double sig[FE_MAXN1];
  for (int k = 0; k < n1; ++k) {
    double mloc = (k == 0 || k == p) ? 2.0 * m->w[0] : m->w[k];
    sig[k] = hamiltonian ? 1.0 / std::sqrt(mloc) : 1.0;
  }
  std::memset(c, 0, sizeof(*c));
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n1; ++k) {
      c->AyM[j][k] = m->M1[j][k] * sig[k];
      c->AyK[j][k] = ay * m->K1[j][k] * sig[k];
      c->AxM[j][k] = m->M1[j][k] * sig[k];
      c->AxK[j][k] = ax * m->K1[j][k] * sig[k];
      c->AzK[j][k] = az * m->K1[j][k];
      c->AzM[j][k] = m->M1[j][k];
    }
  for (int k = 0; k < n1; ++k) { c->sig[k] = sig[k]; c->wz[k] = m->w[k]; }
  c->ax = ax;
  c->ay = ay;
  c->mass_scale = hamiltonian ? 1 : 0;
  c->zin = hamiltonian ? 1.0 / std::sqrt(m->J) : 1.0;
  c->zout = hamiltonian ? 0.5 / std::sqrt(m->J) : 1.0;
}

// The Bloch operator A = M^-1/2 (kx Gx + ky Gy) M^-1/2 (Section 2.1, the -i k.grad term of
// H^k_loc) in the tensor-product form of KronCoef: G^x = (hy hz / 4) G1 (x) M1 (x) M1 over
// the reference matrices (x derivative; y and z masses), G^y likewise; no z derivative, so
// AzK = 0; the symmetric mass scaling of the Hamiltonian without its factor 1/2.
static void build_coef_bloch(fe_mesh* m, KronCoef* c) {
  build_coef(m, true, c);
  const int n1 = m->p + 1;
  const double hx = m->h[0], hy = m->h[1], hz = m->h[2];
  const double gx = m->kx * hy * hz / 4.0, gy = m->ky * hx * hz / 4.0;
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n1; ++k) {
      c->AxK[j][k] = gx * m->G1[j][k] * c->sig[k];
      c->AyK[j][k] = gy * m->G1[j][k] * c->sig[k];
      c->AzK[j][k] = 0.0;
    }
  c->zout = 1.0 / std::sqrt(m->J);
  c->ax = c->ay = 0.0;
  c->cplx = 1;
}

// ---- device helpers -------------------------------------------------------------------------
__global__ void k_coords(int NX, int NY, int NZ, int p, double hx, double hy, double hz,
                         const double* __restrict__ xi, double* __restrict__ out, int64_t n) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n) return;
  int gx = (int)(id % NX);
  int gy = (int)((id / NX) % NY);
  int gz = (int)(id / ((int64_t)NX * NY));
  out[3 * id + 0] = (gx / p) * hx + (xi[gx % p] + 1.0) * 0.5 * hx;
  out[3 * id + 1] = (gy / p) * hy + (xi[gy % p] + 1.0) * 0.5 * hy;
  out[3 * id + 2] = (gz / p) * hz + (xi[gz % p] + 1.0) * 0.5 * hz;
}

__global__ void k_mass(int NX, int NY, int NZ, int p, double J, const double* __restrict__ w,
                       double* __restrict__ out, int64_t n) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n) return;
  int gx = (int)(id % NX);
  int gy = (int)((id / NX) % NY);
  int gz = (int)(id / ((int64_t)NX * NY));
  double mx = (gx % p == 0) ? 2.0 * w[0] : w[gx % p];
  double my = (gy % p == 0) ? 2.0 * w[0] : w[gy % p];
  double mz = (gz % p == 0) ? ((gz == 0 || gz == NZ - 1) ? w[0] : 2.0 * w[0]) : w[gz % p];
  out[id] = J * mx * my * mz;
}

fe_status fe_activate(const fe_mesh* m) {
  FE_CUDA(cudaSetDevice(m->device));
  return FE_OK;
}

fe_status fe_ws(fe_mesh* m, int slot, size_t bytes, void** out) {
  if (m->ws_bytes[slot] < bytes) {
    if (m->ws[slot]) {
      FE_CUDA(cudaStreamSynchronize(m->stream));
      FE_CUDA(cudaFree(m->ws[slot]));
      m->ws[slot] = nullptr;
      m->ws_bytes[slot] = 0;
    }
    if (cudaMalloc(&m->ws[slot], bytes) != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ENOMEM, "workspace of %zu bytes could not be allocated", bytes);
    }
    m->ws_bytes[slot] = bytes;
  }
  *out = m->ws[slot];
  return FE_OK;
}

static double* upload_small(const double* h, int n) {
  double* d = nullptr;
  if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return nullptr;
  cudaMemcpy(d, h, n * sizeof(double), cudaMemcpyHostToDevice);
  return d;
}

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" fe_status fe_mesh_create(const fe_mesh_desc* d, fe_mesh** out) {
  if (!d || !out) return fe_fail(FE_EINVAL, "fe_mesh_create: null argument");
  *out = nullptr;
  if (d->p < 1 || d->p > FE_MAXP) return fe_fail(FE_EINVAL, "p = %d outside [1, %d]", d->p, FE_MAXP);
  for (int k = 0; k < 3; ++k) {
    if (!(d->L[k] > 0.0) || !std::isfinite(d->L[k]))
      return fe_fail(FE_EINVAL, "box length %d must be positive", k);
    if (d->ncell[k] < 1) return fe_fail(FE_EINVAL, "ncell[%d] must be >= 1", k);
  }
  int64_t NX = (int64_t)d->ncell[0] * d->p, NY = (int64_t)d->ncell[1] * d->p;
  int64_t NZ = (int64_t)d->ncell[2] * d->p + 1;
  if (NX * NY * NZ > ((int64_t)1 << 31) - 1)
    return fe_fail(FE_EINVAL, "mesh has more than 2^31 nodes");
  for (int f = 0; f < 2; ++f)
    if (d->psi_z[f] != FE_FACE_NEUMANN && d->psi_z[f] != FE_FACE_DIRICHLET)
      return fe_fail(FE_EINVAL, "psi_z[%d] invalid", f);
  if (d->ncell[2] * d->p - (d->psi_z[0] == FE_FACE_DIRICHLET) - (d->psi_z[1] == FE_FACE_DIRICHLET) < 0)
    return fe_fail(FE_EINVAL, "no psi planes left");

  fe_mesh* m = new (std::nothrow) fe_mesh();
  if (!m) return fe_fail(FE_ENOMEM, "host allocation failed");
  m->desc = *d;
  m->device = d->device;
  m->stream = (cudaStream_t)d->stream;
  m->p = d->p;
  m->nx = d->ncell[0]; m->ny = d->ncell[1]; m->nz = d->ncell[2];
  m->NX = (int)NX; m->NY = (int)NY; m->NZ = (int)NZ;
  m->gz_lo = d->psi_z[0] == FE_FACE_DIRICHLET ? 1 : 0;
  m->gz_hi = d->psi_z[1] == FE_FACE_DIRICHLET ? m->nz * m->p - 1 : m->nz * m->p;
  m->NZs = m->gz_hi - m->gz_lo + 1;
  m->n_phi = NX * NY * NZ;
  m->n_psi = NX * NY * (int64_t)m->NZs;
  m->n_cells = (int64_t)m->nx * m->ny * m->nz;
  for (int k = 0; k < 3; ++k) m->h[k] = d->L[k] / d->ncell[k];
  m->J = m->h[0] * m->h[1] * m->h[2] / 8.0;
  gll_rule(m->p, m->xi, m->w);
  element_matrices(m);
  fe_quad_setup_basis(m);
  build_coef(m, true, &m->coefH);
  build_coef(m, false, &m->coefK);

  fe_status st = fe_activate(m);
  if (st != FE_OK) { delete m; return st; }
  if (cudaMalloc(&m->d_mass, m->n_phi * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fe_fail(FE_ENOMEM, "mass allocation failed");
  }
  double* d_w = upload_small(m->w, m->p + 1);
  if (!d_w) { fe_mesh_destroy(m); return fe_fail(FE_ENOMEM, "allocation failed"); }
  int nb = (int)((m->n_phi + 255) / 256);
  k_mass<<<nb, 256, 0, m->stream>>>(m->NX, m->NY, m->NZ, m->p, m->J, d_w, m->d_mass, m->n_phi); fe_count_launch();
  cudaError_t e = cudaStreamSynchronize(m->stream);
  cudaFree(d_w);
  if (e != cudaSuccess) {
    fe_mesh_destroy(m);
    return fe_fail(FE_ECUDA, "mass kernel: %s", cudaGetErrorString(e));
  }
  if (cublasCreate(&m->cublas) != CUBLAS_STATUS_SUCCESS ||
      cusolverDnCreate(&m->cusolver) != CUSOLVER_STATUS_SUCCESS) {
    fe_mesh_destroy(m);
    return fe_fail(FE_ECUDA, "cuBLAS / cuSOLVER handle creation failed");
  }
  cublasSetStream(m->cublas, m->stream);
  cusolverDnSetStream(m->cusolver, m->stream);
  {
    // FE_FP64_EMULATION=1 lets cuBLAS run the double GEMMs of the Rayleigh-Ritz step with its
    // fixed-point emulation (double-precision accuracy, tensor-core throughput)
    const char* emu = std::getenv("FE_FP64_EMULATION");
    if (emu && emu[0] == '1')
      cublasSetMathMode(m->cublas, CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH);
  }
  if (cudaStreamCreateWithFlags(&m->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    fe_mesh_destroy(m);
    return fe_fail(FE_ECUDA, "stream / event creation failed");
  }
  *out = m;
  return FE_OK;
}

extern "C" fe_status fe_mesh_destroy(fe_mesh* m) {
  if (!m) return FE_OK;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  for (int i = 0; i < FE_NWS; ++i) if (m->ws[i]) cudaFree(m->ws[i]);
  fe_nonlocal_free(m);
  fe_quad_free(m);
  if (m->tc_err_pinned) cudaFreeHost(m->tc_err_pinned);
  if (m->ktc_err_pinned) cudaFreeHost(m->ktc_err_pinned);
  cudaFree(m->d_veff);
  cudaFree(m->d_veff_f);
  cudaFree(m->d_atoms);
  cudaFree(m->d_vlms);
  cudaFree(m->d_rho);
  cudaFree(m->d_b);
  cudaFree(m->d_mass);
  delete[] m->h_atoms;
  if (m->cublas) cublasDestroy(m->cublas);
  if (m->syevj_params) cusolverDnDestroySyevjInfo(m->syevj_params);
  if (m->cusolver) cusolverDnDestroy(m->cusolver);
  if (m->aux_stream) cudaStreamDestroy(m->aux_stream);
  if (m->ev_fork) cudaEventDestroy(m->ev_fork);
  if (m->ev_join) cudaEventDestroy(m->ev_join);
  delete m;
  return FE_OK;
}

extern "C" fe_status fe_mesh_info(const fe_mesh* m, int64_t* n_phi, int64_t* n_psi,
                                  int64_t* n_cells) {
  if (!m) return fe_fail(FE_EINVAL, "fe_mesh_info: null mesh");
  if (n_phi) *n_phi = m->n_phi;
  if (n_psi) *n_psi = m->n_psi;
  if (n_cells) *n_cells = m->n_cells;
  return FE_OK;
}

extern "C" fe_status fe_mesh_set_stream(fe_mesh* m, void* stream) {
  if (!m) return fe_fail(FE_EINVAL, "fe_mesh_set_stream: null mesh");
  m->stream = (cudaStream_t)stream;
  m->desc.stream = stream;
  if (m->cublas) cublasSetStream(m->cublas, m->stream);
  if (m->cusolver) cusolverDnSetStream(m->cusolver, m->stream);
  return FE_OK;
}

extern "C" fe_status fe_set_option(fe_mesh* m, int option, int64_t value) {
  if (!m) return fe_fail(FE_EINVAL, "fe_set_option: null mesh");
  switch (option) {
    case FE_OPT_RR_PRODUCTS:
      if (value != FE_RR_PRODUCTS_F64 && value != FE_RR_PRODUCTS_TC32)
        return fe_fail(FE_EINVAL, "fe_set_option: bad Rayleigh-Ritz product mode");
      m->rr_products = (int)value;
      return FE_OK;
    case FE_OPT_POISSON_PRECOND:
      if (value != FE_PRECOND_JACOBI && value != FE_PRECOND_JACOBI_PLANES &&
          value != FE_PRECOND_JACOBI_PLANES_MODES)
        return fe_fail(FE_EINVAL, "fe_set_option: bad Poisson preconditioner");
      m->poisson_precond = (int)value;
      return FE_OK;
    case FE_OPT_POISSON_ARITH:
      if (value != FE_POISSON_F64 && value != FE_POISSON_MIXED)
        return fe_fail(FE_EINVAL, "fe_set_option: bad Poisson arithmetic");
      m->poisson_arith = (int)value;
      return FE_OK;
    case FE_OPT_POISSON_ITER:
      if (value != FE_POISSON_ITER_PERSISTENT && value != FE_POISSON_ITER_LAUNCHES)
        return fe_fail(FE_EINVAL, "fe_set_option: bad Poisson iteration mode");
      m->poisson_iter = (int)value;
      return FE_OK;
    case FE_OPT_TEST_CG_STALL:
      if (value < -1 || value > 0x7fffffff)
        return fe_fail(FE_EINVAL, "fe_set_option: bad stalled block");
      m->cg_stall = (int)value;
      return FE_OK;
    case FE_OPT_RR_EIGEN:
      if (value != FE_RR_EIGEN_SYEVD && value != FE_RR_EIGEN_SYEVJ)
        return fe_fail(FE_EINVAL, "fe_set_option: bad Rayleigh-Ritz eigensolver");
      m->rr_eigen = (int)value;
      return FE_OK;
    default:
      return fe_fail(FE_EINVAL, "fe_set_option: unknown option %d", option);
  }
}

extern "C" fe_status fe_node_coords(const fe_mesh* m, double* xyz) {
  if (!m || !xyz) return fe_fail(FE_EINVAL, "fe_node_coords: null argument");
  FE_TRY(fe_activate(m));
  double* d_xi = upload_small(m->xi, m->p + 1);
  if (!d_xi) return fe_fail(FE_ENOMEM, "allocation failed");
  int nb = (int)((m->n_phi + 255) / 256);
  k_coords<<<nb, 256, 0, m->stream>>>(m->NX, m->NY, m->NZ, m->p, m->h[0], m->h[1], m->h[2],
                                      d_xi, xyz, m->n_phi); fe_count_launch();
  cudaError_t e = cudaStreamSynchronize(m->stream);
  cudaFree(d_xi);
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "coords kernel: %s", cudaGetErrorString(e));
  return FE_OK;
}

extern "C" fe_status fe_lumped_mass(const fe_mesh* m, double* out) {
  if (!m || !out) return fe_fail(FE_EINVAL, "fe_lumped_mass: null argument");
  FE_TRY(fe_activate(m));
  FE_CUDA(cudaMemcpyAsync(out, m->d_mass, m->n_phi * sizeof(double), cudaMemcpyDeviceToDevice,
                          m->stream));
  return FE_OK;
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

extern "C" fe_status fe_set_potential(fe_mesh* m, const double* veff) {
  if (!m || !veff) return fe_fail(FE_EINVAL, "fe_set_potential: null argument");
  FE_TRY(fe_activate(m));
  if (!m->d_veff) {
    if (cudaMalloc(&m->d_veff, m->n_psi * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_veff_f, m->n_psi * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ENOMEM, "potential allocation failed");
    }
  }
  FE_CUDA(cudaMemcpyAsync(m->d_veff, veff, m->n_psi * sizeof(double), cudaMemcpyDeviceToDevice,
                          m->stream));
  int nb = (int)((m->n_psi + 255) / 256);
  k_d2f<<<nb, 256, 0, m->stream>>>(m->d_veff, m->d_veff_f, m->n_psi); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  m->has_potential = true;
  m->has_quad = false;   // back to the collocated potential
  return FE_OK;
}

extern "C" fe_status fe_set_atoms(fe_mesh* m, int n, const double* R, const double* Z,
                                  double sigma_b, double rc_loc, double sigma_rho) {
  if (!m || n < 0 || (n > 0 && (!R || !Z)))
    return fe_fail(FE_EINVAL, "fe_set_atoms: bad arguments");
  if (!(sigma_b > 0) || !(rc_loc > 0) || !(sigma_rho > 0))
    return fe_fail(FE_EINVAL, "fe_set_atoms: widths must be positive");
  FE_TRY(fe_activate(m));
  delete[] m->h_atoms;
  m->h_atoms = new (std::nothrow) double[4 * (size_t)(n > 0 ? n : 1)];
  if (!m->h_atoms) return fe_fail(FE_ENOMEM, "host allocation failed");
  for (int a = 0; a < n; ++a) {
    for (int k = 0; k < 3; ++k) m->h_atoms[4 * a + k] = R[3 * a + k];
    m->h_atoms[4 * a + 3] = Z[a];
  }
  m->natoms = n;
  m->sigma_b = sigma_b;
  m->rc_loc = rc_loc;
  m->sigma_rho = sigma_rho;
  cudaFree(m->d_atoms);
  m->d_atoms = nullptr;
  if (n > 0) {
    FE_CUDA(cudaMalloc(&m->d_atoms, 4 * sizeof(double) * n));
    FE_CUDA(cudaMemcpy(m->d_atoms, m->h_atoms, 4 * sizeof(double) * n, cudaMemcpyHostToDevice));
  }
  return fe_fields_build(m);
}

KronGeom fe_geom(const fe_mesh* m, bool psi) {
  KronGeom g;
  g.p = m->p;
  g.NX = m->NX;
  g.NY = m->NY;
  g.nz = m->nz;
  g.gz_lo = psi ? m->gz_lo : 0;
  g.NZs = psi ? m->NZs : m->NZ;
  g.bx = g.by = g.zseg = g.nbx = g.nby = 0;   // chosen by the launcher
  return g;
}

extern "C" fe_status fe_set_kpoint(fe_mesh* m, double kx, double ky) {
  if (!m) return fe_fail(FE_EINVAL, "fe_set_kpoint: null mesh");
  if (!std::isfinite(kx) || !std::isfinite(ky))
    return fe_fail(FE_EINVAL, "fe_set_kpoint: k must be finite");
  m->kx = kx;
  m->ky = ky;
  m->has_k = kx != 0.0 || ky != 0.0;
  if (m->has_k) build_coef_bloch(m, &m->coefA);
  return FE_OK;
}

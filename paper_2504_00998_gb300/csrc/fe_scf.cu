// Self-consistent closure: the electron density of a block of orbitals, Fermi-Dirac
// occupations, and Anderson / Pulay density mixing.
//
// Density (Section 2.1, below Eq. Tsexc): rho = 2 sum_n f_n |psi_n|^2.  The library's
// blocks hold xt_n = M^1/2 u_n (Euclidean-orthonormal columns of Ht = M^-1/2 H M^-1/2,
// Section 2.3), so at psi node I, rho_I = sum_n occ_n xt_{I,n}^2 / M_II with occ_n = 2 f_n;
// the homogeneous-Dirichlet z planes carry no psi node and get rho = 0.
// Local-density exchange (Dirac, spin unpolarised; the optional exchange term of the
// self-consistent potential): e_x = -(3/4)(3/pi)^(1/3) rho^(4/3) per volume,
// v_x = -(3/pi)^(1/3) rho^(1/3), negative densities taken as zero.
// Occupations: Fermi-Dirac at smearing temperature kT, mu by bisection on
// 2 sum_n f_n = N_e.  Mixing: Anderson (J. ACM 12, 1965) / Pulay (Chem. Phys. Lett. 73,
// 1980) on the density with the lumped-mass inner product.
#include <cmath>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

// e_x at every phi node (for the lumped-mass sum) and veff += v_x at the psi nodes
__global__ void k_lda_exchange(const double* __restrict__ rho, double* __restrict__ ex,
                               double* __restrict__ veff, int64_t off, int64_t npsi,
                               int64_t nphi) {
  const double c = 0.98474502184269641;   // (3/pi)^(1/3)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nphi;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = rho[i] > 0.0 ? rho[i] : 0.0;
    const double cr = cbrt(r);
    ex[i] = -0.75 * c * r * cr;
    const int64_t j = i - off;
    if (veff && j >= 0 && j < npsi) veff[j] += -c * cr;
  }
}

// one warp per psi node: lanes stride over the vectors
// (cshift 1: complex orbitals as interleaved (re, im) lanes, lanes 2n and 2n+1 share occ_n)
template <typename T>
__global__ void k_density(const T* __restrict__ X, int64_t ld, int64_t nvec,
                          const double* __restrict__ occ, const double* __restrict__ mass,
                          int64_t off, int64_t npsi, double* __restrict__ rho, int cshift) {
  extern __shared__ double s_occ[];
  for (int64_t v = threadIdx.x; v < nvec; v += blockDim.x) s_occ[v] = occ[v >> cshift];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < npsi;
       i += warps) {
    const T* row = X + i * ld;
    double acc = 0.0;
    if constexpr (sizeof(T) == 4) {
      float a = 0.0f;   // a lane's few terms in float, the lane sum in double
      for (int64_t v = lane; v < nvec; v += 32) a += (float)s_occ[v] * row[v] * row[v];
      acc = (double)a;
    } else {
      for (int64_t v = lane; v < nvec; v += 32) acc += s_occ[v] * row[v] * row[v];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rho[off + i] = acc / mass[off + i];
  }
}

__global__ void k_mix_residual(const double* __restrict__ rin, const double* __restrict__ rout,
                               double* __restrict__ R, const double* __restrict__ prevR,
                               const double* __restrict__ prevRho, double* __restrict__ dR,
                               double* __restrict__ drho, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = rout[i] - rin[i];
    if (dR) {
      dR[i] = r - prevR[i];
      drho[i] = rin[i] - prevRho[i];
    }
    R[i] = r;
  }
}

constexpr int MIX_MAX = 16;
struct MixCoef {
  const double* drho[MIX_MAX];
  const double* dR[MIX_MAX];
  double gamma[MIX_MAX];
  int k;
  double alpha;
};

// rho_next = rho_in + alpha R - sum_i gamma_i (drho_i + alpha dR_i); keeps rho_in, R as the
// previous input and residual
__global__ void k_mix_update(double* __restrict__ rin, const double* __restrict__ R,
                             double* __restrict__ prevR, double* __restrict__ prevRho,
                             MixCoef c, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = rin[i], r = R[i];
    double v = x + c.alpha * r;
    for (int j = 0; j < c.k; ++j) v -= c.gamma[j] * (c.drho[j][i] + c.alpha * c.dR[j][i]);
    prevRho[i] = x;
    prevR[i] = r;
    rin[i] = v;
  }
}

// weighted dot products <u_j, w v> for several u_j at once, one partial per block and j
constexpr int WD_MAX = MIX_MAX + 1;
struct WdArgs {
  const double* u[WD_MAX];
  int nu;
};
__global__ void k_wdot_partial(WdArgs a, const double* __restrict__ v, const double* __restrict__ w,
                               int64_t n, double* __restrict__ part) {
  __shared__ double sh[fe::RED_THREADS];
  for (int j = 0; j < a.nu; ++j) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)fe::RED_THREADS + threadIdx.x; i < n;
         i += (int64_t)fe::RED_BLOCKS * fe::RED_THREADS)
      s += a.u[j][i] * w[i] * v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = fe::RED_THREADS / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)j * fe::RED_BLOCKS + blockIdx.x] = sh[0];
    __syncthreads();
  }
}
__global__ void k_wdot_final(const double* __restrict__ part, int nu, double* __restrict__ out) {
  __shared__ double sh[fe::RED_THREADS];
  for (int j = 0; j < nu; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < fe::RED_BLOCKS; b += fe::RED_THREADS)
      s += part[(int64_t)j * fe::RED_BLOCKS + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = fe::RED_THREADS / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sh[0];
    __syncthreads();
  }
}

// symmetric eigen-decomposition of a small matrix by cyclic Jacobi rotations (host)
void jacobi_eig(std::vector<double>& A, int k, std::vector<double>& V) {
  V.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
    if (off < 1e-300) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[(size_t)p * k + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < k; ++r) {
          const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
          A[(size_t)r * k + p] = c * arp - s * arq;
          A[(size_t)r * k + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {
          const double apr = A[(size_t)p * k + r], aqr = A[(size_t)q * k + r];
          A[(size_t)p * k + r] = c * apr - s * aqr;
          A[(size_t)q * k + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < k; ++r) {
          const double vrp = V[(size_t)r * k + p], vrq = V[(size_t)r * k + q];
          V[(size_t)r * k + p] = c * vrp - s * vrq;
          V[(size_t)r * k + q] = s * vrp + c * vrq;
        }
      }
  }
}

}  // namespace

extern "C" fe_status fe_density(fe_mesh* m, const void* X, int64_t nvec, int64_t ld,
                                const double* occ, double* rho, fe_precision prec) {
  if (!m || !X || !occ || !rho) return fe_fail(FE_EINVAL, "fe_density: null argument");
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_density: FE_F64 and FE_F32 blocks only");
  if (nvec < 1 || ld < nvec || nvec > 4096)
    return fe_fail(FE_EINVAL, "fe_density: need 1 <= nvec <= ld, nvec <= 4096");
  const int cshift = m->has_k ? 1 : 0;   // complex orbitals: |u|^2 = re^2 + im^2
  nvec <<= cshift;
  ld <<= cshift;
  FE_TRY(fe_activate(m));
  cudaStream_t st = m->stream;
  const int64_t plane = (int64_t)m->NX * m->NY;
  const int64_t off = (int64_t)m->gz_lo * plane;
  // planes without psi nodes (homogeneous Dirichlet faces) carry no density
  if (off > 0) FE_CUDA(cudaMemsetAsync(rho, 0, sizeof(double) * off, st));
  const int64_t tail = m->n_phi - off - m->n_psi;
  if (tail > 0) FE_CUDA(cudaMemsetAsync(rho + off + m->n_psi, 0, sizeof(double) * tail, st));
  const int threads = 256;
  int64_t blocks = (m->n_psi + (threads / 32) - 1) / (threads / 32);
  if (blocks > 152 * 64) blocks = 152 * 64;
  const size_t smem = sizeof(double) * (size_t)nvec;
  if (prec == FE_F64)
    k_density<double><<<(int)blocks, threads, smem, st>>>((const double*)X, ld, nvec, occ, m->d_mass,
                                                          off, m->n_psi, rho, cshift);
  else
    k_density<float><<<(int)blocks, threads, smem, st>>>((const float*)X, ld, nvec, occ, m->d_mass,
                                                         off, m->n_psi, rho, cshift);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

extern "C" fe_status fe_occupations(const double* eig, int n, double n_electrons, double kT,
                                    double* occ, double* mu_out) {
  if (!eig || !occ || n < 1) return fe_fail(FE_EINVAL, "fe_occupations: bad arguments");
  if (!(kT > 0.0)) return fe_fail(FE_EINVAL, "fe_occupations: need kT > 0");
  if (!(n_electrons >= 0.0 && n_electrons <= 2.0 * n))
    return fe_fail(FE_EINVAL, "fe_occupations: electron count outside [0, 2 n]");
  double emin = eig[0], emax = eig[0];
  for (int i = 1; i < n; ++i) { emin = std::fmin(emin, eig[i]); emax = std::fmax(emax, eig[i]); }
  double lo = emin - 50.0 * kT - 1.0, hi = emax + 50.0 * kT + 1.0;
  auto filled = [&](double mu) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += 1.0 - std::tanh(0.5 * (eig[i] - mu) / kT);
    return s;   // = 2 sum_i f_i
  };
  for (int it = 0; it < 200; ++it) {
    const double mu = 0.5 * (lo + hi);
    if (filled(mu) > n_electrons) hi = mu; else lo = mu;
  }
  const double mu = 0.5 * (lo + hi);
  for (int i = 0; i < n; ++i) occ[i] = 1.0 - std::tanh(0.5 * (eig[i] - mu) / kT);
  if (mu_out) *mu_out = mu;
  return FE_OK;
}

// ---- Anderson mixer ------------------------------------------------------------------------
struct fe_mixer {
  fe_mesh* mesh = nullptr;
  int64_t n = 0;
  int m = 0;
  double alpha = 0.3;
  double* buf = nullptr;      // R, prevR, prevRho, m x dR, m x drho, partials, dots
  int count = 0;              // differences stored
  int head = 0;               // ring slot of the next difference
  bool have_prev = false;
};

extern "C" fe_status fe_mixer_create(fe_mesh* m, int history, double alpha, fe_mixer** out) {
  if (!m || !out) return fe_fail(FE_EINVAL, "fe_mixer_create: null argument");
  *out = nullptr;
  if (history < 0 || history > MIX_MAX)
    return fe_fail(FE_EINVAL, "fe_mixer_create: history in [0, %d]", MIX_MAX);
  if (!(alpha > 0.0 && alpha <= 1.0)) return fe_fail(FE_EINVAL, "fe_mixer_create: alpha in (0, 1]");
  FE_TRY(fe_activate(m));
  fe_mixer* x = new fe_mixer;
  x->mesh = m;
  x->n = m->n_phi;
  x->m = history;
  x->alpha = alpha;
  const size_t vecs = 3 + 2 * (size_t)history;
  const size_t bytes = sizeof(double) * (vecs * (size_t)x->n + (size_t)WD_MAX * fe::RED_BLOCKS + 512);
  if (cudaMalloc(&x->buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return fe_fail(FE_ENOMEM, "fe_mixer_create: %zu bytes", bytes);
  }
  *out = x;
  return FE_OK;
}

extern "C" fe_status fe_mixer_destroy(fe_mixer* x) {
  if (!x) return FE_OK;
  fe_status st = FE_OK;
  if (cudaSetDevice(x->mesh->device) != cudaSuccess ||
      cudaStreamSynchronize(x->mesh->stream) != cudaSuccess || cudaFree(x->buf) != cudaSuccess) {
    cudaGetLastError();
    st = fe_fail(FE_ECUDA, "fe_mixer_destroy: could not release the history");
  }
  delete x;
  return st;
}

extern "C" fe_status fe_mixer_step(fe_mixer* x, double* rho_in, const double* rho_out,
                                   double* resid_norm) {
  if (!x || !rho_in || !rho_out) return fe_fail(FE_EINVAL, "fe_mixer_step: null argument");
  fe_mesh* m = x->mesh;
  FE_TRY(fe_activate(m));
  cudaStream_t st = m->stream;
  const int64_t n = x->n;
  double* R = x->buf;
  double* prevR = R + n;
  double* prevRho = prevR + n;
  double* dRs = prevRho + n;
  double* drhos = dRs + (size_t)x->m * n;
  double* part = drhos + (size_t)x->m * n;
  double* dots = part + (size_t)WD_MAX * fe::RED_BLOCKS;   // [32]: <dR_i, R>, <R, R>
  double* gram = dots + 32;                                 // row j: <dR_i, dR_j>, i <= j
  const int gb = fe::grid_for(n);
  // residual and, with history, the newest differences
  double* dR_new = nullptr;
  double* drho_new = nullptr;
  if (x->have_prev && x->m > 0) {
    dR_new = dRs + (size_t)x->head * n;
    drho_new = drhos + (size_t)x->head * n;
  }
  k_mix_residual<<<gb, 256, 0, st>>>(rho_in, rho_out, R, prevR, prevRho, dR_new, drho_new, n);
  fe_count_launch();
  if (dR_new) {
    x->head = (x->head + 1) % x->m;
    if (x->count < x->m) ++x->count;
  }
  x->have_prev = true;
  // the differences in order of age, oldest first
  const int k = x->count;
  std::vector<int> slot(k);
  for (int i = 0; i < k; ++i) slot[i] = ((x->head - k + i) % x->m + x->m) % x->m;
  // <dR_i, dR_j>, <dR_i, R>, <R, R> in the lumped-mass inner product
  std::vector<double> A((size_t)k * k), rhs(k);
  double rr = 0.0;
  {
    WdArgs a{};
    for (int i = 0; i < k; ++i) a.u[i] = dRs + (size_t)slot[i] * n;
    a.u[k] = R;
    a.nu = k + 1;
    k_wdot_partial<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(a, R, m->d_mass, n, part);
    fe_count_launch();
    k_wdot_final<<<1, fe::RED_THREADS, 0, st>>>(part, k + 1, dots);
    fe_count_launch();
    std::vector<double> h(k + 1);
    FE_CUDA(cudaMemcpyAsync(h.data(), dots, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
    for (int j = 0; j < k; ++j) {
      WdArgs b{};
      for (int i = 0; i <= j; ++i) b.u[i] = dRs + (size_t)slot[i] * n;
      b.nu = j + 1;
      k_wdot_partial<<<fe::RED_BLOCKS, fe::RED_THREADS, 0, st>>>(b, dRs + (size_t)slot[j] * n,
                                                                  m->d_mass, n, part);
      fe_count_launch();
      k_wdot_final<<<1, fe::RED_THREADS, 0, st>>>(part, j + 1, gram + (size_t)j * WD_MAX);
      fe_count_launch();
    }
    std::vector<double> g((size_t)k * WD_MAX);
    if (k) FE_CUDA(cudaMemcpyAsync(g.data(), gram, sizeof(double) * k * WD_MAX,
                                   cudaMemcpyDeviceToHost, st));
    FE_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) rhs[i] = h[i];
    rr = h[k];
    for (int j = 0; j < k; ++j)
      for (int i = 0; i <= j; ++i) A[(size_t)i * k + j] = A[(size_t)j * k + i] = g[(size_t)j * WD_MAX + i];
  }
  // gamma = A^+ rhs (minimum-norm least squares through the eigen-decomposition of A)
  MixCoef c{};
  c.k = k;
  c.alpha = x->alpha;
  if (k) {
    std::vector<double> E(A), V;
    jacobi_eig(E, k, V);
    double emax = 0.0;
    for (int i = 0; i < k; ++i) emax = std::fmax(emax, std::fabs(E[(size_t)i * k + i]));
    const double cut = emax * k * 2.220446049250313e-16;
    std::vector<double> gamma(k, 0.0);
    for (int e = 0; e < k; ++e) {
      const double lam = E[(size_t)e * k + e];
      if (std::fabs(lam) <= cut) continue;
      double proj = 0.0;
      for (int i = 0; i < k; ++i) proj += V[(size_t)i * k + e] * rhs[i];
      for (int i = 0; i < k; ++i) gamma[i] += V[(size_t)i * k + e] * proj / lam;
    }
    for (int i = 0; i < k; ++i) {
      c.gamma[i] = gamma[i];
      c.drho[i] = drhos + (size_t)slot[i] * n;
      c.dR[i] = dRs + (size_t)slot[i] * n;
    }
  }
  k_mix_update<<<gb, 256, 0, st>>>(rho_in, R, prevR, prevRho, c, n);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  if (resid_norm) *resid_norm = std::sqrt(std::fmax(rr, 0.0));
  return FE_OK;
}

extern "C" fe_status fe_lda_exchange(fe_mesh* m, const double* rho, double* veff,
                                     double* ex_host) {
  if (!m || !rho) return fe_fail(FE_EINVAL, "fe_lda_exchange: null argument");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_phi;
  void* wsp = nullptr;
  FE_TRY(fe_ws(m, WS_XC, sizeof(double) * ((size_t)n + fe::RED_BLOCKS + 8), &wsp));
  double* ex = static_cast<double*>(wsp);
  double* part = ex + n;
  double* out = part + fe::RED_BLOCKS;
  const int64_t off = (int64_t)m->gz_lo * m->NX * m->NY;
  k_lda_exchange<<<fe::grid_for(n), 256, 0, m->stream>>>(rho, ex, veff, off, m->n_psi, n);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  if (ex_host) {
    FE_TRY(fe::dot_async(m->d_mass, ex, n, 1, part, out, m->stream));
    FE_CUDA(cudaMemcpyAsync(ex_host, out, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
  }
  return FE_OK;
}

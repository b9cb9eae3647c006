// Hamiltonian application, the fused Chebyshev filter, the Poisson operator and the
// Lanczos spectral bounds.
//
// Eq. Veff and Hloc with Section 2.3: Ht = 1/2 M^-1/2 K M^-1/2 + diag(V_eff) on psi nodes.
// Chebyshev filter: scaled three-term recurrence of Zhou & Saad (J. Comput. Phys. 2006):
//   Y_1 = (s_1/e)(Ht - c) X,  Y_{k+1} = (2 s_{k+1}/e)(Ht - c) Y_k - s_k s_{k+1} Y_{k-1},
//   s_1 = e/(a0 - c), s_{k+1} = 1/(2/s_1 - s_k); each step is one fused operator launch that
//   reads Y_k and Y_{k-1} and overwrites Y_{k-1} in place.
// Lanczos bounds: Zhou & Li (2011), upper bound = largest Ritz value + ||f_k||.
#include <cmath>
#include <cstdint>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

namespace {

fe_status check_block(const fe_mesh* m, const void* X, int64_t nvec, int64_t ld, int elem,
                      const char* what) {
  if (!m) return fe_fail(FE_EINVAL, "%s: null mesh", what);
  if (!X) return fe_fail(FE_EINVAL, "%s: null block", what);
  if (nvec < 1 || ld < nvec) return fe_fail(FE_EINVAL, "%s: need 1 <= nvec <= ld", what);
  if (((uintptr_t)X) % 16 != 0) return fe_fail(FE_EINVAL, "%s: block not 16-byte aligned", what);
  if ((ld * elem) % 16 != 0)
    return fe_fail(FE_EINVAL, "%s: ld * element size must be a multiple of 16 bytes", what);
  return FE_OK;
}

int elem_bytes(fe_precision p) { return p == FE_F64 ? 8 : 4; }

bool valid_prec(fe_precision p) {
  return p == FE_F64 || p == FE_F32 || p == FE_BF16_F32ACC || p == FE_F32_F32ACC;
}

}  // namespace

// Tensor-core variants: the dense cell-matrix product (bf16, fe_tc.cu) and the
// FP32-accurate sum-factorised operator with split-TF32 in-plane contractions
// (fe_kron_tc.cu).
fe_status fe_tc_apply(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec,
                      int64_t ld, float alpha, float beta, float shift, fe_precision prec);
fe_status fe_ktc_apply(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec,
                       int64_t ld, float alpha, float beta, float shift);

// Y = alpha (Ht - shift) X + beta Z in the requested arithmetic.
// (plus alpha Ht_nloc X when the mesh carries the nonlocal term)
// With a Bloch wave vector (Section 2.1, H^k_loc), Ht_k = Ht_0 + |k|^2 / 2 - i A on complex
// blocks stored as interleaved (re, im) lanes; nvec and ld count real lanes here.  The first
// launch applies Ht_0 + |k|^2 / 2 to every lane with the Chebyshev combination, the second
// accumulates alpha (-i A X) into Y (A = M^-1/2 (kx Gx + ky Gy) M^-1/2, real antisymmetric).
fe_status fe_hx_step(fe_mesh* m, const void* X, void* Y, const void* Z, int64_t nvec, int64_t ld,
                     double alpha, double beta, double shift, fe_precision prec) {
  if (m->has_k) {
    if (prec != FE_F64 && prec != FE_F32)
      return fe_fail(FE_EUNSUPPORTED, "Bloch operator: FE_F64 and FE_F32 only");
    if (m->nl.natoms > 0)
      return fe_fail(FE_EUNSUPPORTED, "Bloch operator: the nonlocal term is Gamma-point only");
    const double sh = shift - 0.5 * (m->kx * m->kx + m->ky * m->ky);
    const KronGeom g = fe_geom(m, true);
    if (prec == FE_F64) {
      KronIO<double> io{(const double*)X, ld, (double*)Y, ld, (const double*)Z, ld, m->d_veff,
                        nvec, alpha, beta, sh};
      FE_TRY(fe::kron_f64(m->coefH, g, io, m->stream));
      KronIO<double> ia{(const double*)X, ld, (double*)Y, ld, (const double*)Y, ld, nullptr,
                        nvec, alpha, 1.0, 0.0};
      FE_TRY(fe::kron_f64(m->coefA, g, ia, m->stream));
    } else {
      KronIO<float> io{(const float*)X, ld, (float*)Y, ld, (const float*)Z, ld, m->d_veff_f,
                       nvec, (float)alpha, (float)beta, (float)sh};
      FE_TRY(fe::kron_f32(m->coefH, g, io, m->stream));
      KronIO<float> ia{(const float*)X, ld, (float*)Y, ld, (const float*)Y, ld, nullptr, nvec,
                       (float)alpha, 1.0f, 0.0f};
      FE_TRY(fe::kron_f32(m->coefA, g, ia, m->stream));
    }
    // the real symmetric quadrature potential acts on the (re, im) lanes alike
    return fe_quad_apply(m, X, Y, nvec, ld, alpha, prec == FE_F64);
  }
  if (prec == FE_F64) {
    KronIO<double> io{(const double*)X, ld, (double*)Y, ld, (const double*)Z, ld, m->d_veff,
                      nvec, alpha, beta, shift};
    FE_TRY(fe::kron_f64(m->coefH, fe_geom(m, true), io, m->stream));
  } else if (prec == FE_F32) {
    KronIO<float> io{(const float*)X, ld, (float*)Y, ld, (const float*)Z, ld, m->d_veff_f,
                     nvec, (float)alpha, (float)beta, (float)shift};
    FE_TRY(fe::kron_f32(m->coefH, fe_geom(m, true), io, m->stream));
  } else if (prec == FE_F32_F32ACC) {
    FE_TRY(fe_ktc_apply(m, (const float*)X, (float*)Y, (const float*)Z, nvec, ld, (float)alpha,
                        (float)beta, (float)shift));
  } else {
    FE_TRY(fe_tc_apply(m, (const float*)X, (float*)Y, (const float*)Z, nvec, ld, (float)alpha,
                       (float)beta, (float)shift, prec));
  }
  FE_TRY(fe_quad_apply(m, X, Y, nvec, ld, alpha, prec == FE_F64));
  return fe_nonlocal_apply(m, X, Y, nvec, ld, alpha, prec == FE_F64);
}

extern "C" fe_status fe_apply_H(fe_mesh* m, const void* X, void* Y, int64_t nvec, int64_t ld,
                                fe_precision prec) {
  if (!valid_prec(prec)) return fe_fail(FE_EINVAL, "fe_apply_H: bad precision");
  if (m && m->has_k) { nvec *= 2; ld *= 2; }   // complex entries -> (re, im) lanes
  FE_TRY(check_block(m, X, nvec, ld, elem_bytes(prec), "fe_apply_H"));
  FE_TRY(check_block(m, Y, nvec, ld, elem_bytes(prec), "fe_apply_H"));
  if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_apply_H: call fe_set_potential first");
  size_t bytes = (size_t)m->n_psi * ld * elem_bytes(prec);
  const char *xs = (const char*)X, *ys = (const char*)Y;
  if (xs < ys + bytes && ys < xs + bytes) return fe_fail(FE_EINVAL, "fe_apply_H: X and Y overlap");
  FE_TRY(fe_activate(m));
  return fe_hx_step(m, X, Y, nullptr, nvec, ld, 1.0, 0.0, 0.0, prec);
}

extern "C" fe_status fe_cheb_filter(fe_mesh* m, void* X, int64_t nvec, int64_t ld, int degree,
                                    double a, double b, double a0, fe_precision prec) {
  if (!valid_prec(prec)) return fe_fail(FE_EINVAL, "fe_cheb_filter: bad precision");
  if (m && m->has_k) { nvec *= 2; ld *= 2; }   // complex entries -> (re, im) lanes
  FE_TRY(check_block(m, X, nvec, ld, elem_bytes(prec), "fe_cheb_filter"));
  if (degree < 1) return fe_fail(FE_EINVAL, "fe_cheb_filter: degree must be >= 1");
  if (!(a0 < a && a < b) || !std::isfinite(a0) || !std::isfinite(b))
    return fe_fail(FE_EINVAL, "fe_cheb_filter: need a0 < a < b");
  if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_cheb_filter: call fe_set_potential first");
  FE_TRY(fe_activate(m));
  const int eb = elem_bytes(prec);
  size_t bytes = (size_t)m->n_psi * ld * eb;
  void* W;
  FE_TRY(fe_ws(m, WS_CHEB, bytes, &W));
  const double e = (b - a) / 2.0, c = (b + a) / 2.0;
  double sigma = e / (a0 - c);
  const double tau = 2.0 / sigma;
  // Y1 = (s1/e)(H - c) X  -> W
  FE_TRY(fe_hx_step(m, X, W, nullptr, nvec, ld, sigma / e, 0.0, c, prec));
  void* cur = W;   // Y_k
  void* prev = X;  // Y_{k-1}
  for (int i = 2; i <= degree; ++i) {
    double sn = 1.0 / (tau - sigma);
    // Y_{k+1} overwrites Y_{k-1}
    FE_TRY(fe_hx_step(m, cur, prev, prev, nvec, ld, 2.0 * sn / e, -sigma * sn, c, prec));
    void* t = cur;
    cur = prev;
    prev = t;
    sigma = sn;
  }
  if (cur != X) {
    FE_CUDA(cudaMemcpy2DAsync(X, ld * eb, cur, ld * eb, nvec * eb, m->n_psi,
                              cudaMemcpyDeviceToDevice, m->stream));
  }
  return FE_OK;
}

extern "C" fe_status fe_poisson_apply_K(fe_mesh* m, const double* x, double* y) {
  if (!m || !x || !y) return fe_fail(FE_EINVAL, "fe_poisson_apply_K: null argument");
  if (((uintptr_t)x) % 8 || ((uintptr_t)y) % 8)
    return fe_fail(FE_EINVAL, "fe_poisson_apply_K: arrays must be 8-byte aligned");
  if (x == y) return fe_fail(FE_EINVAL, "fe_poisson_apply_K: x and y must differ");
  FE_TRY(fe_activate(m));
  KronIO<double> io{x, 1, y, 1, nullptr, 1, nullptr, 1, 1.0, 0.0, 0.0};
  return fe::kron_k1(m->coefK, fe_geom(m, false), io, m->stream);
}

extern "C" fe_status fe_poisson_apply_K_f32(fe_mesh* m, const float* x, float* y) {
  if (!m || !x || !y) return fe_fail(FE_EINVAL, "fe_poisson_apply_K_f32: null argument");
  if (((uintptr_t)x) % 4 || ((uintptr_t)y) % 4)
    return fe_fail(FE_EINVAL, "fe_poisson_apply_K_f32: arrays must be 4-byte aligned");
  if (x == y) return fe_fail(FE_EINVAL, "fe_poisson_apply_K_f32: x and y must differ");
  FE_TRY(fe_activate(m));
  return fe_kcell_apply_f32(m, x, y);
}

// ---- Lanczos ---------------------------------------------------------------------------------
namespace {

__global__ void k_lz_init(const double* __restrict__ v0, double* __restrict__ v,
                          double* __restrict__ f, const double* __restrict__ nrm2, int64_t n) {
  double s = 1.0 / sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v[2 * i] = v0[i] * s;
    v[2 * i + 1] = 0.0;
    f[2 * i] = 0.0;
    f[2 * i + 1] = 0.0;
  }
}

// f -= s u with the scalar s read on the device
// (inc 2: the first lane of each node; inc 1: both lanes, the real form of a complex vector)
__global__ void k_lz_axpy(double* __restrict__ f, const double* __restrict__ u,
                          const double* __restrict__ s, int64_t n, int inc) {
  double a = *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    f[inc * i] -= a * u[inc * i];
}

__global__ void k_sqrt(double* x) { *x = sqrt(*x); }

// vold <- v, v <- f / beta
__global__ void k_lz_shift(const double* __restrict__ f, double* __restrict__ v,
                           double* __restrict__ vold, const double* __restrict__ beta, int64_t n,
                           int inc) {
  // (an exactly invariant Krylov space, beta = 0, leaves v = 0; the host reports it)
  const double b = *beta;
  const double s = b > 0.0 ? 1.0 / b : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    vold[inc * i] = v[inc * i];
    v[inc * i] = f[inc * i] * s;
  }
}

// number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm count)
int sturm(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    double off = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) ++cnt;
  }
  return cnt;
}

double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, int idx) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < d.size(); ++i) {
    double r = (i ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? std::fabs(e[i]) : 0.0);
    lo = std::fmin(lo, d[i] - r);
    hi = std::fmax(hi, d[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm(d, e, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" fe_status fe_lanczos_bounds(fe_mesh* m, const double* v0, int steps, double* lo,
                                       double* hi) {
  if (!m || !v0 || !lo || !hi) return fe_fail(FE_EINVAL, "fe_lanczos_bounds: null argument");
  if (steps < 2 || steps > 1000) return fe_fail(FE_EINVAL, "fe_lanczos_bounds: steps in [2, 1000]");
  if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_lanczos_bounds: call fe_set_potential first");
  FE_TRY(fe_activate(m));
  const int64_t n = m->n_psi;
  void* wsp;
  size_t vec_bytes = (size_t)n * 2 * sizeof(double);
  FE_TRY(fe_ws(m, WS_LANCZOS, 3 * vec_bytes + sizeof(double) * (2 * steps + 8 + fe::RED_BLOCKS),
               &wsp));
  double* v = (double*)wsp;
  double* vold = v + 2 * n;
  double* f = vold + 2 * n;
  double* scal = f + 2 * n;  // alpha[steps], beta[steps], tmp
  double* alpha = scal;
  double* beta = scal + steps;
  double* tmp = scal + 2 * steps;
  double* part = tmp + 8;
  cudaStream_t st = m->stream;
  const int gb = fe::grid_for(n);
  FE_TRY(fe::dot_async(v0, v0, n, 1, part, tmp, st));
  k_lz_init<<<gb, 256, 0, st>>>(v0, v, f, tmp, n); fe_count_launch();
  FE_CUDA(cudaMemsetAsync(vold, 0, vec_bytes, st));
  // with a Bloch wave vector the iteration runs on the real form of one complex vector (both
  // lanes of every node): [[Ht_0 + |k|^2/2, A], [-A, Ht_0 + |k|^2/2]] is symmetric (A is
  // antisymmetric) and has the spectrum of Ht_k
  const int lanes = m->has_k ? 2 : 1;
  const int inc = 2 / lanes;
  const int64_t nl = n * lanes;
  for (int j = 0; j < steps; ++j) {
    // f = Ht v - beta_{j-1} v_old; alpha_j = f . v; f -= alpha_j v
    FE_TRY(fe_hx_step(m, v, f, nullptr, lanes, 2, 1.0, 0.0, 0.0, FE_F64));
    if (j) { k_lz_axpy<<<gb, 256, 0, st>>>(f, vold, beta + j - 1, nl, inc); fe_count_launch(); }
    FE_TRY(fe::dot_async(f, v, nl, inc, part, alpha + j, st));
    k_lz_axpy<<<gb, 256, 0, st>>>(f, v, alpha + j, nl, inc); fe_count_launch();
    FE_TRY(fe::dot_async(f, f, nl, inc, part, beta + j, st));
    k_sqrt<<<1, 1, 0, st>>>(beta + j); fe_count_launch();
    if (j + 1 < steps) {
      k_lz_shift<<<gb, 256, 0, st>>>(f, v, vold, beta + j, nl, inc); fe_count_launch();
    }
  }
  FE_CUDA(cudaGetLastError());
  std::vector<double> hs(2 * steps);
  FE_CUDA(cudaMemcpyAsync(hs.data(), scal, sizeof(double) * 2 * steps, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  std::vector<double> d(hs.begin(), hs.begin() + steps);
  std::vector<double> e(hs.begin() + steps, hs.begin() + 2 * steps - 1);
  double fnorm = hs[2 * steps - 1];
  for (double x : hs)
    if (!std::isfinite(x))
      return fe_fail(FE_EINVAL, "fe_lanczos_bounds: the start vector is zero or not finite");
  // Breakdown: beta_j ~ 0 before the last step means that v0 lies in an invariant subspace
  // of Ht; the Krylov space then never sees the rest of the spectrum, so theta_max + |f| is
  // no bound of it
  // (j + 1 steps spanning the whole space of nl unknowns is the one exact exception: the
  // tridiagonal matrix then holds the whole spectrum)
  double scale = 0.0;
  for (int j = 0; j + 1 < steps; ++j) {
    scale = std::fmax(scale, std::fabs(d[j]));
    if (j) scale = std::fmax(scale, e[j - 1]);
    if (e[j] > 1e-10 * scale) continue;
    if (j + 1 >= nl) {
      d.resize(j + 1);
      e.resize(j);
      fnorm = 0.0;
      break;
    }
    return fe_fail(FE_EBREAKDOWN, "fe_lanczos_bounds: breakdown at step %d (the start "
                   "vector lies in an invariant subspace of Ht); use a start vector with "
                   "components along the whole spectrum, e.g. a random one", j + 1);
  }
  *lo = tridiag_eig(d, e, 0);
  *hi = tridiag_eig(d, e, (int)d.size() - 1) + fnorm;
  return FE_OK;
}

// Orthonormalisation and Rayleigh-Ritz in double precision.
//
// The Kohn-Sham problem needs the lowest N eigenpairs of H u = eps M u under the
// orthonormality constraint <psi_i|psi_j> = delta_ij (Section 2.1).  In the symmetric form
// used here the constraint is the Euclidean one on X.  Steps:
//   1. S = X^T X, column scaling D = diag(S)^1/2, Cholesky of D^-1 S D^-1; if it fails the
//      shifted Cholesky-QR3 shift s = 11 (N n + n (n+1)) u n is added (Fukaya, Kannan,
//      Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020); X <- X D^-1 R^-1.
//   2. One more Cholesky-QR pass (Cholesky-QR2), or two after a shifted pass.
//   3. Hs = X^T (Ht X), symmetrised; Hs = Q diag(eps) Q^T (dense symmetric eigensolver);
//      X <- X Q.
// The wavefunction block is node-major with the vectors contiguous; in column-major BLAS
// terms it is A = X^T (nvec x N, lda = ld).  Gram matrices and products are plain cuBLAS
// double GEMMs, the n x n factorisations are cuSOLVER calls.
#include <cmath>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

fe_status fe_hx_step(fe_mesh* m, const void* X, void* Y, const void* Z, int64_t nvec, int64_t ld,
                     double alpha, double beta, double shift, fe_precision prec);

namespace {

__global__ void k_f2d(const float* __restrict__ a, int64_t lda, double* __restrict__ b,
                      int64_t ldb, int64_t nvec, int64_t n) {
  int64_t tot = n * nvec;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / nvec, c = i % nvec;
    b[r * ldb + c] = (double)a[r * lda + c];
  }
}

__global__ void k_d2f2(const double* __restrict__ a, int64_t lda, float* __restrict__ b,
                       int64_t ldb, int64_t nvec, int64_t n) {
  int64_t tot = n * nvec;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / nvec, c = i % nvec;
    b[r * ldb + c] = (float)a[r * lda + c];
  }
}

// d[j] = 1/sqrt(S[j][j]); S <- D S D; optional diagonal shift
__global__ void k_scale_gram(double* __restrict__ S, int n, double* __restrict__ d, double shift) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) d[j] = 1.0 / sqrt(S[(int64_t)j * n + j]);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < (int64_t)n * n; i += blockDim.x) {
    int r = (int)(i % n), c = (int)(i / n);
    S[i] *= d[r] * d[c];
    if (r == c) S[i] += shift;
  }
}

__global__ void k_scale_cols(double* __restrict__ X, int64_t ld, int64_t nvec, int64_t n,
                             const double* __restrict__ d) {
  int64_t tot = n * nvec;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / nvec, c = i % nvec;
    X[r * ld + c] *= d[c];
  }
}

__global__ void k_symmetrize(double* __restrict__ S, int n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(i % n), c = (int)(i / n);
    if (r < c) {
      double v = 0.5 * (S[(int64_t)c * n + r] + S[(int64_t)r * n + c]);
      S[(int64_t)c * n + r] = v;
      S[(int64_t)r * n + c] = v;
    }
  }
}

struct RrWs {
  double *S, *Q, *d, *eig, *work;
  int* info;
  int lwork;
};

fe_status gram(fe_mesh* m, const double* A, int64_t lda, const double* B, int64_t ldb,
               int64_t nvec, double* S) {
  const double one = 1.0, zero = 0.0;
  // S = A B^T with A, B = nvec x N column-major
  FE_CUBLAS(cublasDgemm(m->cublas, CUBLAS_OP_N, CUBLAS_OP_T, (int)nvec, (int)nvec,
                        (int)m->n_psi, &one, A, (int)lda, B, (int)ldb, &zero, S, (int)nvec));
  return FE_OK;
}

// one (optionally shifted) scaled Cholesky-QR pass on the double block; *broke = 1 if the
// Cholesky factorisation failed
fe_status cholqr_pass(fe_mesh* m, double* X, int64_t ld, int64_t nvec, RrWs& w, double shift,
                      int* broke) {
  const int n = (int)nvec;
  FE_TRY(gram(m, X, ld, X, ld, nvec, w.S));
  k_scale_gram<<<1, 256, 0, m->stream>>>(w.S, n, w.d, shift); fe_count_launch();
  k_scale_cols<<<fe::grid_for(m->n_psi * nvec), 256, 0, m->stream>>>(X, ld, nvec, m->n_psi, w.d); fe_count_launch();
  FE_CUSOLVER(cusolverDnDpotrf(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, w.S, n, w.work, w.lwork,
                               w.info));
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  if (hinfo != 0) { *broke = 1; return FE_OK; }
  *broke = 0;
  const double one = 1.0;
  // A <- R^-T A  (X <- X R^-1)
  FE_CUBLAS(cublasDtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                        CUBLAS_DIAG_NON_UNIT, n, (int)m->n_psi, &one, w.S, n, X, (int)ld));
  return FE_OK;
}

}  // namespace

// Orthonormalise and Rayleigh-Ritz the double block X64 [n_psi][ld64] in place.
fe_status fe_rr_f64(fe_mesh* m, double* X, int64_t nvec, int64_t ld, double* eig) {
  const int n = (int)nvec;
  cudaStream_t st = m->stream;
  // small workspace
  int lw_potrf = 0, lw_syevd = 0;
  void* wsp;
  FE_TRY(fe_ws(m, WS_RR_SMALL, sizeof(double) * ((size_t)2 * n * n + 2 * n) + 64, &wsp));
  RrWs w;
  w.S = (double*)wsp;
  w.Q = w.S + (size_t)n * n;
  w.d = w.Q + (size_t)n * n;
  w.eig = w.d + n;
  FE_CUSOLVER(cusolverDnDpotrf_bufferSize(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, w.S, n, &lw_potrf));
  FE_CUSOLVER(cusolverDnDsyevd_bufferSize(m->cusolver, CUSOLVER_EIG_MODE_VECTOR,
                                          CUBLAS_FILL_MODE_UPPER, n, w.Q, n, w.eig, &lw_syevd));
  w.lwork = lw_potrf > lw_syevd ? lw_potrf : lw_syevd;
  void* wk;
  FE_TRY(fe_ws(m, WS_TC, sizeof(double) * ((size_t)w.lwork + 8), &wk));
  w.work = (double*)wk;
  w.info = (int*)(w.work + w.lwork);

  // Cholesky-QR2, or shifted Cholesky-QR3 when the first factorisation breaks down
  int broke = 0;
  FE_TRY(cholqr_pass(m, X, ld, nvec, w, 0.0, &broke));
  int extra = 1;
  if (broke) {
    const double u = 1.1102230246251565e-16;
    double s = 11.0 * ((double)m->n_psi * n + (double)n * (n + 1)) * u * n;
    FE_TRY(cholqr_pass(m, X, ld, nvec, w, s, &broke));
    if (broke) return fe_fail(FE_EBREAKDOWN, "shifted Cholesky-QR failed: block rank deficient");
    extra = 2;
  }
  for (int i = 0; i < extra; ++i) {
    FE_TRY(cholqr_pass(m, X, ld, nvec, w, 0.0, &broke));
    if (broke) return fe_fail(FE_EBREAKDOWN, "Cholesky-QR pass failed after orthonormalisation");
  }
  // Rayleigh-Ritz
  void* hxp;
  FE_TRY(fe_ws(m, WS_RR_HX, sizeof(double) * (size_t)m->n_psi * ld, &hxp));
  double* HX = (double*)hxp;
  FE_TRY(fe_hx_step(m, X, HX, nullptr, nvec, ld, 1.0, 0.0, 0.0, FE_F64));
  FE_TRY(gram(m, X, ld, HX, ld, nvec, w.Q));
  k_symmetrize<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.Q, n); fe_count_launch();
  FE_CUSOLVER(cusolverDnDsyevd(m->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n,
                               w.Q, n, w.eig, w.work, w.lwork, w.info));
  // X <- X Q:  A_new = Q^T A, into HX then copy back
  const double one = 1.0, zero = 0.0;
  FE_CUBLAS(cublasDgemm(m->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, (int)m->n_psi, n, &one, w.Q, n,
                        X, (int)ld, &zero, HX, (int)ld));
  FE_CUDA(cudaMemcpy2DAsync(X, ld * 8, HX, ld * 8, nvec * 8, m->n_psi, cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(eig, w.eig, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) return fe_fail(FE_ECUDA, "syevd info %d", hinfo);
  return FE_OK;
}

extern "C" fe_status fe_rayleigh_ritz(fe_mesh* m, void* X, int64_t nvec, int64_t ld, double* eig,
                                      fe_precision prec) {
  if (!m || !X || !eig) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: null argument");
  if (nvec < 1 || ld < nvec || nvec > 16384)
    return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: need 1 <= nvec <= ld, nvec <= 16384");
  if (nvec > m->n_psi) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: nvec exceeds the node count");
  int eb = prec == FE_F64 ? 8 : 4;
  if (((uintptr_t)X) % 16 || (ld * eb) % 16)
    return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: block alignment");
  if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: call fe_set_potential first");
  FE_TRY(fe_activate(m));
  if (prec == FE_F64) return fe_rr_f64(m, (double*)X, nvec, ld, eig);
  // float storage: promote to a double workspace, work there, demote
  int64_t ld64 = (nvec + 1) / 2 * 2;
  void* xp;
  FE_TRY(fe_ws(m, WS_RR_X, sizeof(double) * (size_t)m->n_psi * ld64, &xp));
  double* X64 = (double*)xp;
  const int gb = fe::grid_for(m->n_psi * nvec);
  k_f2d<<<gb, 256, 0, m->stream>>>((const float*)X, ld, X64, ld64, nvec, m->n_psi); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  FE_TRY(fe_rr_f64(m, X64, nvec, ld64, eig));
  k_d2f2<<<gb, 256, 0, m->stream>>>(X64, ld64, (float*)X, ld, nvec, m->n_psi); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

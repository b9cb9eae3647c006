// Orthonormalisation and Rayleigh-Ritz in double precision.
//
// The Kohn-Sham problem needs the lowest N eigenpairs of H u = eps M u under the
// orthonormality constraint <psi_i|psi_j> = delta_ij (Section 2.1).  In the symmetric form
// used here the constraint is the Euclidean one on X.
//
// Default (Gram) path, five N n^2 double flops instead of thirteen:
//   S = X^T X (SYRK), Hs = X^T (Ht X) (GEMM), D = diag(S)^-1/2,
//   D S D = R^T R (Cholesky), G = R^-T D Hs D R^-1, G = Q diag(eps) Q^T,
//   X <- X C with C = D R^-1 Q (GEMM).
// X C is the Rayleigh-Ritz basis of span(X) with C^T S C = I: the same result as
// Cholesky-QR followed by Rayleigh-Ritz, with the orthonormalisation folded into the n x n
// problem.  Its orthogonality degrades like cond(D S D) u, so when the Cholesky fails or
// the factor's diagonal indicates cond(D S D) > 1e8 (1e4 with FP32-accurate products; cold
// starts from random blocks) the explicit path runs instead:
//   scaled Cholesky-QR2, or shifted Cholesky-QR3 when the first factorisation breaks down
//   (shift 11 (N n + n (n+1)) u n; Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM
//   J. Sci. Comput. 2020), then Hs = X^T (Ht X), eigh, X <- X Q.
// The block is node-major with the vectors contiguous; in column-major BLAS terms it is
// A = X^T (nvec x N, lda = ld).  The big products are plain cuBLAS double GEMM / SYRK
// calls, the n x n factorisations cuSOLVER calls.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fe_blas.cuh"
#include "fe_internal.h"

// the lower triangle of a SYRK result (upper stored) is filled in (defined below)
__global__ void k_fill_lower(double* __restrict__ S, int n);

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

// eigenpairs of the symmetric n x n matrix in w.Q (upper triangle): eigenvectors overwrite
// w.Q, ascending eigenvalues into w.eig, the solver's status into w.info (checked by the
// caller); divide-and-conquer or cyclic Jacobi (FE_OPT_RR_EIGEN)
fe_status sym_eig(fe_mesh* m, int n, RrWs& w) {
  if (m->rr_eigen == FE_RR_EIGEN_SYEVJ) {
    FE_CUSOLVER(cusolverDnDsyevj(m->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n,
                                 w.Q, n, w.eig, w.work, w.lwork, w.info, m->syevj_params));
  } else {
    FE_CUSOLVER(cusolverDnDsyevd(m->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n,
                                 w.Q, n, w.eig, w.work, w.lwork, w.info));
  }
  return FE_OK;
}

// one (optionally shifted) scaled Cholesky-QR pass on the double block; *broke = 1 if the
// Cholesky factorisation failed
fe_status cholqr_pass(fe_mesh* m, double* X, int64_t ld, int64_t nvec, RrWs& w, double shift,
                      int* broke) {
  const int n = (int)nvec;
  const double one_ = 1.0, zero_ = 0.0;
  FE_CUBLAS(cublasDsyrk(m->cublas, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, n, (int)m->n_psi, &one_,
                        X, (int)ld, &zero_, w.S, n));
  k_fill_lower<<<fe::grid_for((int64_t)n * n), 256, 0, m->stream>>>(w.S, n); fe_count_launch();
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

__global__ void k_scale_sym(double* __restrict__ A, int n, const double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(i % n), c = (int)(i / n);
    A[i] *= d[r] * d[c];
  }
}

// d[j] = 1 / sqrt(S_jj) (diagonal scaling of the Gram matrix)
__global__ void k_inv_sqrt_diag(const double* __restrict__ S, int n, double* __restrict__ d) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    d[j] = 1.0 / sqrt(S[(int64_t)j * n + j]);
}

__global__ void k_fill_lower(double* __restrict__ S, int n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(i % n), c = (int)(i / n);
    if (r > c) S[i] = S[(int64_t)r * n + c];
  }
}

__global__ void k_scale_rows(double* __restrict__ C, int n, const double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x)
    C[i] *= d[(int)(i % n)];
}

__global__ void k_diag(const double* __restrict__ R, int n, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    out[j] = R[(int64_t)j * n + j];
}

// n x n part of the Gram path.  On entry w.S holds X^T X (upper triangle at least) and w.Q
// holds X^T Ht X; on exit w.Q holds C = D R^-1 Q and eig the Ritz values, or *ill is set
// when the scaled Gram matrix is not safely positive definite (cond above cond_max).
fe_status rr_small(fe_mesh* m, int64_t nvec, RrWs& w, double* eig, bool* ill, double cond_max) {
  const int n = (int)nvec;
  cudaStream_t st = m->stream;
  const double one = 1.0;
  *ill = false;
  k_inv_sqrt_diag<<<(n + 255) / 256, 256, 0, st>>>(w.S, n, w.d); fe_count_launch();
  k_fill_lower<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.S, n); fe_count_launch();
  k_scale_sym<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.S, n, w.d); fe_count_launch();
  k_symmetrize<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.Q, n); fe_count_launch();
  k_scale_sym<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.Q, n, w.d); fe_count_launch();
  FE_CUSOLVER(cusolverDnDpotrf(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, w.S, n, w.work, w.lwork,
                               w.info));
  k_diag<<<(n + 255) / 256, 256, 0, st>>>(w.S, n, w.eig); fe_count_launch();
  std::vector<double> rdiag(n), dinv(n);
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaMemcpyAsync(rdiag.data(), w.eig, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaMemcpyAsync(dinv.data(), w.d, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  // a zero column (or a NaN / infinity in one) makes the block rank deficient whatever the
  // orthonormalisation: report it before any pass scales the block by 1 / |column|
  for (int j = 0; j < n; ++j)
    if (!std::isfinite(dinv[j]))
      return fe_fail(FE_EBREAKDOWN, "fe_rayleigh_ritz: column %d of the block is zero or not "
                     "finite (rank-deficient block)", j);
  if (hinfo != 0) { *ill = true; return FE_OK; }
  double rmax = 0.0, rmin = 1e300;
  for (int j = 0; j < n; ++j) {
    rmax = std::fmax(rmax, std::fabs(rdiag[j]));
    rmin = std::fmin(rmin, std::fabs(rdiag[j]));
  }
  if (!(rmin > 0.0) || (rmax / rmin) * (rmax / rmin) > cond_max) { *ill = true; return FE_OK; }
  // G = R^-T Hs R^-1
  FE_CUBLAS(cublasDtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, w.S, n, w.Q, n));
  FE_CUBLAS(cublasDtrsm(m->cublas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, w.S, n, w.Q, n));
  k_symmetrize<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.Q, n); fe_count_launch();
  FE_TRY(sym_eig(m, n, w));
  // C = D R^-1 Q
  FE_CUBLAS(cublasDtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, w.S, n, w.Q, n));
  k_scale_rows<<<fe::grid_for((int64_t)n * n), 256, 0, st>>>(w.Q, n, w.d); fe_count_launch();
  FE_CUDA(cudaMemcpyAsync(eig, w.eig, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(&hinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) return fe_fail(FE_ECUDA, "dense eigensolver info %d", hinfo);
  return FE_OK;
}

// Gram path with double products.  HX is the block Ht X (double, same layout); Xout <- X C.
fe_status rr_gram_path(fe_mesh* m, const double* X, int64_t ld, const double* HX, int64_t ldh,
                       int64_t nvec, RrWs& w, double* Xout, int64_t ldo, double* eig, bool* ill) {
  const int n = (int)nvec;
  const double one = 1.0, zero = 0.0;
  // S = A A^T (upper), Hs = A B^T
  FE_CUBLAS(cublasDsyrk(m->cublas, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, n, (int)m->n_psi, &one,
                        X, (int)ld, &zero, w.S, n));
  FE_TRY(gram(m, X, ld, HX, ldh, nvec, w.Q));
  FE_TRY(rr_small(m, nvec, w, eig, ill, kGramCondF64));
  if (*ill) return FE_OK;
  // Xout^T = C^T A
  FE_CUBLAS(cublasDgemm(m->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, (int)m->n_psi, n, &one, w.Q, n,
                        X, (int)ld, &zero, Xout, (int)ldo));
  return FE_OK;
}

__global__ void k_f2d_n(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void k_d2f_n(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Gram path for float storage with the three block products on the tensor cores in cuBLAS's
// FP32-accurate BF16x9 emulation; the n x n part stays in double.  X <- X C in place.
fe_status rr_gram_path_tc32(fe_mesh* m, float* X, int64_t ld, const float* HX, int64_t nvec,
                            RrWs& w, float* tmp, double* eig, bool* ill) {
  const int n = (int)nvec;
  const int N = (int)m->n_psi;
  const float one = 1.0f, zero = 0.0f;
  void* sp;
  FE_TRY(fe_ws(m, WS_RR_TC32, sizeof(float) * (size_t)2 * n * n + 64, &sp));
  float* Sf = (float*)sp;
  float* Hf = Sf + (size_t)n * n;
  const cublasComputeType_t ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  FiniteEmulationGuard finite(m->cublas);
  FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, X, CUDA_R_32F,
                         (int)ld, X, CUDA_R_32F, (int)ld, &zero, Sf, CUDA_R_32F, n, ct,
                         CUBLAS_GEMM_DEFAULT));
  FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, X, CUDA_R_32F,
                         (int)ld, HX, CUDA_R_32F, (int)ld, &zero, Hf, CUDA_R_32F, n, ct,
                         CUBLAS_GEMM_DEFAULT));
  const int64_t nn = (int64_t)n * n;
  k_f2d_n<<<fe::grid_for(nn), 256, 0, m->stream>>>(Sf, w.S, nn); fe_count_launch();
  k_f2d_n<<<fe::grid_for(nn), 256, 0, m->stream>>>(Hf, w.Q, nn); fe_count_launch();
  FE_TRY(rr_small(m, nvec, w, eig, ill, kGramCondTC32));
  if (*ill) return FE_OK;
  k_d2f_n<<<fe::grid_for(nn), 256, 0, m->stream>>>(w.Q, Sf, nn); fe_count_launch();
  // tmp^T = C^T A
  FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, N, n, &one, Sf, CUDA_R_32F, n,
                         X, CUDA_R_32F, (int)ld, &zero, tmp, CUDA_R_32F, (int)ld, ct,
                         CUBLAS_GEMM_DEFAULT));
  FE_CUDA(cudaMemcpy2DAsync(X, ld * 4, tmp, ld * 4, nvec * 4, m->n_psi, cudaMemcpyDeviceToDevice,
                            m->stream));
  return FE_OK;
}

fe_status rr_setup_small(fe_mesh* m, int n, RrWs& w) {
  int lw_potrf = 0, lw_syevd = 0, lw_syevj = 0;
  void* wsp;
  FE_TRY(fe_ws(m, WS_RR_SMALL, sizeof(double) * ((size_t)2 * n * n + 2 * n) + 64, &wsp));
  w.S = (double*)wsp;
  w.Q = w.S + (size_t)n * n;
  w.d = w.Q + (size_t)n * n;
  w.eig = w.d + n;
  FE_CUSOLVER(cusolverDnDpotrf_bufferSize(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, w.S, n, &lw_potrf));
  FE_CUSOLVER(cusolverDnDsyevd_bufferSize(m->cusolver, CUSOLVER_EIG_MODE_VECTOR,
                                          CUBLAS_FILL_MODE_UPPER, n, w.Q, n, w.eig, &lw_syevd));
  if (m->rr_eigen == FE_RR_EIGEN_SYEVJ) {
    if (!m->syevj_params) {
      FE_CUSOLVER(cusolverDnCreateSyevjInfo(&m->syevj_params));
      FE_CUSOLVER(cusolverDnXsyevjSetTolerance(m->syevj_params, 1e-14));
      FE_CUSOLVER(cusolverDnXsyevjSetMaxSweeps(m->syevj_params, 100));
    }
    FE_CUSOLVER(cusolverDnDsyevj_bufferSize(m->cusolver, CUSOLVER_EIG_MODE_VECTOR,
                                            CUBLAS_FILL_MODE_UPPER, n, w.Q, n, w.eig, &lw_syevj,
                                            m->syevj_params));
  }
  w.lwork = std::max(lw_potrf, std::max(lw_syevd, lw_syevj));
  void* wk;
  FE_TRY(fe_ws(m, WS_TC, sizeof(double) * ((size_t)w.lwork + 8), &wk));
  w.work = (double*)wk;
  w.info = (int*)(w.work + w.lwork);
  return FE_OK;
}

// Orthonormalise and Rayleigh-Ritz the double block X64 [n_psi][ld64] in place (explicit
// path: Cholesky-QR2 or shifted Cholesky-QR3, then Rayleigh-Ritz with an FP64 Ht X).
fe_status fe_rr_f64(fe_mesh* m, double* X, int64_t nvec, int64_t ld, double* eig) {
  const int n = (int)nvec;
  cudaStream_t st = m->stream;
  RrWs w;
  FE_TRY(rr_setup_small(m, n, w));

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
  FE_TRY(sym_eig(m, n, w));
  // X <- X Q:  A_new = Q^T A, into HX then copy back
  const double one = 1.0, zero = 0.0;
  FE_CUBLAS(cublasDgemm(m->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, (int)m->n_psi, n, &one, w.Q, n,
                        X, (int)ld, &zero, HX, (int)ld));
  FE_CUDA(cudaMemcpy2DAsync(X, ld * 8, HX, ld * 8, nvec * 8, m->n_psi, cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(eig, w.eig, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) return fe_fail(FE_ECUDA, "dense eigensolver info %d", hinfo);
  return FE_OK;
}

extern "C" fe_status fe_rayleigh_ritz(fe_mesh* m, void* X, int64_t nvec, int64_t ld, double* eig,
                                      fe_precision prec) {
  if (!m || !X || !eig) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: null argument");
  if (nvec < 1 || ld < nvec || nvec > 16384)
    return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: need 1 <= nvec <= ld, nvec <= 16384");
  if (nvec > m->n_psi) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: nvec exceeds the node count");
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_BF16_F32ACC && prec != FE_F32_F32ACC)
    return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: bad precision");
  if (m->has_k) {
    // complex block (interleaved re, im; nvec and ld count complex entries)
    const int ceb = prec == FE_F64 ? 16 : 8;
    if (((uintptr_t)X) % 16 || (ld * ceb) % 16)
      return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: block alignment");
    if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: call fe_set_potential first");
    FE_TRY(fe_activate(m));
    return fe_rr_complex(m, X, nvec, ld, eig, prec);
  }
  const int eb = prec == FE_F64 ? 8 : 4;
  if (((uintptr_t)X) % 16 || (ld * eb) % 16)
    return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: block alignment");
  if (!m->has_potential) return fe_fail(FE_EINVAL, "fe_rayleigh_ritz: call fe_set_potential first");
  FE_TRY(fe_activate(m));
  const int n = (int)nvec;
  const int64_t N = m->n_psi;
  RrWs w;
  FE_TRY(rr_setup_small(m, n, w));
  const int gb = fe::grid_for(N * nvec);
  const int64_t ld64 = (nvec + 1) / 2 * 2;
  void* hxp;
  FE_TRY(fe_ws(m, WS_RR_HX, sizeof(double) * (size_t)N * (prec == FE_F64 ? ld : ld64), &hxp));
  double* HX = (double*)hxp;
  bool ill = false;
  if (prec == FE_F64) {
    double* Xd = (double*)X;
    FE_TRY(fe_hx_step(m, Xd, HX, nullptr, nvec, ld, 1.0, 0.0, 0.0, FE_F64));
    void* tp;
    FE_TRY(fe_ws(m, WS_RR_X, sizeof(double) * (size_t)N * ld, &tp));
    FE_TRY(rr_gram_path(m, Xd, ld, HX, ld, nvec, w, (double*)tp, ld, eig, &ill));
    if (!ill) {
      FE_CUDA(cudaMemcpy2DAsync(Xd, ld * 8, tp, ld * 8, nvec * 8, N, cudaMemcpyDeviceToDevice,
                                m->stream));
      return FE_OK;
    }
    return fe_rr_f64(m, Xd, nvec, ld, eig);
  }
  if (m->rr_products == 1) {
    // block products on the tensor cores (FP32-accurate emulation), n x n part in double
    void* hp;
    FE_TRY(fe_ws(m, WS_RR_HX, sizeof(float) * (size_t)N * ld * 2, &hp));
    float* HXf = (float*)hp;
    float* tmp = HXf + (size_t)N * ld;
    FE_TRY(fe_hx_step(m, X, HXf, nullptr, nvec, ld, 1.0, 0.0, 0.0, FE_F32));
    FE_TRY(rr_gram_path_tc32(m, (float*)X, ld, HXf, nvec, w, tmp, eig, &ill));
    if (!ill) return FE_OK;
    FE_TRY(fe_ws(m, WS_RR_HX, sizeof(double) * (size_t)N * ld64, &hxp));
    HX = (double*)hxp;
  }
  // float storage: Ht X in float (sum-factorised), Gram, projection and rotation in double
  void* xp;
  const size_t half = sizeof(double) * (size_t)N * ld64;
  const size_t second = std::max(half, sizeof(float) * (size_t)N * ld);
  FE_TRY(fe_ws(m, WS_RR_X, half + second, &xp));
  double* X64 = (double*)xp;
  double* T64 = X64 + (size_t)N * ld64;
  float* HXf = (float*)T64;   // float Ht X staged in the second half before promotion
  FE_TRY(fe_hx_step(m, X, HXf, nullptr, nvec, ld, 1.0, 0.0, 0.0, FE_F32));
  k_f2d<<<gb, 256, 0, m->stream>>>(HXf, ld, HX, ld64, nvec, N); fe_count_launch();
  k_f2d<<<gb, 256, 0, m->stream>>>((const float*)X, ld, X64, ld64, nvec, N); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  FE_TRY(rr_gram_path(m, X64, ld64, HX, ld64, nvec, w, T64, ld64, eig, &ill));
  if (ill) {
    FE_TRY(fe_rr_f64(m, X64, nvec, ld64, eig));
    T64 = X64;
  }
  k_d2f2<<<gb, 256, 0, m->stream>>>(T64, ld64, (float*)X, ld, nvec, N); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// Rayleigh-Ritz of a complex (Bloch k-point) block, Section 2.1 with Bloch's theorem: the
// block X holds nvec complex vectors per psi node as interleaved (re, im) lanes (float or
// double); the subspace problem is Hermitian.
//
// In double complex arithmetic: with A the n x N column-major view of the block
// (A(i, I) = X[I][i]) and B that of Ht_k X, the products S = A A^H and T = A B^H are the
// complex conjugates of the Gram matrix X^H X and of X^H Ht_k X.  Conjugation keeps the
// (real) eigenvalues of the pencil and conjugates its eigenvectors y, so the rotated block
// is A <- y^H A.  The pencil is reduced by the Cholesky factor of the diagonally scaled S
// (D S D = U^H U), Hh = U^-H D T D U^-1, y = D U^-1 w for Hh w = lambda w.
#include <cmath>
#include <cuComplex.h>

#include "fe_blas.cuh"
#include "fe_internal.h"

fe_status fe_hx_step(fe_mesh* m, const void* X, void* Y, const void* Z, int64_t nvec, int64_t ld,
                     double alpha, double beta, double shift, fe_precision prec);

namespace {

template <typename T>
__global__ void k_to_z(const T* __restrict__ X, int64_t ld, int64_t n, int64_t N,
                       cuDoubleComplex* __restrict__ Z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i / n, j = i - I * n;
    Z[i] = make_cuDoubleComplex((double)X[I * 2 * ld + 2 * j], (double)X[I * 2 * ld + 2 * j + 1]);
  }
}

template <typename T>
__global__ void k_from_z(const cuDoubleComplex* __restrict__ Z, int64_t ld, int64_t n, int64_t N,
                         T* __restrict__ X) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = i / n, j = i - I * n;
    X[I * 2 * ld + 2 * j] = (T)cuCreal(Z[i]);
    X[I * 2 * ld + 2 * j + 1] = (T)cuCimag(Z[i]);
  }
}

// d_i = 1 / sqrt(S_ii)
__global__ void k_pencil_scale(const cuDoubleComplex* S, double* d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = 1.0 / sqrt(cuCreal(S[(int64_t)i * n + i]));
}

// S <- D S D, T <- D T D
__global__ void k_scale_pencil(cuDoubleComplex* S, cuDoubleComplex* T, const double* d, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double s = d[e % n] * d[e / n];
    S[e] = make_cuDoubleComplex(cuCreal(S[e]) * s, cuCimag(S[e]) * s);
    T[e] = make_cuDoubleComplex(cuCreal(T[e]) * s, cuCimag(T[e]) * s);
  }
}

// rows of the n x n column-major Y scaled by d (Y <- D Y)
__global__ void k_scale_rows(cuDoubleComplex* Y, const double* d, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double s = d[e % n];
    Y[e] = make_cuDoubleComplex(cuCreal(Y[e]) * s, cuCimag(Y[e]) * s);
  }
}

}  // namespace

fe_status fe_rr_complex(fe_mesh* m, void* X, int64_t nvec, int64_t ld, double* eig,
                        fe_precision prec) {
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_rayleigh_ritz: complex blocks in FE_F64 or FE_F32");
  const int n = (int)nvec;
  const int64_t N = m->n_psi;
  cudaStream_t st = m->stream;
  int lw_potrf = 0, lw_heevd = 0;
  // workspace: block, Ht_k block, rotated block (N n each); S, T (n n each); d, eig (n);
  // solver scratch; info
  const size_t zb = sizeof(cuDoubleComplex);
  void* wsp;
  const size_t big = (size_t)N * n, small = (size_t)n * n;
  FE_TRY(fe_ws(m, WS_KPT, zb * (3 * big + 2 * small) + sizeof(double) * 2 * n + 256, &wsp));
  cuDoubleComplex* Z = (cuDoubleComplex*)wsp;
  cuDoubleComplex* HZ = Z + big;
  cuDoubleComplex* R = HZ + big;
  cuDoubleComplex* S = R + big;
  cuDoubleComplex* T = S + small;
  double* d = (double*)(T + small);
  double* w = d + n;
  FE_CUSOLVER(cusolverDnZpotrf_bufferSize(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, S, n, &lw_potrf));
  FE_CUSOLVER(cusolverDnZheevd_bufferSize(m->cusolver, CUSOLVER_EIG_MODE_VECTOR,
                                          CUBLAS_FILL_MODE_UPPER, n, T, n, w, &lw_heevd));
  const int lwork = lw_potrf > lw_heevd ? lw_potrf : lw_heevd;
  void* wk;
  FE_TRY(fe_ws(m, WS_TC, zb * ((size_t)lwork + 4), &wk));
  cuDoubleComplex* work = (cuDoubleComplex*)wk;
  int* info = (int*)(work + lwork);

  const int gb = fe::grid_for((int64_t)big);
  if (prec == FE_F64)
    k_to_z<double><<<gb, 256, 0, st>>>((const double*)X, ld, n, N, Z);
  else
    k_to_z<float><<<gb, 256, 0, st>>>((const float*)X, ld, n, N, Z);
  fe_count_launch();
  // Ht_k Z (lanes: 2 n per node)
  FE_TRY(fe_hx_step(m, Z, HZ, nullptr, 2 * nvec, 2 * nvec, 1.0, 0.0, 0.0, FE_F64));
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  FE_CUBLAS(cublasZgemm(m->cublas, CUBLAS_OP_N, CUBLAS_OP_C, n, n, (int)N, &one, Z, n, Z, n,
                        &zero, S, n));
  FE_CUBLAS(cublasZgemm(m->cublas, CUBLAS_OP_N, CUBLAS_OP_C, n, n, (int)N, &one, Z, n, HZ, n,
                        &zero, T, n));
  const int gs = fe::grid_for((int64_t)small);
  k_pencil_scale<<<(n + 255) / 256, 256, 0, st>>>(S, d, n); fe_count_launch();
  k_scale_pencil<<<gs, 256, 0, st>>>(S, T, d, n); fe_count_launch();
  FE_CUSOLVER(cusolverDnZpotrf(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, S, n, work, lwork, info));
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0)
    return fe_fail(FE_EBREAKDOWN, "fe_rayleigh_ritz: complex block rank deficient (potrf %d)", hinfo);
  // Hh = U^-H T U^-1
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_C,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  FE_CUSOLVER(cusolverDnZheevd(m->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, T,
                               n, w, work, lwork, info));
  // y = D U^-1 w (in T), then the rotated block R = y^H Z
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  k_scale_rows<<<gs, 256, 0, st>>>(T, d, n); fe_count_launch();
  FE_CUBLAS(cublasZgemm(m->cublas, CUBLAS_OP_C, CUBLAS_OP_N, n, (int)N, n, &one, T, n, Z, n,
                        &zero, R, n));
  if (prec == FE_F64)
    k_from_z<double><<<gb, 256, 0, st>>>(R, ld, n, N, (double*)X);
  else
    k_from_z<float><<<gb, 256, 0, st>>>(R, ld, n, N, (float*)X);
  fe_count_launch();
  FE_CUDA(cudaMemcpyAsync(eig, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) return fe_fail(FE_ECUDA, "fe_rayleigh_ritz: heevd info %d", hinfo);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

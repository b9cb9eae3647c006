// Rayleigh-Ritz of a complex (Bloch k-point) block, Section 2.1 with Bloch's theorem: the
// block X holds nvec complex vectors per psi node as interleaved (re, im) lanes (float or
// double); the subspace problem is Hermitian.
//
// Float blocks with tensor-core products (the default for float storage): the block is read
// as its real N x 2n lane array R, and the three block products are real FP32-accurate BF16x9
// GEMMs of the same shape as at the Gamma point with 2n vectors:
//   G = R^T R and C = R^T (Ht_k R) hold every (re, im) x (re, im) product pair, so
//     (X^H X)_jk   = G(2j,2k) + G(2j+1,2k+1) + i (G(2j,2k+1) - G(2j+1,2k)),
//     (X^H Ht X)_jk = the same combination of C;
//   the pencil Tx y = lambda Sx y is reduced in double complex by the Cholesky factor of the
//   diagonally scaled Gram matrix (D Sx D = U^H U, Hh = U^-H D Tx D U^-1, y = D U^-1 w), and
//   X <- X Y is the real product R W with the 2n x 2n matrix W(2j,2k) = W(2j+1,2k+1) = Re Y_jk,
//   W(2j,2k+1) = Im Y_jk, W(2j+1,2k) = -Im Y_jk.
// When the scaled Gram matrix is not safely positive definite for FP32-accurate products (its
// factor's diagonal spread gives cond > 1e4) the block is handed, unchanged, to the double
// complex path below.
//
// Double complex path (double blocks, float blocks without tensor-core products, and the
// fallback): with A the n x N column-major view of the block (A(i, I) = X[I][i]) and B that of
// Ht_k X, the products S = A A^H and T = A B^H are the complex conjugates of the Gram matrix
// X^H X and of X^H Ht_k X.  Conjugation keeps the (real) eigenvalues of the pencil and
// conjugates its eigenvectors y, so the rotated block is A <- y^H A.  The pencil is reduced as
// above with S and T.
#include <cmath>
#include <vector>
#include <cuComplex.h>

#include "fe_blas.cuh"
#include "fe_internal.h"

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


// Hermitian part of the complex n x n matrix formed from the real 2n x 2n product P (column
// major, P(a, b) = sum_I R[I][a] Q[I][b]):  Z_jk = sum_I conj(x_Ij) q_Ik, Z <- (Z + Z^H) / 2
__global__ void k_lane_combine(const float* __restrict__ P, int n, cuDoubleComplex* __restrict__ Z) {
  const int64_t nr = 2 * (int64_t)n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e % n, k = e / n;
    auto at = [&](int64_t a, int64_t b) { return (double)P[b * nr + a]; };
    const double re_jk = at(2 * j, 2 * k) + at(2 * j + 1, 2 * k + 1);
    const double im_jk = at(2 * j, 2 * k + 1) - at(2 * j + 1, 2 * k);
    const double re_kj = at(2 * k, 2 * j) + at(2 * k + 1, 2 * j + 1);
    const double im_kj = at(2 * k, 2 * j + 1) - at(2 * k + 1, 2 * j);
    Z[e] = make_cuDoubleComplex(0.5 * (re_jk + re_kj), 0.5 * (im_jk - im_kj));
  }
}

// real diagonal of a complex n x n matrix
__global__ void k_zdiag(const cuDoubleComplex* __restrict__ U, int n, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    out[j] = cuCreal(U[(int64_t)j * n + j]);
}

// the real 2n x 2n form W of the complex rotation Y (column major, see above)
__global__ void k_rotation_lanes(const cuDoubleComplex* __restrict__ Y, int n, float* __restrict__ W) {
  const int64_t nr = 2 * (int64_t)n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e % n, k = e / n;
    const float yr = (float)cuCreal(Y[e]), yi = (float)cuCimag(Y[e]);
    W[(2 * k) * nr + 2 * j] = yr;
    W[(2 * k) * nr + 2 * j + 1] = -yi;
    W[(2 * k + 1) * nr + 2 * j] = yi;
    W[(2 * k + 1) * nr + 2 * j + 1] = yr;
  }
}

// Float block with tensor-core products; *ill when the scaled Gram matrix is too ill
// conditioned for the Gram path (X untouched then).
fe_status rr_complex_tc32(fe_mesh* m, float* X, int64_t nvec, int64_t ld, double* eig,
                          bool* ill) {
  *ill = false;
  const int n = (int)nvec, nr = 2 * n;
  const int64_t N = m->n_psi, ldr = 2 * ld;
  cudaStream_t st = m->stream;
  // Ht_k R and the rotated lanes (N x 2 ld floats each)
  void* hp;
  FE_TRY(fe_ws(m, WS_RR_HX, sizeof(float) * (size_t)N * ldr * 2, &hp));
  float* HR = (float*)hp;
  float* tmp = HR + (size_t)N * ldr;
  // the two real 2n x 2n products (the first reused for W)
  void* sp;
  FE_TRY(fe_ws(m, WS_RR_TC32, sizeof(float) * (size_t)2 * nr * nr + 64, &sp));
  float* Gf = (float*)sp;
  float* Cf = Gf + (size_t)nr * nr;
  // S, T (n x n complex), d, w, diag (n)
  const size_t small = (size_t)n * n;
  void* zp;
  FE_TRY(fe_ws(m, WS_KPT, sizeof(cuDoubleComplex) * 2 * small + sizeof(double) * 3 * n + 256, &zp));
  cuDoubleComplex* S = (cuDoubleComplex*)zp;
  cuDoubleComplex* T = S + small;
  double* d = (double*)(T + small);
  double* w = d + n;
  double* dg = w + n;
  int lw_potrf = 0, lw_heevd = 0;
  FE_CUSOLVER(cusolverDnZpotrf_bufferSize(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, S, n, &lw_potrf));
  FE_CUSOLVER(cusolverDnZheevd_bufferSize(m->cusolver, CUSOLVER_EIG_MODE_VECTOR,
                                          CUBLAS_FILL_MODE_UPPER, n, T, n, w, &lw_heevd));
  const int lwork = lw_potrf > lw_heevd ? lw_potrf : lw_heevd;
  void* wk;
  FE_TRY(fe_ws(m, WS_TC, sizeof(cuDoubleComplex) * ((size_t)lwork + 4), &wk));
  cuDoubleComplex* work = (cuDoubleComplex*)wk;
  int* info = (int*)(work + lwork);

  FE_TRY(fe_hx_step(m, X, HR, nullptr, nr, ldr, 1.0, 0.0, 0.0, FE_F32));
  const float onef = 1.0f, zerof = 0.0f;
  const cublasComputeType_t ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  {
    FiniteEmulationGuard finite(m->cublas);
    FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_N, CUBLAS_OP_T, nr, nr, (int)N, &onef, X,
                           CUDA_R_32F, (int)ldr, X, CUDA_R_32F, (int)ldr, &zerof, Gf, CUDA_R_32F,
                           nr, ct, CUBLAS_GEMM_DEFAULT));
    FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_N, CUBLAS_OP_T, nr, nr, (int)N, &onef, X,
                           CUDA_R_32F, (int)ldr, HR, CUDA_R_32F, (int)ldr, &zerof, Cf, CUDA_R_32F,
                           nr, ct, CUBLAS_GEMM_DEFAULT));
  }
  const int gs = fe::grid_for((int64_t)small);
  k_lane_combine<<<gs, 256, 0, st>>>(Gf, n, S); fe_count_launch();
  k_lane_combine<<<gs, 256, 0, st>>>(Cf, n, T); fe_count_launch();
  k_pencil_scale<<<(n + 255) / 256, 256, 0, st>>>(S, d, n); fe_count_launch();
  k_scale_pencil<<<gs, 256, 0, st>>>(S, T, d, n); fe_count_launch();
  FE_CUSOLVER(cusolverDnZpotrf(m->cusolver, CUBLAS_FILL_MODE_UPPER, n, S, n, work, lwork, info));
  k_zdiag<<<(n + 255) / 256, 256, 0, st>>>(S, n, dg); fe_count_launch();
  std::vector<double> rdiag(n);
  int hinfo = 0;
  FE_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaMemcpyAsync(rdiag.data(), dg, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) { *ill = true; return FE_OK; }
  double rmax = 0.0, rmin = 1e300;
  for (int j = 0; j < n; ++j) {
    rmax = std::fmax(rmax, std::fabs(rdiag[j]));
    rmin = std::fmin(rmin, std::fabs(rdiag[j]));
  }
  if (!(rmin > 0.0) || (rmax / rmin) * (rmax / rmin) > kGramCondTC32) { *ill = true; return FE_OK; }
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  // Hh = U^-H T U^-1, Hh w = lambda w, Y = D U^-1 w
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_C,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  FE_CUSOLVER(cusolverDnZheevd(m->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, T,
                               n, w, work, lwork, info));
  FE_CUBLAS(cublasZtrsm(m->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, n, n, &one, S, n, T, n));
  k_scale_rows<<<gs, 256, 0, st>>>(T, d, n); fe_count_launch();
  k_rotation_lanes<<<gs, 256, 0, st>>>(T, n, Gf); fe_count_launch();
  {
    // tmp (column-major 2n x N, ld 2 ld) = W^T R^T
    FiniteEmulationGuard finite(m->cublas);
    FE_CUBLAS(cublasGemmEx(m->cublas, CUBLAS_OP_T, CUBLAS_OP_N, nr, (int)N, nr, &onef, Gf,
                           CUDA_R_32F, nr, X, CUDA_R_32F, (int)ldr, &zerof, tmp, CUDA_R_32F,
                           (int)ldr, ct, CUBLAS_GEMM_DEFAULT));
  }
  FE_CUDA(cudaMemcpy2DAsync(X, ldr * 4, tmp, ldr * 4, (size_t)nr * 4, N,
                            cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(eig, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  FE_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) return fe_fail(FE_ECUDA, "fe_rayleigh_ritz: heevd info %d", hinfo);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // namespace

fe_status fe_rr_complex(fe_mesh* m, void* X, int64_t nvec, int64_t ld, double* eig,
                        fe_precision prec) {
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_rayleigh_ritz: complex blocks in FE_F64 or FE_F32");
  if (prec == FE_F32 && m->rr_products == 1) {
    bool ill = false;
    FE_TRY(rr_complex_tc32(m, (float*)X, nvec, ld, eig, &ill));
    if (!ill) return FE_OK;
  }
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

// Internal declarations of libfe (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/fe.h"

#define FE_MAXP 6
#define FE_MAXN1 (FE_MAXP + 1)
#define FE_NWS 19   // workspace slots of a mesh

// ---- error state ------------------------------------------------------------------------
fe_status fe_fail(fe_status st, const char* fmt, ...);

// ---- instrumentation: number of this library's kernels enqueued (graph replays included) ----
void fe_count_launch(int64_t n = 1);

#define FE_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return (cudaGetLastError(),                                                      \
              fe_fail(FE_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                      cudaGetErrorString(e_)));                                        \
  } while (0)

#define FE_CUBLAS(call)                                                                \
  do {                                                                                 \
    cublasStatus_t s_ = (call);                                                        \
    if (s_ != CUBLAS_STATUS_SUCCESS)                                                   \
      return fe_fail(FE_ECUDA, "%s:%d %s: cublas status %d", __FILE__, __LINE__, #call, \
                     (int)s_);                                                         \
  } while (0)

#define FE_CUSOLVER(call)                                                              \
  do {                                                                                 \
    cusolverStatus_t s_ = (call);                                                      \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                 \
      return fe_fail(FE_ECUDA, "%s:%d %s: cusolver status %d", __FILE__, __LINE__,     \
                     #call, (int)s_);                                                  \
  } while (0)

// ---- programmatic dependent launch ---------------------------------------------------------
// Short kernels that run back to back on one stream (the float CG iteration) are launched with
// programmatic stream serialization: the next kernel may be scheduled while the current one
// drains, and waits at its entry (griddepcontrol.wait) until its predecessor has completed and
// its writes are visible, so the ordering is exactly that of plain launches.  Each such kernel
// also lets its own dependent be scheduled as soon as all of its CTAs have started.  In a
// kernel launched without the attribute both instructions are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void fe_pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t fe_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

#define FE_TRY(expr)                  \
  do {                                \
    fe_status t_ = (expr);            \
    if (t_ != FE_OK) return t_;       \
  } while (0)

// ---- cuBLAS's FP32-accurate BF16x9 emulation on finite blocks ----------------------------
// The Rayleigh-Ritz products of float blocks run as BF16x9 emulated GEMMs.  By default cuBLAS
// first scans both operands for infinities and NaNs; the blocks here are finite, so the
// guard turns that scan off for its lifetime and restores the previous setting after.
struct FiniteEmulationGuard {
  cublasHandle_t h;
  cudaEmulationSpecialValuesSupport old = CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT;
  explicit FiniteEmulationGuard(cublasHandle_t handle) : h(handle) {
    if (cublasGetEmulationSpecialValuesSupport(h, &old) != CUBLAS_STATUS_SUCCESS)
      old = CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT;
    cublasSetEmulationSpecialValuesSupport(h, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
  }
  ~FiniteEmulationGuard() { cublasSetEmulationSpecialValuesSupport(h, old); }
  FiniteEmulationGuard(const FiniteEmulationGuard&) = delete;
  FiniteEmulationGuard& operator=(const FiniteEmulationGuard&) = delete;
};

// ---- Gram-path acceptance -------------------------------------------------------------------
// Largest cond(D S D) (D S D the diagonally scaled Gram matrix) for which the Rayleigh-Ritz
// Gram path is used: its results degrade like cond times the relative error of the Gram
// products, so double products (about 1e-16) allow 1e8 and FP32-accurate tensor-core ones
// (about 1e-7) 1e4.  Above it the block takes the explicit or double path.
constexpr double kGramCondF64 = 1e8;
constexpr double kGramCondTC32 = 1e4;

// ---- tensor-product operator arguments ----------------------------------------------------
// The assembled stiffness of the tensor-product mesh is
//   K = ax K1 (x) M1 (x) M1 + ay M1 (x) K1 (x) M1 + az M1 (x) M1 (x) K1   (x (x) y (x) z),
// with K1, M1 the exact 1D reference element matrices assembled along each axis, and the
// lumped overlap is M = J mx (x) my (x) mz.  The operator kernel applies
//   Y = alpha (oscale * K (S X) + (V - c) X) + beta Z,  S = diag(input scale),
// sweeping z.  Coefficient tables carry the per-local-index input scales.
struct KronCoef {
  // in-plane: y contraction (a = Ay_M U, b = Ay_K U) then x contraction
  // (W1 = Ax_M a, W2 = Ax_K a + Ax_M b); rows = output local index, cols = input local index
  double AyM[FE_MAXN1][FE_MAXN1], AyK[FE_MAXN1][FE_MAXN1];
  double AxM[FE_MAXN1][FE_MAXN1], AxK[FE_MAXN1][FE_MAXN1];
  // z contraction (cell-local): acc[j] += AzK[j][k] W1 + AzM[j][k] W2
  double AzK[FE_MAXN1][FE_MAXN1], AzM[FE_MAXN1][FE_MAXN1];
  double sig[FE_MAXN1];   // per-local-index in-plane output scale factor (x and y)
  double wz[FE_MAXN1];    // GLL weights (for the z mass factor of a plane)
  double zin;             // J^-1/2 (or 1 for the Poisson operator)
  double zout;            // 1/2 J^-1/2 (or 1)
  double ax, ay;          // the in-plane stiffness scales hy hz / (2 hx), hx hz / (2 hy)
  int mass_scale;         // 1: Hamiltonian (mass-scaled), 0: plain K
  int cplx;               // 1: the Bloch first-derivative operator A; the launch writes -i A X
                          //    on interleaved (re, im) lanes
};

struct KronGeom {
  int p, NX, NY, nz;      // nodes per periodic row, cells in z
  int gz_lo, NZs;         // first stored plane, number of stored planes
  int bx, by, zseg;       // cells per block in x, y; layers per z segment
  int nbx, nby;           // blocks in x, y
};

template <typename T>
struct KronIO {
  const T* X; int64_t ldx;
  T* Y; int64_t ldy;
  const T* Z; int64_t ldz;   // previous Chebyshev iterate (nullptr: beta ignored)
  const T* V;                // potential per stored node (nullptr: none)
  int64_t nvec;
  T alpha, beta, shift;      // Y = alpha (H - shift) X + beta Z
};

// One instance of a batched operator launch (device-resident array, ascending cta0).
template <typename T>
struct KronInst {
  KronGeom g;
  KronIO<T> io;
  int64_t cta0;              // first CTA of this instance in the batched 1D grid
  int64_t nvt;               // vector tiles of this instance
  int full;                  // complete xy blocks and vector tiles (set by the plan)
};


// operator launchers: double with 16-byte chunks, float with 16-byte chunks, and double
// with one element per node (single-vector Poisson operator)
// (the tile fields of g are chosen by the launcher)
namespace fe {
fe_status kron_f64(const KronCoef& cf, const KronGeom& g, const KronIO<double>& io,
                   cudaStream_t st);
fe_status kron_f32(const KronCoef& cf, const KronGeom& g, const KronIO<float>& io,
                   cudaStream_t st);
fe_status kron_k1(const KronCoef& cf, const KronGeom& g, const KronIO<double>& io,
                  cudaStream_t st);
// Batched launches: plan fills the tile fields, z segmentation, nvt and cta0 of n host
// instances (g from fe_geom, io.nvec set) and returns the total CTA count; launch runs one
// operator application over the device copy of those instances.
// zseg_req > 0 asks for that z-segment length (cells per CTA along z); counter != nullptr
// launches the persistent, dynamically scheduled form (counter: one device word, reset by
// the launch).
int64_t kron_batch_plan_f64(int p, KronInst<double>* inst, int n, int zseg_req);
int64_t kron_batch_plan_f32(int p, KronInst<float>* inst, int n, int zseg_req);
fe_status kron_batch_f64(const KronCoef& cf, int p, const KronInst<double>* d_inst, int n,
                         int64_t total_ctas, bool use_z, bool full, cudaStream_t st,
                         unsigned long long* counter);
fe_status kron_batch_f32(const KronCoef& cf, int p, const KronInst<float>* d_inst, int n,
                         int64_t total_ctas, bool use_z, bool full, cudaStream_t st,
                         unsigned long long* counter);
}  // namespace fe

// ---- nonlocal projector tables (fe_nonlocal.cu) --------------------------------------------
struct FeNonlocal {
  int natoms = 0, nnz = 0, ntouched = 0;
  int* atom_ptr = nullptr;     // [natoms + 1] entries of each atom
  int* ent_node = nullptr;     // [nnz] psi node of each entry
  int* ent_atom = nullptr;     // [nnz]
  double* ent_val = nullptr;   // [nnz][4] M^1/2 p_beta at the node
  float* ent_val_f = nullptr;
  double* D = nullptr;         // [natoms][4]
  float* D_f = nullptr;
  int* tn_node = nullptr;      // [ntouched] psi nodes carrying entries
  int* tn_ptr = nullptr;       // [ntouched + 1]
  int* tn_ent = nullptr;       // [nnz] entries in node order
};

// ---- the mesh ---------------------------------------------------------------------------
struct fe_mesh {
  fe_mesh_desc desc;
  int p, nx, ny, nz;
  int NX, NY, NZ;          // NZ = nz p + 1 phi planes
  int gz_lo, gz_hi, NZs;   // stored psi planes
  int64_t n_phi, n_psi, n_cells;
  double h[3], J;
  double xi[FE_MAXN1], w[FE_MAXN1];
  double K1[FE_MAXN1][FE_MAXN1], M1[FE_MAXN1][FE_MAXN1];
  double G1[FE_MAXN1][FE_MAXN1];   // int l_i l_j' on the reference interval
  cudaStream_t stream;
  int device;
  cudaStream_t aux_stream = nullptr;   // library-owned, non-blocking: graph capture
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  KronCoef coefH;          // Hamiltonian (mass-scaled, 1/2 factor)
  KronCoef coefK;          // plain stiffness
  // Bloch wave vector (x, y) and the antisymmetric operator M^-1/2 (kx Gx + ky Gy) M^-1/2
  double kx = 0.0, ky = 0.0;
  bool has_k = false;
  KronCoef coefA;

  double* d_veff = nullptr;   // [n_psi]
  float* d_veff_f = nullptr;  // [n_psi]
  bool has_potential = false;

  int natoms = 0;
  double* d_atoms = nullptr;  // [natoms][4] = x, y, z, Z
  double* h_atoms = nullptr;
  double sigma_b = 0.5, rc_loc = 1.0, sigma_rho = 1.0;
  double* d_vlms = nullptr;   // V_loc - V_sm at phi nodes
  double* d_rho = nullptr;    // model density at phi nodes (renormalised)
  double* d_b = nullptr;      // smeared nuclear charge at phi nodes (renormalised)
  double* d_mass = nullptr;   // lumped mass at phi nodes
  double rho_scale = 1.0;     // rho = rho_scale * sum_a Z_a g_{sigma_rho}
  double n_electrons = 0.0;

  // workspaces (grown on demand, freed with the mesh)
  void* ws[FE_NWS] = {nullptr};
  size_t ws_bytes[FE_NWS] = {0};

  // Rayleigh-Ritz block products for float storage: 0 double GEMMs, 1 tensor-core BF16x9
  int rr_products = 0;
  int rr_eigen = 0;                 // FE_RR_EIGEN_SYEVD / FE_RR_EIGEN_SYEVJ
  syevjInfo_t syevj_params = nullptr;
  // Poisson CG preconditioner: 0 Jacobi, 1 Jacobi plus the exact z-plane coarse solve
  int poisson_precond = 2;          // FE_PRECOND_JACOBI_PLANES_MODES
  // Poisson arithmetic: 0 double CG, 1 float corrections with double residuals
  int poisson_arith = 1;
  int poisson_iter = 0;             // FE_POISSON_ITER_PERSISTENT / FE_POISSON_ITER_LAUNCHES
  int cg_stall = -1;                // FE_OPT_TEST_CG_STALL
  FeNonlocal nl;            // nonlocal term (natoms == 0: none)
  // potential by Gauss quadrature (fe_quadpot.cu): Bq[q][i] = l_i(gauss point q), wq the
  // Gauss weights (p + 1 points); W = w |J| V at every cell's Gauss points; M^-1/2 at psi nodes
  double Bq[FE_MAXN1][FE_MAXN1] = {}, wq[FE_MAXN1] = {};
  bool has_quad = false;
  double* d_qW = nullptr;
  float* d_qW_f = nullptr;
  double* d_rsq = nullptr;
  float* d_rsq_f = nullptr;

  // cached coarse-space inverse (WS_PCOARSE): valid for the constraint set of pc_key
  int pc_state = 0;          // 0 none, 1 valid, 2 not SPD (Jacobi only for this key)
  int pc_modes = 0;          // in-plane mode coarse space: 0 not built, 1 valid, 2 not used
  int pc_nz = 0;
  fe_poisson_bc pc_key = {};

  // tensor-core path: p of the uploaded cell-matrix image, pinned wait-expiry flag
  int tc_img_p = -1;
  int* tc_err_pinned = nullptr;
  // tensor-core sum-factorised operator (fe_kron_tc.cu): operator images uploaded, and the
  // host copy of its wait-expiry flag
  bool ktc_ready = false;
  int* ktc_err_pinned = nullptr;

  cublasHandle_t cublas = nullptr;
  cusolverDnHandle_t cusolver = nullptr;

};

enum { WS_CHEB = 0, WS_RR_X = 1, WS_RR_HX = 2, WS_RR_SMALL = 3, WS_CG = 4, WS_RED = 5,
       WS_LANCZOS = 6, WS_TC = 7, WS_TC_IMG = 8, WS_YCELL = 9, WS_RR_TC32 = 10,
       WS_PCOARSE = 11, WS_NL = 12, WS_KCELL = 13, WS_XC = 14, WS_KPT = 15, WS_KTC = 16,
       WS_CGF = 17, WS_PMODES = 18 };

fe_status fe_ws(fe_mesh* m, int slot, size_t bytes, void** out);
// Rayleigh-Ritz of a complex (Bloch) block: nvec, ld count complex entries (fe_kpoint.cu)
fe_status fe_rr_complex(fe_mesh* m, void* X, int64_t nvec, int64_t ld, double* eig,
                        fe_precision prec);
// single-vector float stiffness product through cell-local products (fe_kcell.cu); its
// scratch (WS_KCELL) is fe_kcell_scratch_bytes
size_t fe_kcell_scratch_bytes(const fe_mesh* m);
fe_status fe_kcell_apply_f32(fe_mesh* m, const float* x, float* y);
fe_status fe_activate(const fe_mesh* m);
KronGeom fe_geom(const fe_mesh* m, bool psi);
// Y = alpha (Ht - shift) X + beta Z (plus alpha Ht_nloc X and the quadrature potential when
// the mesh carries them) in the requested arithmetic; nvec and ld count real lanes
// (fe_hx.cu)
fe_status fe_hx_step(fe_mesh* m, const void* X, void* Y, const void* Z, int64_t nvec, int64_t ld,
                     double alpha, double beta, double shift, fe_precision prec);

// nonlocal term -- fe_nonlocal.cu: Y += alpha Ht_nloc X; release of the tables
fe_status fe_nonlocal_apply(fe_mesh* m, const void* X, void* Y, int64_t nvec, int64_t ld,
                            double alpha, bool dbl);
void fe_nonlocal_free(fe_mesh* m);
// potential by Gauss quadrature -- fe_quadpot.cu: Y += alpha M^-1/2 V_quad M^-1/2 X (no-op
// unless fe_set_potential_quad is in effect); basis tables at mesh creation; release
fe_status fe_quad_apply(fe_mesh* m, const void* X, void* Y, int64_t nvec, int64_t ld,
                        double alpha, bool dbl);
void fe_quad_setup_basis(fe_mesh* m);
void fe_quad_free(fe_mesh* m);

// fields (potentials, densities) -- fe_fields.cu
fe_status fe_fields_build(fe_mesh* m);
// deterministic reductions -- fe_blas.cu
fe_status fe_dot(fe_mesh* m, const double* x, const double* y, int64_t n, double* out_dev);

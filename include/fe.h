/*
 * fe.h -- C ABI of libfe, a GB300 (sm_103a) library for the data-parallel hot path of
 * real-space finite-element Kohn-Sham DFT for slabs under an external potential bias
 * (Ramakrishnan, Sai Gautam, Motamarri, "Real-space methods for ab initio modeling of
 * surfaces and interfaces under external potential bias").
 *
 * Discrete problem (Section 2.3, FE discretization): C0 Lagrange elements of degree p on
 * GLL nodes over a uniform hexahedral mesh of the box [0,Lx) x [0,Ly) x [0,Lz], periodic
 * in x and y.  The Kohn-Sham eigenproblem H u = eps M u (Section 2.3) is handled in the
 * symmetric standard form  Ht = M^-1/2 H M^-1/2 = 1/2 M^-1/2 K M^-1/2 + diag(V_eff),
 * K_IJ = int grad N_I . grad N_J (Section 2.3), M the GLL-lumped overlap, V_eff collocated
 * at the nodes (Eq. Veff and Hloc; the exchange-correlation term is not part of this
 * library).  The Poisson problem -1/(4 pi) Lap phi = rho + b (Eq. Poissons equation) is
 * K phi = 4 pi c, c_I = M_II (rho + b)(x_I), with the bias setups of Section 2.2:
 * CEF (Eq. governing_equations CEF) and CPD / L-CPD (Eq. governing_equations APD).
 *
 * Node numbering.  Global node (gx, gy, gz), gx in [0, nx p), gy in [0, ny p),
 * gz in [0, nz p]; node coordinate along an axis with cell size h: (g / p) h +
 * (xi_{g mod p} + 1) h / 2 with xi the GLL points on [-1, 1].
 *   phi node id = gx + NX (gy + NY gz)                    (NX = nx p, NY = ny p)
 *   psi node id = gx + NX (gy + NY (gz - gz_lo))          gz_lo = 1 if the bottom psi face
 *                 is homogeneous Dirichlet, else 0; the top Dirichlet face drops gz = nz p.
 *
 * Conventions for every call:
 *   - All arrays are owned by the caller and are never freed by the library.  Arrays
 *     named *_dev are device pointers on the mesh's device; *_host are host pointers.
 *   - Wavefunction blocks are node-major with the vectors contiguous: element (node i,
 *     vector j) is at X[i * ld + j], 0 <= j < nvec <= ld.  FE_F64 blocks are double,
 *     all other precisions use float storage.  X must be 16-byte aligned and
 *     ld * sizeof(element) must be a multiple of 16 bytes.
 *   - Work is enqueued on the mesh's stream in order.  Calls that return host scalars
 *     (info structs, bounds) synchronise that stream; the others do not.
 *   - Errors are reported as status codes, never by aborting; fe_last_error() gives a
 *     thread-local message for the last non-FE_OK status.  Arguments are validated on
 *     the host before anything is enqueued; a failing call leaves outputs unspecified.
 *   - Iterative device loops carry an iteration cap and report FE_ENOCONV; no device
 *     code waits without a bound.
 */
#ifndef FE_H
#define FE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FE_OK = 0,
  FE_EINVAL = 1,        /* invalid argument (null pointer, bad size, misalignment)     */
  FE_ENOMEM = 2,        /* device allocation failed                                     */
  FE_ECUDA = 3,         /* a CUDA / cuBLAS / cuSOLVER call failed                       */
  FE_ENOCONV = 4,       /* an iteration hit its cap before the tolerance                */
  FE_EBREAKDOWN = 5,    /* Cholesky of a Gram matrix failed (not positive definite)     */
  FE_ETIMEOUT = 6,      /* reserved: a bounded device wait expired                      */
  FE_EUNSUPPORTED = 7   /* valid request that the library does not implement           */
} fe_status;

/* Arithmetic of the Hamiltonian application.
 *   FE_F64          double storage, double sum-factorised products (exact path).
 *   FE_F32          float storage, float sum-factorised products, float accumulation.
 *   FE_BF16_F32ACC  float storage, per-cell dense stiffness products with bf16 operands
 *                   on the tcgen05 tensor cores, float accumulation in tensor memory.
 *   FE_F32_F32ACC   reserved for per-cell dense products with the float operands split
 *                   into bf16 high and low parts on tcgen05; not built in this version:
 *                   every entry point returns FE_EUNSUPPORTED for it.                    */
typedef enum { FE_F64 = 0, FE_F32 = 1, FE_BF16_F32ACC = 2, FE_F32_F32ACC = 3 } fe_precision;

/* Wavefunction boundary condition on a z face (x and y are always periodic). */
typedef enum { FE_FACE_NEUMANN = 0, FE_FACE_DIRICHLET = 1 } fe_face_bc;

typedef struct fe_mesh fe_mesh; /* opaque, library-owned */

typedef struct {
  double L[3];            /* box lengths Lx, Ly, Lz (bohr), > 0                       */
  int ncell[3];           /* cells per direction, >= 1                                  */
  int p;                  /* polynomial degree, 1 <= p <= 6                              */
  fe_face_bc psi_z[2];    /* psi condition on the z = 0 and z = Lz faces                 */
  int device;             /* CUDA device ordinal                                         */
  void* stream;           /* cudaStream_t for all work of this mesh (NULL = legacy)      */
} fe_mesh_desc;

/* Create a mesh (Section 2.3).  Builds the 1D GLL rules and element matrices on the host
 * and uploads the node tables.  *out receives a handle owned by the library. */
fe_status fe_mesh_create(const fe_mesh_desc* desc, fe_mesh** out);
fe_status fe_mesh_destroy(fe_mesh* mesh);
fe_status fe_mesh_info(const fe_mesh* mesh, int64_t* n_phi, int64_t* n_psi, int64_t* n_cells);
/* Replace the stream used by all later calls on this mesh. */
fe_status fe_mesh_set_stream(fe_mesh* mesh, void* stream);

/* Per-mesh options.
 *   FE_OPT_RR_PRODUCTS: arithmetic of the three block products of fe_rayleigh_ritz for
 *     float-storage blocks.  FE_RR_PRODUCTS_F64 (default): double GEMMs on a promoted copy.
 *     FE_RR_PRODUCTS_TC32: X^T X, X^T (Ht X) and X C as tensor-core GEMMs in cuBLAS's
 *     FP32-accurate BF16x9 emulation on the float block (relative error ~1e-7, the
 *     precision of the float storage itself); the n x n Cholesky, projection and
 *     eigensolve stay in double.  FE_F64 blocks always use double GEMMs. */
enum { FE_OPT_RR_PRODUCTS = 0, FE_OPT_POISSON_PRECOND = 1, FE_OPT_POISSON_ARITH = 2 };
enum { FE_RR_PRODUCTS_F64 = 0, FE_RR_PRODUCTS_TC32 = 1 };
/*   FE_OPT_POISSON_PRECOND: preconditioner of the Poisson CG.  FE_PRECOND_JACOBI: the
 *     diagonal of K.  FE_PRECOND_JACOBI_PLANES: the diagonal plus an exact solve
 *     on the coarse space of z-planes (one basis function per phi plane: the indicator of
 *     its free nodes), i.e. M^-1 = D^-1 + R^T (R K R^T)^-1 R with R the free-node plane
 *     sums.  The coarse matrix is banded (planes within one cell layer couple) and is
 *     factorised once per solve.  It removes the slow modes that are constant over x and y,
 *     which dominate on long slabs.  The converged solution is the same; only the
 *     iteration count changes. */
/*     FE_PRECOND_JACOBI_PLANES_MODES (default): the plane coarse space enriched, on every
 *     plane, with the in-plane Fourier modes of wavenumber one (cos and sin of 2 pi x / Lx
 *     and of 2 pi y / Ly on the plane's nodes); on a mesh without constrained phi nodes (the
 *     CEF setup) they are decoupled from one another by the cell-translation invariance of
 *     K, so each is one more exact nz x nz coarse solve.  Used by the persistent float
 *     iteration (FE_OPT_POISSON_ITER) on such meshes when they span at least 8 cells along
 *     both x and y (on narrower slabs these modes are not slow ones) and the planes hold a
 *     multiple of four nodes along x; elsewhere it acts as FE_PRECOND_JACOBI_PLANES.  Built
 *     once per mesh and constraint set (4 x (2p + 1) more double operator applications). */
enum { FE_PRECOND_JACOBI = 0, FE_PRECOND_JACOBI_PLANES = 1, FE_PRECOND_JACOBI_PLANES_MODES = 2 };
/*   FE_OPT_POISSON_ARITH: arithmetic of the Poisson solve.  FE_POISSON_F64: CG in double.
 *     FE_POISSON_MIXED (default): a float CG (operator, vectors and preconditioner in float,
 *     dot products accumulated in double) with reliable updates -- whenever its residual has
 *     dropped by 1e2, phi (double) takes the float iterate and the residual is replaced by
 *     the double residual f - K phi (the search direction restarts when the two residuals
 *     have drifted apart); if an update interval stops reducing that residual,
 *     double CG finishes from the current phi.  The stopping test (rtol on the double
 *     residual) and so the accuracy of phi are those of FE_POISSON_F64. */
enum { FE_POISSON_F64 = 0, FE_POISSON_MIXED = 1 };
/*   FE_OPT_RR_EIGEN: dense symmetric eigensolver of the n x n projected matrix in
 *     fe_rayleigh_ritz (double precision either way).  FE_RR_EIGEN_SYEVD (default):
 *     divide-and-conquer (cuSOLVER syevd).  FE_RR_EIGEN_SYEVJ: cyclic Jacobi (cuSOLVER
 *     syevj) to a residual tolerance of 1e-14 relative, at most 100 sweeps; FE_ECUDA if it
 *     does not converge. */
enum { FE_OPT_RR_EIGEN = 3 };
enum { FE_RR_EIGEN_SYEVD = 0, FE_RR_EIGEN_SYEVJ = 1 };
/*   FE_OPT_POISSON_ITER: how the float CG of FE_POISSON_MIXED runs its iterations.
 *     FE_POISSON_ITER_PERSISTENT (default): one cooperative kernel runs the iterations
 *     between two reliable updates, its steps separated by grid-wide barriers (each wait
 *     bounded: a barrier that gives up ends the solve with FE_ETIMEOUT); used with the
 *     plane coarse space when the device supports cooperative launches and the phi planes
 *     hold a multiple of four nodes, otherwise the launch-per-step iteration runs.
 *     FE_POISSON_ITER_LAUNCHES: one kernel launch per step (seven per iteration), replayed
 *     from CUDA graphs.  The arithmetic of an iteration is the same; the dot products are
 *     summed in another fixed order, so iterates agree to rounding, not bitwise. */
enum { FE_OPT_POISSON_ITER = 4 };
enum { FE_POISSON_ITER_PERSISTENT = 0, FE_POISSON_ITER_LAUNCHES = 1 };
/*   FE_OPT_TEST_CG_STALL: a test aid for the bounded waits of the persistent iteration.  A
 *     value b >= 0 makes block b of its grid return before the first grid barrier, so no
 *     barrier completes: the other blocks' waits run out (2 s), the launch ends and the
 *     solve returns FE_ETIMEOUT with the mesh still usable.  -1 (the default) turns it
 *     off. */
enum { FE_OPT_TEST_CG_STALL = 5 };
fe_status fe_set_option(fe_mesh* mesh, int option, int64_t value);

/* Node coordinates in phi order, xyz_dev[n_phi][3] (Section 2.3 node layout). */
fe_status fe_node_coords(const fe_mesh* mesh, double* xyz_dev);
/* Diagonal of the GLL-lumped overlap M on phi nodes, m_dev[n_phi]. */
fe_status fe_lumped_mass(const fe_mesh* mesh, double* m_dev);

/* Pseudo-atoms (Eq. Governing equations1): positions R_host[n][3] (bohr) and valence
 * charges Z_host[n].  Defines V_loc^a = -Z erf(r/rc_loc)/r, the smeared nuclear charge
 * b^a = -Z g_{sigma_b} (g_s a normalised Gaussian of standard deviation s) with
 * V_sm^a = -Z erf(r/(sqrt2 sigma_b))/r, and the model electron density
 * rho = sum_a Z_a g_{sigma_rho}.  Periodic x/y images are summed; every atom-centred
 * function is cut at 10 bohr.  b^a is renormalised per atom and rho globally so that
 * their lumped integrals are exactly -Z_a and sum Z_a.  The arrays are copied. */
fe_status fe_set_atoms(fe_mesh* mesh, int n, const double* R_host, const double* Z_host,
                       double sigma_b, double rc_loc, double sigma_rho);

/* Nonlocal pseudopotential term (Eq. V_nloc) with synthetic projectors: per atom a one s
 * and three p channels, g = exp(-|d|^2 / (2 sigma_a^2)), p_s = g, p_x = (d_x / sigma_a) g,
 * p_y, p_z likewise (d = x - R_a over the periodic x/y images, cut at |d| <= rc), and
 * coefficients D_host[a][4] (s, x, y, z).  With the lumped quadrature the scaled operator
 * gains Ht_nloc = M^1/2 P D P^T M^1/2, applied inside every Ht X of fe_apply_H,
 * fe_cheb_filter, fe_rayleigh_ritz and fe_lanczos_bounds (all precisions).  natoms = 0
 * removes the term.  Arrays are host arrays and are copied.  A mesh carrying the term is
 * refused by fe_batch_create and fe_cheb_filter_static (FE_EUNSUPPORTED). */
fe_status fe_set_nonlocal(fe_mesh* mesh, int natoms, const double* R_host,
                          const double* sigma_host, const double* D_host, double rc);

/* Bloch wave vector (Section 2.1: Bloch's theorem along the periodic x and y directions,
 * psi = e^{i k.x} u, H^k_loc = -1/2 Laplacian - i k.grad + 1/2 |k|^2 + V_eff on u).  With
 * k = (kx, ky) != 0 the scaled operator becomes the Hermitian
 * Ht_k = Ht_0 + |k|^2 / 2 - i M^-1/2 (kx Gx + ky Gy) M^-1/2 (G^d_IJ = int N_I dN_J/dx_d,
 * exact; the |k|^2 term with the lumped overlap), and the blocks of fe_apply_H,
 * fe_cheb_filter and fe_rayleigh_ritz are complex: interleaved (re, im) pairs of float
 * (FE_F32) or double (FE_F64), nvec and ld counting complex entries (16-byte aligned rows).
 * fe_rayleigh_ritz then solves the Hermitian subspace problem (n x n part in double complex;
 * for float blocks with FE_RR_PRODUCTS_TC32 the block products are real FP32-accurate
 * tensor-core GEMMs over the (re, im) lanes, else double complex GEMMs); fe_density
 * sums occ_n |u_n|^2 over the complex columns; fe_lanczos_bounds bounds the spectrum of
 * Ht_k.  k = (0, 0) restores the real Gamma-point operator.  Not combined with the nonlocal
 * term, the tensor-core precisions, fe_batch_create or fe_cheb_filter_static
 * (FE_EUNSUPPORTED).  FE_EINVAL for a null mesh or a non-finite k. */
fe_status fe_set_kpoint(fe_mesh* mesh, double kx, double ky);

/* V_eff at psi nodes, veff_dev[n_psi] (Eq. Veff and Hloc without exchange-correlation:
 * V_eff = phi + V_loc - V_sm + V_app).  Copied into the mesh. */
fe_status fe_set_potential(fe_mesh* mesh, const double* veff_dev);

/* Potential term integrated by Gauss quadrature instead of GLL collocation: the consistent
 * FE matrix V_IJ = int N_I V_eff N_J dx of the discretised Kohn-Sham operator (Section 2.3),
 * evaluated cell by cell with the (p+1)-point Gauss-Legendre rule per direction from V_eff
 * at the Gauss points: vq_dev[n_cells][(p+1)^3] (device, double), cells with cx fastest then
 * cy then cz, point (a, b, c) (a along x) at a + (p+1)(b + (p+1) c), Gauss points ascending
 * on each cell's interval.  The operator becomes Ht = M^-1/2 (1/2 K + V) M^-1/2 with the
 * lumped overlap M; the cell matrices are applied in sum-factorised form, never stored.
 * Values are copied into the mesh (weights w |J| V folded in).  Replaces the collocated
 * potential for fe_apply_H, fe_cheb_filter(_static), fe_lanczos_bounds and
 * fe_rayleigh_ritz (any precision; complex blocks too) until fe_set_potential is called
 * again; fe_batch_create and the batched entry points refuse such a mesh (FE_EUNSUPPORTED).
 * FE_EINVAL for null arguments, FE_ENOMEM when its tables cannot be allocated. */
fe_status fe_set_potential_quad(fe_mesh* mesh, const double* vq_dev);

/* Values at every cell's Gauss points (layout of fe_set_potential_quad) of the FE field
 * with nodal values f_phi_dev[n_phi] (device, double): f(x_q) = sum_I N_I(x_q) f_I
 * (Section 2.3 basis).  out_dev[n_cells][(p+1)^3] (device, double, caller-owned). */
fe_status fe_interp_quad(fe_mesh* mesh, const double* f_phi_dev, double* out_dev);

/* Y = Ht X (Eq. Veff and Hloc, Section 2.3).  X, Y [n_psi][ld], nvec vectors; X and Y
 * must not overlap.  Needs fe_set_potential first. */
fe_status fe_apply_H(fe_mesh* mesh, const void* X, void* Y, int64_t nvec, int64_t ld,
                     fe_precision prec);

/* Adjoint of fe_apply_H with respect to the potential (Eq. Veff and Hloc: V_eff enters
 * Ht = 1/2 M^-1/2 K M^-1/2 + diag(V_eff) only through the diagonal term).  Given X and
 * Ybar = dL/dY for Y = Ht X: gV_dev[I] = sum_v Ybar[I][v] X[I][v], the gradient dL/dV_eff
 * of the collocated potential.  X, Ybar [n_psi][ld] in the storage type of prec (double
 * for FE_F64, float otherwise), nvec vectors; complex (Bloch) blocks: nvec and ld count
 * complex entries and the sum runs over both (re, im) lanes.  gV_dev [n_psi] double,
 * caller-owned, overwritten.  The adjoint with respect to X is fe_apply_H on Ybar (Ht is
 * symmetric).  Stream-ordered; deterministic (fixed summation order).  FE_EINVAL for null
 * arguments or nvec > ld; FE_EUNSUPPORTED while the Gauss-quadrature potential
 * (fe_set_potential_quad) is in effect. */
fe_status fe_potential_vjp(fe_mesh* mesh, const void* X, const void* Ybar, int64_t nvec,
                           int64_t ld, double* gV_dev, fe_precision prec);

/* In-place degree-m scaled Chebyshev filter of X (Zhou & Saad three-term recurrence):
 * X <- T_m((Ht - c)/e) X / T_m((a0 - c)/e), e = (b - a)/2, c = (b + a)/2, a0 < a < b;
 * degree counts applications of Ht.  Uses one library-owned workspace of X's size. */
fe_status fe_cheb_filter(fe_mesh* mesh, void* X, int64_t nvec, int64_t ld, int degree,
                         double a, double b, double a0, fe_precision prec);

/* Allocation-free variant of fe_cheb_filter.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library call cudaMalloc -- a process whose
 * framework allocator has already reserved the free device memory, a service that keeps a
 * fixed memory budget after start-up, or a latency-sensitive loop where cudaMalloc's
 * implicit device synchronisation would stall other streams.  Same arguments and result as
 * fe_cheb_filter for FE_F64 and FE_F32 (other precisions return FE_EUNSUPPORTED); the
 * recurrence's scratch block lives in a 64 MiB static device array compiled into the
 * library, so n_psi * ld * sizeof(element) must not exceed 64 MiB (FE_EINVAL otherwise).
 * The call performs no cudaMalloc / cudaFree and no allocating library call.
 * Set-up: the first call on a device looks up the array's device address with that device
 * current (cudaGetSymbolAddress); make that first call before any stream capture.  The
 * address is kept for the life of the process: like the meshes and their workspaces, it
 * does not survive cudaDeviceReset.  a0, a and b as for fe_cheb_filter (finite,
 * a0 < a < b; FE_EINVAL otherwise).
 * Sharing: every call on a device uses that device's one copy of the array, which keeps
 * the last call's contents (the filter writes the scratch before reading it, so stale
 * contents never matter); calls that overlap on the GPU, for example on two streams or two
 * meshes at once, race on it. */
fe_status fe_cheb_filter_static(fe_mesh* mesh, void* X, int64_t nvec, int64_t ld, int degree,
                                double a, double b, double a0, fe_precision prec);

/* ---- batches of independent slabs -------------------------------------------------------
 * A bias sweep (Section 3: one slab under a series of fields or potential differences, or
 * slabs of several thicknesses) is a set of independent eigenproblems.  A batch applies
 * each operator step to all of them in ONE kernel launch: Ht_i X_i for every instance i,
 * with the instance's own geometry, potential and block.  Instances must share p and the
 * cell size h (one element coefficient table); their cell counts, psi z-face conditions and
 * potentials may differ.  All meshes must be on one device and one stream; batched calls
 * run on that stream.  The batch borrows the meshes (destroy it before them) and owns only
 * a small device array of per-instance descriptors.  Only FE_F64 and FE_F32 are batched
 * (FE_EUNSUPPORTED otherwise).  A different p or cell size returns FE_EUNSUPPORTED. */
typedef struct fe_batch fe_batch;
fe_status fe_batch_create(fe_mesh* const* meshes, int n, fe_batch** out);
fe_status fe_batch_destroy(fe_batch* batch);

/* Y_i = Ht_i X_i for every instance (fe_apply_H per instance, one launch).  X, Y: host
 * arrays of n device pointers; nvec, ld: host arrays of n counts; same layout and alignment
 * rules as fe_apply_H per instance. */
fe_status fe_batch_apply_H(fe_batch* batch, const void* const* X, void* const* Y,
                           const int64_t* nvec, const int64_t* ld, fe_precision prec);

/* In-place filter of every X_i with its own bounds a[i] < b[i], a0[i] (host arrays): the
 * result equals fe_cheb_filter per instance; each of the degree steps is one launch over
 * all instances.  Uses each mesh's filter workspace. */
fe_status fe_batch_cheb_filter(fe_batch* batch, void* const* X, const int64_t* nvec,
                               const int64_t* ld, int degree, const double* a,
                               const double* b, const double* a0, fe_precision prec);

/* Cholesky-QR + Rayleigh-Ritz of every instance (the result of fe_rayleigh_ritz per
 * instance, Section 2.3's smallest eigenpairs): X host array of n device blocks with the
 * same nvec, ld host array, eig host array of n device pointers to [nvec] doubles
 * (ascending Ritz values).  Ht X is one batched launch and the n x n steps are batched
 * cuBLAS / cuSOLVER calls over all instances.  FE_F64 blocks use double products; FE_F32
 * blocks need FE_OPT_RR_PRODUCTS = FE_RR_PRODUCTS_TC32 on every mesh (FE_EUNSUPPORTED
 * otherwise).  An instance whose scaled Gram matrix is not safely positive definite is
 * redone by fe_rayleigh_ritz.  Uses each mesh's Rayleigh-Ritz workspace and a batch-owned
 * n x n work array. */
fe_status fe_batch_rayleigh_ritz(fe_batch* batch, void* const* X, int64_t nvec,
                                 const int64_t* ld, double* const* eig, fe_precision prec);

/* Launch configuration of the batched operator, chosen by the library's autotuner (the
 * paper runs each bias value as its own calculation; batching is this library's).  A
 * batched launch covers (instance, xy block, vector tile, z segment) work items; on the
 * first batched operator call of a batch every candidate -- the z-segment length (cell
 * layers per item: the occupancy heuristic, 2, 4, 8, 16, or each slab's whole height)
 * crossed with the grid form (one CTA per item, or a persistent grid of resident CTAs
 * taking items from a device counter, which balances slabs of uneven height) -- runs one
 * operator launch on the batch's own blocks, and the fastest is kept.  The choice is cached
 * for the process per device, precision and batch shape (later batches of the same shape
 * skip the timing).  fe_batch_tuning reports it: *zseg (0: the heuristic's length),
 * *persistent (0 or 1), *best_ms (the chosen launch's time; 0 when not timed for this
 * batch), *ncand (candidates timed for this batch; 0 when the choice came from the cache
 * or from fe_batch_set_launch).  FE_EINVAL before the first batched operator call.
 * fe_batch_set_launch fixes the configuration instead (zseg >= 0, persistent 0 or 1); the
 * results do not depend on it. */
fe_status fe_batch_tuning(const fe_batch* batch, int* zseg, int* persistent, double* best_ms,
                          int* ncand);
fe_status fe_batch_set_launch(fe_batch* batch, int zseg, int persistent);

/* ---- analysis outputs (Section 3) ---------------------------------------------------------
 * Per phi plane of a phi-node field f_dev [n_phi], out_dev [NZ] (NZ = nz p + 1 planes, in
 * z order): FE_PLANAR_INTEGRAL gives int_{S_z} f dx dy (Section 3.3's rho0(z)),
 * FE_PLANAR_AVERAGE gives (1/A_z) int_{S_z} f dx dy (V0_bare(z)); lumped (GLL) quadrature. */
enum { FE_PLANAR_INTEGRAL = 0, FE_PLANAR_AVERAGE = 1 };
fe_status fe_planar(fe_mesh* mesh, const double* f_dev, int mode, double* out_dev);

/* Dipole moment about the domain centre (Section 3.1), mu_z = int (b + rho)(z - Lz/2):
 * rho_dev [n_phi] or NULL for the atoms' model density; b from fe_set_atoms; mu_z on the
 * host.  The polarisability of Section 3.1 is the slope of mu_z over two fields. */
fe_status fe_dipole(fe_mesh* mesh, const double* rho_dev, double* mu_z);

/* ---- self-consistent closure ------------------------------------------------------------
 * Density of a block (Section 2.1, below Eq. Tsexc: rho = 2 sum_n f_n |psi_n|^2): the
 * block holds xt_n = M^1/2 u_n (orthonormal columns of Ht, Section 2.3), so
 * rho_dev[I] = sum_n occ_dev[n] X[I][n]^2 / M_II at psi nodes (occ = 2 f, device array of
 * nvec doubles) and 0 on the planes without psi nodes; rho_dev is [n_phi] (phi order), so
 * it feeds fe_poisson_solve directly.  FE_F64 and FE_F32 blocks, nvec <= 4096. */
fe_status fe_density(fe_mesh* mesh, const void* X, int64_t nvec, int64_t ld,
                     const double* occ_dev, double* rho_dev, fe_precision prec);

/* Fermi-Dirac occupations at smearing temperature kT (host arrays): occ_host[i] =
 * 2 / (1 + exp((eig[i] - mu)/kT)) with mu (bisection) such that sum occ = n_electrons
 * (0 <= n_electrons <= 2 n).  The paper defers the smearing to earlier work; this is the
 * reading used here.  Needs no GPU. */
fe_status fe_occupations(const double* eig_host, int n, double n_electrons, double kT,
                         double* occ_host, double* mu);

/* Local-density exchange for the self-consistent potential (Section 2.1: the exchange-
 * correlation potential enters V_eff as dE_xc/drho; this optional term is the closed-form
 * exchange of the homogeneous electron gas, spin unpolarised, without correlation — a
 * simplification of the paper's functional).  For the density rho_dev [n_phi] (values
 * below zero taken as zero): adds v_x = -(3/pi)^(1/3) rho^(1/3) at the psi nodes to
 * veff_dev [n_psi] in place (may be NULL), and writes E_x = sum_I M_II e_x(rho_I),
 * e_x = -(3/4)(3/pi)^(1/3) rho^(4/3), to *ex_host (may be NULL; the call then synchronises
 * the mesh stream).  FE_EINVAL for a null mesh or density. */
fe_status fe_lda_exchange(fe_mesh* mesh, const double* rho_dev, double* veff_dev,
                          double* ex_host);

/* Anderson / Pulay mixing of phi-node densities (D. G. Anderson 1965, P. Pulay 1980) with
 * the lumped-mass inner product: with R = rho_out - rho_in and the differences dR_i,
 * drho_i of the last `history` (0..16) steps, gamma minimises |R - sum gamma_i dR_i| and
 * rho_in <- rho_in + alpha R - sum gamma_i (drho_i + alpha dR_i) (history 0: linear
 * mixing).  The mixer owns (3 + 2 history) n_phi doubles on the mesh's device; calls run
 * on the mesh's stream; resid_norm (host) gets |R| in the same inner product. */
typedef struct fe_mixer fe_mixer;
fe_status fe_mixer_create(fe_mesh* mesh, int history, double alpha, fe_mixer** out);
fe_status fe_mixer_destroy(fe_mixer* mixer);
fe_status fe_mixer_step(fe_mixer* mixer, double* rho_in_dev, const double* rho_out_dev,
                        double* resid_norm);

typedef enum { FE_BIAS_CEF = 0, FE_BIAS_CPD = 1 } fe_bias_kind;

typedef struct {
  fe_bias_kind kind;
  double field;               /* CEF: E (Ha/bohr); V_app has slope -E on [0.1Lz, 0.9Lz]    */
  double dV, zA, zB;          /* CPD: phi_tilde = 0 for z <= zA, dV for z >= zB            */
  int has_patch;              /* L-CPD: restrict the z >= zB set to the patch below        */
  double patch_lo[2], patch_hi[2];
  double rtol;                /* relative residual target of the CG, e.g. 1e-10            */
  int max_iter;               /* CG iteration cap                                          */
} fe_poisson_bc;

typedef struct { int iters; double rel_residual; int status; } fe_solve_info;

/* Solve the Poisson problem with the bias setup in *bc (Eq. governing_equations CEF /
 * APD) by Jacobi-preconditioned CG on the matrix-free operator.
 *   rho_dev   electron density at phi nodes [n_phi], or NULL for the atoms' model density
 *             (fe_set_atoms is required in both cases for b and V_loc - V_sm).
 *   phi_dev   output potential phi at phi nodes [n_phi]; CEF: sum M phi = 0.
 *   vbare_dev optional output [n_psi]: phi + V_loc - V_sm + V_app at psi nodes, i.e. the
 *             V_eff of this library (Section 3.2 calls it V_bare).
 *   info      optional: iterations, final relative residual, status.
 * Returns FE_ENOCONV if max_iter is reached first, and FE_EINVAL (before any iteration)
 * when the initial residual is not finite: a NaN or infinity in rho, the atoms or the
 * constraint values. */
fe_status fe_poisson_solve(fe_mesh* mesh, const double* rho_dev, const fe_poisson_bc* bc,
                           double* phi_dev, double* vbare_dev, fe_solve_info* info);

/* V_bare = phi + (V_loc - V_sm) + V_app on every phi node (Section 3.3; V_app of the bias
 * for CEF, zero for CPD), out_dev [n_phi]. */
fe_status fe_vbare_phi(fe_mesh* mesh, const double* phi_dev, const fe_poisson_bc* bc,
                       double* out_dev);

/* Same solve for a given load f_dev [n_phi] (K phi = f on the free nodes) instead of
 * 4 pi M (rho + b).  CPD / L-CPD: constrained nodes take phic_dev [n_phi] (read on the
 * constrained set only), or the physical values -(V_loc - V_sm) / dV - (V_loc - V_sm) when
 * phic_dev is NULL.  CEF: the load is projected and sum M phi = 0 as above.  This is also
 * the adjoint solve: K is symmetric, so the gradient of a loss L(phi) with respect to f is
 * the solution for the load dL/dphi with zero constrained values. */
fe_status fe_poisson_solve_load(fe_mesh* mesh, const double* f_dev, const fe_poisson_bc* bc,
                                const double* phic_dev, double* phi_dev, fe_solve_info* info);

/* The constrained node set of bc (Eq. governing_equations APD; empty for CEF) as a byte
 * mask_dev [n_phi] (1 = constrained) and the physical constrained values values_dev
 * [n_phi] (-(V_loc - V_sm) on Omega_0, dV - (V_loc - V_sm) on Omega_1, 0 elsewhere). */
fe_status fe_poisson_constraints(fe_mesh* mesh, const fe_poisson_bc* bc, unsigned char* mask_dev,
                                 double* values_dev);

/* y = K x on phi nodes (Section 2.3), x, y [n_phi] doubles; no constraints applied. */
fe_status fe_poisson_apply_K(fe_mesh* mesh, const double* x_dev, double* y_dev);

/* The same product in float, x, y [n_phi] floats (distinct arrays, 4-byte aligned): the
 * operator of the float Poisson iterations.  Formed cell by cell (sum-factorised cell
 * products into a mesh-owned scratch of (p+1)^3 floats per cell, allocated on first use, then
 * a per-node sum of the cell copies in a fixed order), so repeated calls give identical bits.
 * FE_EINVAL for null or aliased arrays, FE_ENOMEM if the scratch cannot be allocated. */
fe_status fe_poisson_apply_K_f32(fe_mesh* mesh, const float* x_dev, float* y_dev);

/* Poisson load 4 pi M (rho + b) at phi nodes [n_phi] for the atoms (rho_dev NULL) or the
 * given density; f_dev [n_phi]; rho_out_dev / b_out_dev optional [n_phi] copies. */
fe_status fe_poisson_rhs(fe_mesh* mesh, const double* rho_dev, double* f_dev,
                         double* rho_out_dev, double* b_out_dev);

/* Rayleigh-Ritz of span(X) for Ht with orthonormal output: X <- X C with X^T X = I,
 * X^T Ht X = diag(eig), eig_dev[nvec] ascending Ritz values (Section 2.1 orthonormality).
 * Default: C from the Cholesky factor of the scaled Gram matrix and the projected matrix
 * (equivalent to Cholesky-QR then Rayleigh-Ritz); when the scaled Gram matrix is
 * ill-conditioned (cond above 1e8 with double products, 1e4 with tensor-core products)
 * the block is orthonormalised explicitly first (scaled Cholesky-QR2, shifted
 * Cholesky-QR3 on breakdown) in double.  The n x n factorisations and eigensolver are in
 * double; the three block products (Gram matrix, projected matrix, rotation) are double
 * GEMMs on a library-owned double copy of a float block, or, for float blocks with
 * FE_OPT_RR_PRODUCTS = FE_RR_PRODUCTS_TC32, FP32-accurate tensor-core GEMMs on the block
 * itself.  The one Ht X product runs in double for FE_F64 and in float (sum-factorised)
 * for the float-storage precisions.  Complex (Bloch) blocks: see fe_set_kpoint.
 * FE_EBREAKDOWN, with X unchanged, when a column of X is zero or not finite; FE_EBREAKDOWN
 * also when the shifted Cholesky-QR3 fallback cannot orthonormalise a rank-deficient block. */
fe_status fe_rayleigh_ritz(fe_mesh* mesh, void* X, int64_t nvec, int64_t ld, double* eig_dev,
                           fe_precision prec);

/* Copies of the atom fields at phi nodes [n_phi] (any output may be NULL): the model
 * density rho, the smeared nuclear charge b and V_loc - V_sm (see fe_set_atoms). */
fe_status fe_atom_fields(fe_mesh* mesh, double* rho_dev, double* b_dev, double* vlms_dev);

/* Electrostatic energy of the slab at fixed density for the potential phi_dev [n_phi]
 * returned by fe_poisson_solve with the same bc (Eq. electrostatics Energy, Eq. local
 * pseudopotential and the V_app term of Eq. KS DFT variational problem cef, lumped
 * quadrature; self energy excluded):
 *   E = c.phi - phi^T K phi / (8 pi) + sum M (V_loc - V_sm) rho + sum M (rho + b) V_app.
 * Because phi maximises E over the free nodes, the derivatives are explicit: *dE_dfield
 * (CEF, = -dipole when all charge lies on the linear part of V_app), *dE_ddV (CPD, the
 * reaction charge on Omega_1), and the node fields g_rho_dev, g_b_dev, g_vlms_dev [n_phi]
 * = dE/d rho, dE/d b, dE/d (V_loc - V_sm) for fe_atom_fields_vjp.  Synchronises. */
fe_status fe_energy(fe_mesh* mesh, const fe_poisson_bc* bc, const double* phi_dev, double* E_host,
                    double* dE_dfield_host, double* dE_ddV_host, double* g_rho_dev,
                    double* g_b_dev, double* g_vlms_dev);

/* Vector-Jacobian product of the atom fields with respect to the positions:
 * dR_host[a][k] = sum_I g_rho_I d rho_I / dR_ak + g_b_I d b_I / dR_ak
 *                 + g_vlms_I d (V_loc - V_sm)_I / dR_ak,
 * analytic, including the per-atom and global renormalisations of fe_set_atoms.
 * Synchronises. */
fe_status fe_atom_fields_vjp(fe_mesh* mesh, const double* g_rho_dev, const double* g_b_dev,
                             const double* g_vlms_dev, double* dR_host);

/* k-step Lanczos on Ht from the start vector v0_dev[n_psi] (Zhou & Li bounds):
 * *lo = smallest Ritz value, *hi = largest Ritz value + ||f_k||.  Synchronises.
 * FE_EINVAL for a zero or non-finite start vector; FE_EBREAKDOWN when the Krylov space
 * becomes invariant before the last step (beta_j <= 1e-10 of the largest alpha / beta so
 * far: v0 lies in an invariant subspace, and no bound of the whole spectrum follows). */
fe_status fe_lanczos_bounds(fe_mesh* mesh, const double* v0_dev, int steps, double* lo,
                            double* hi);

/* Number of this library's own CUDA kernels enqueued since it was loaded (replays of its
 * internal CUDA graphs included; cuBLAS / cuSOLVER kernels excluded).  Instrumentation for
 * benchmarks; process-wide, never reset. */
int64_t fe_kernel_launches(void);

/* Thread-local message describing the last non-FE_OK status on this thread. */
const char* fe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FE_H */

// Batched Hamiltonian application and Chebyshev filter over independent slabs.
//
// A bias sweep (Section 3: one slab geometry under a series of fields or potential
// differences, or slabs of several thicknesses) is a set of independent eigenproblems, each
// too small to fill the GPU alone.  A batch runs one operator kernel per Chebyshev step over
// every instance: the instances' CTA grids are concatenated into one 1D grid, and each
// instance keeps its own geometry, potential, block pointers and recurrence coefficients
// (alpha, beta, shift), read from a device array of per-instance descriptors.  The shared
// element coefficient table requires a common p and cell size.
//
// Launch configuration (autotuned): the work of one batched launch is the set of (instance,
// xy block, vector tile, z segment) items.  Two of its parameters decide how that work maps
// onto the GPU and are chosen per batch by timing: the z-segment length (cell layers per
// item: short segments give more, smaller items and better balance across slabs of uneven
// height, long ones amortise the halo planes each segment re-reads) and the grid form (one
// CTA per item, or a persistent grid of resident CTAs that take items from a device
// counter as they finish).  On the first batched operator call every candidate runs one
// operator launch on the batch's own blocks (into the filter's scratch block) and the
// fastest is kept; the choice is cached for the process per device, precision and batch
// shape, so later batches of the same shape skip the timing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fe_internal.h"

struct fe_batch {
  std::vector<fe_mesh*> meshes;
  int p = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  void* d_desc = nullptr;   // per-instance descriptors of the pending launches
  size_t desc_bytes = 0;
  void* d_rr = nullptr;     // n x n work of the batched Rayleigh-Ritz
  size_t rr_bytes = 0;
  std::vector<char> h_rr;   // host work of the batched eigensolver
  // launch configuration: z-segment length (0: occupancy heuristic), persistent grid
  int zseg = 0;
  int persistent = 0;
  bool configured = false;  // chosen by the tuner, taken from the cache, or set by the caller
  double tuned_ms = 0.0;    // the chosen candidate's launch time when timed here
  int ncand = 0;            // candidates timed for this batch (0: cache or caller)
  unsigned long long* d_counter = nullptr;   // work counter of the persistent grid
};

namespace {

int elem_bytes(fe_precision p) { return p == FE_F64 ? 8 : 4; }

fe_status grow_desc(fe_batch* b, size_t bytes) {
  if (b->desc_bytes >= bytes) return FE_OK;
  if (b->d_desc) {
    FE_CUDA(cudaStreamSynchronize(b->stream));
    FE_CUDA(cudaFree(b->d_desc));
    b->d_desc = nullptr;
    b->desc_bytes = 0;
  }
  if (cudaMalloc(&b->d_desc, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fe_fail(FE_ENOMEM, "batch descriptors of %zu bytes could not be allocated", bytes);
  }
  b->desc_bytes = bytes;
  return FE_OK;
}

fe_status check_blocks(const fe_batch* b, const void* const* X, const int64_t* nvec,
                       const int64_t* ld, fe_precision prec, const char* what) {
  if (!X || !nvec || !ld) return fe_fail(FE_EINVAL, "%s: null argument array", what);
  const int eb = elem_bytes(prec);
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    if (!X[i]) return fe_fail(FE_EINVAL, "%s: instance %zu: null block", what, i);
    if (nvec[i] < 1 || ld[i] < nvec[i])
      return fe_fail(FE_EINVAL, "%s: instance %zu: need 1 <= nvec <= ld", what, i);
    if (((uintptr_t)X[i]) % 16 != 0 || (ld[i] * eb) % 16 != 0)
      return fe_fail(FE_EINVAL, "%s: instance %zu: block must be 16-byte aligned and ld * %d "
                     "a multiple of 16", what, i, eb);
    if (!b->meshes[i]->has_potential)
      return fe_fail(FE_EINVAL, "%s: instance %zu: call fe_set_potential first", what, i);
    if (b->meshes[i]->has_quad || b->meshes[i]->has_k || b->meshes[i]->nl.natoms > 0)
      return fe_fail(FE_EUNSUPPORTED, "%s: instance %zu: batched operators take the Gamma-point "
                     "local operator with a collocated potential only", what, i);
  }
  return FE_OK;
}

// Fill one descriptor per instance for Y = alpha (Ht - shift) X + beta Z.
template <typename T>
void fill_io(const fe_batch* b, KronInst<T>* inst, const void* const* X, void* const* Y,
             const void* const* Z, const int64_t* nvec, const int64_t* ld,
             const double* alpha, const double* beta, const double* shift) {
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    const fe_mesh* m = b->meshes[i];
    KronIO<T>& io = inst[i].io;
    io.X = (const T*)X[i];
    io.ldx = ld[i];
    io.Y = (T*)Y[i];
    io.ldy = ld[i];
    io.Z = (Z && beta[i] != 0.0) ? (const T*)Z[i] : nullptr;
    io.ldz = ld[i];
    if constexpr (sizeof(T) == 8) io.V = (const T*)m->d_veff;
    else io.V = (const T*)m->d_veff_f;
    io.nvec = nvec[i];
    io.alpha = (T)alpha[i];
    io.beta = (T)beta[i];
    io.shift = (T)shift[i];
  }
}

template <typename T>
int64_t plan_with(const fe_batch* b, KronInst<T>* inst, int zseg) {
  const int n = (int)b->meshes.size();
  for (int i = 0; i < n; ++i) inst[i].g = fe_geom(b->meshes[i], true);
  if constexpr (sizeof(T) == 8) return fe::kron_batch_plan_f64(b->p, inst, n, zseg);
  else return fe::kron_batch_plan_f32(b->p, inst, n, zseg);
}

template <typename T>
int64_t plan(const fe_batch* b, KronInst<T>* inst) {
  return plan_with(b, inst, b->zseg);
}

fe_status ensure_counter(fe_batch* b) {
  if (b->d_counter) return FE_OK;
  if (cudaMalloc((void**)&b->d_counter, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    b->d_counter = nullptr;
    return fe_fail(FE_ENOMEM, "batch work counter could not be allocated");
  }
  return FE_OK;
}

template <typename T>
fe_status launch_with(fe_batch* b, const KronInst<T>* d_inst, int64_t total, bool use_z,
                      bool full, int persistent) {
  const int n = (int)b->meshes.size();
  unsigned long long* counter = nullptr;
  if (persistent) {
    FE_TRY(ensure_counter(b));
    counter = b->d_counter;
  }
  if constexpr (sizeof(T) == 8)
    return fe::kron_batch_f64(b->meshes[0]->coefH, b->p, d_inst, n, total, use_z, full, b->stream,
                              counter);
  else
    return fe::kron_batch_f32(b->meshes[0]->coefH, b->p, d_inst, n, total, use_z, full, b->stream,
                              counter);
}

template <typename T>
fe_status launch(fe_batch* b, const KronInst<T>* d_inst, int64_t total, bool use_z, bool full) {
  return launch_with(b, d_inst, total, use_z, full, b->persistent);
}

template <typename T>
bool all_full(const KronInst<T>* inst, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!inst[i].full) return false;
  return true;
}

// ---- autotuner --------------------------------------------------------------------------------
std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;   // shape key -> (zseg, persistent)

std::string tune_key(const fe_batch* b, int eb, const int64_t* nvec) {
  std::string k = std::to_string(b->device) + "|" + std::to_string(b->p) + "|" +
                  std::to_string(eb);
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    const fe_mesh* m = b->meshes[i];
    k += "|" + std::to_string(m->nx) + "," + std::to_string(m->ny) + "," +
         std::to_string(m->nz) + "," + std::to_string(m->NZs) + "," + std::to_string(nvec[i]);
  }
  return k;
}

// Time every candidate launch configuration on the batch's blocks (X -> the instances'
// filter scratch blocks W, which the caller owns for the duration) and keep the fastest.
template <typename T>
fe_status tune(fe_batch* b, const void* const* X, void* const* W, const int64_t* nvec,
               const int64_t* ld) {
  if (b->configured) return FE_OK;
  const std::string key = tune_key(b, (int)sizeof(T), nvec);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->zseg = it->second.first;
      b->persistent = it->second.second;
      b->configured = true;
      b->ncand = 0;
      return FE_OK;
    }
  }
  const size_t n = b->meshes.size();
  std::vector<KronInst<T>> inst(n);
  std::vector<double> one(n, 1.0), zero(n, 0.0);
  cudaEvent_t e0, e1;
  FE_CUDA(cudaEventCreate(&e0));
  FE_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int best_z = 0, best_p = 0, tried = 0;
  std::vector<int> resolved;
  fe_status st = FE_OK;
  for (int zreq : {0, 2, 4, 8, 16, 1 << 30}) {
    for (size_t i = 0; i < n; ++i) inst[i].io.nvec = nvec[i];
    const int64_t total = plan_with(b, inst.data(), zreq);
    const int zres = inst[0].g.zseg;
    if (std::find(resolved.begin(), resolved.end(), zres) != resolved.end()) continue;
    resolved.push_back(zres);
    fill_io(b, inst.data(), X, W, nullptr, nvec, ld, one.data(), zero.data(), zero.data());
    st = grow_desc(b, n * sizeof(KronInst<T>));
    if (st != FE_OK) break;
    if (cudaMemcpyAsync(b->d_desc, inst.data(), n * sizeof(KronInst<T>), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess) {
      cudaGetLastError();
      st = fe_fail(FE_ECUDA, "batch tuner: descriptor upload failed");
      break;
    }
    const bool full = all_full(inst.data(), n);
    for (int pers = 0; pers <= 1 && st == FE_OK; ++pers) {
      const KronInst<T>* d = (const KronInst<T>*)b->d_desc;
      st = launch_with(b, d, total, false, full, pers);   // warm-up
      if (st != FE_OK) break;
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 2 && st == FE_OK; ++r) st = launch_with(b, d, total, false, full, pers);
      cudaEventRecord(e1, b->stream);
      if (st != FE_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        st = fe_fail(FE_ECUDA, "batch tuner: timing failed");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ++tried;
      if (ms / 2.0 < best) {
        best = ms / 2.0;
        best_z = zreq == 0 ? 0 : zres;
        best_p = pers;
      }
    }
    if (st != FE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FE_TRY(st);
  b->zseg = best_z;
  b->persistent = best_p;
  b->tuned_ms = best;
  b->ncand = tried;
  b->configured = true;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = {best_z, best_p};
  return FE_OK;
}

template <typename T>
fe_status batch_apply(fe_batch* b, const void* const* X, void* const* Y, const int64_t* nvec,
                      const int64_t* ld) {
  const size_t n = b->meshes.size();
  FE_TRY(tune<T>(b, X, Y, nvec, ld));
  std::vector<KronInst<T>> inst(n);
  std::vector<double> one(n, 1.0), zero(n, 0.0);
  for (size_t i = 0; i < n; ++i) inst[i].io.nvec = nvec[i];
  const int64_t total = plan(b, inst.data());
  fill_io(b, inst.data(), X, Y, nullptr, nvec, ld, one.data(), zero.data(), zero.data());
  FE_TRY(grow_desc(b, n * sizeof(KronInst<T>)));
  FE_CUDA(cudaMemcpyAsync(b->d_desc, inst.data(), n * sizeof(KronInst<T>),
                          cudaMemcpyHostToDevice, b->stream));
  return launch(b, (const KronInst<T>*)b->d_desc, total, false, all_full(inst.data(), n));
}

// The recurrence of fe_cheb_filter, per instance, with every step one batched launch.  All
// descriptors (degree x n) are uploaded with one copy before the first step.
template <typename T>
fe_status batch_filter(fe_batch* b, void* const* X, const int64_t* nvec, const int64_t* ld,
                       int degree, const double* a, const double* bb, const double* a0) {
  const size_t n = b->meshes.size();
  const int eb = (int)sizeof(T);
  std::vector<void*> W(n);
  for (size_t i = 0; i < n; ++i)
    FE_TRY(fe_ws(b->meshes[i], WS_CHEB, (size_t)b->meshes[i]->n_psi * ld[i] * eb, &W[i]));
  FE_TRY(tune<T>(b, (const void* const*)X, W.data(), nvec, ld));
  std::vector<KronInst<T>> inst((size_t)degree * n);
  for (size_t i = 0; i < n; ++i) inst[i].io.nvec = nvec[i];
  const int64_t total = plan(b, inst.data());
  for (int s = 1; s < degree; ++s)
    for (size_t i = 0; i < n; ++i) inst[s * n + i] = inst[i];
  std::vector<double> e(n), c(n), sigma(n), tau(n), alpha(n), beta(n);
  for (size_t i = 0; i < n; ++i) {
    e[i] = (bb[i] - a[i]) / 2.0;
    c[i] = (bb[i] + a[i]) / 2.0;
    sigma[i] = e[i] / (a0[i] - c[i]);
    tau[i] = 2.0 / sigma[i];
    alpha[i] = sigma[i] / e[i];
    beta[i] = 0.0;
  }
  // step 1: W = (s1/e)(Ht - c) X
  std::vector<const void*> src(X, X + n);
  fill_io(b, inst.data(), src.data(), W.data(), nullptr, nvec, ld, alpha.data(), beta.data(),
          c.data());
  // later steps: Y_{k+1} overwrites Y_{k-1}; cur / prev alternate between W and X
  std::vector<void*> cur(W), prev(X, X + n);
  for (int s = 1; s < degree; ++s) {
    for (size_t i = 0; i < n; ++i) {
      const double sn = 1.0 / (tau[i] - sigma[i]);
      alpha[i] = 2.0 * sn / e[i];
      beta[i] = -sigma[i] * sn;
      sigma[i] = sn;
    }
    std::vector<const void*> xin(cur.begin(), cur.end()), zin(prev.begin(), prev.end());
    fill_io(b, inst.data() + s * n, xin.data(), prev.data(), zin.data(), nvec, ld,
            alpha.data(), beta.data(), c.data());
    std::swap(cur, prev);
  }
  const size_t bytes = inst.size() * sizeof(KronInst<T>);
  FE_TRY(grow_desc(b, bytes));
  FE_CUDA(cudaMemcpyAsync(b->d_desc, inst.data(), bytes, cudaMemcpyHostToDevice, b->stream));
  const KronInst<T>* d = (const KronInst<T>*)b->d_desc;
  const bool full = all_full(inst.data(), n);
  for (int s = 0; s < degree; ++s) FE_TRY(launch(b, d + s * n, total, s > 0, full));
  for (size_t i = 0; i < n; ++i)
    if (cur[i] != X[i])
      FE_CUDA(cudaMemcpy2DAsync(X[i], ld[i] * eb, cur[i], ld[i] * eb, nvec[i] * eb,
                                b->meshes[i]->n_psi, cudaMemcpyDeviceToDevice, b->stream));
  return FE_OK;
}

}  // namespace

extern "C" fe_status fe_batch_create(fe_mesh* const* meshes, int n, fe_batch** out) {
  if (!meshes || !out) return fe_fail(FE_EINVAL, "fe_batch_create: null argument");
  *out = nullptr;
  if (n < 1 || n > 65536) return fe_fail(FE_EINVAL, "fe_batch_create: need 1 <= n <= 65536");
  for (int i = 0; i < n; ++i)
    if (!meshes[i]) return fe_fail(FE_EINVAL, "fe_batch_create: mesh %d is null", i);
  const fe_mesh* m0 = meshes[0];
  for (int i = 0; i < n; ++i) {
    if (meshes[i]->nl.natoms > 0)
      return fe_fail(FE_EUNSUPPORTED, "fe_batch_create: mesh %d carries the nonlocal term", i);
    if (meshes[i]->has_k)
      return fe_fail(FE_EUNSUPPORTED, "fe_batch_create: mesh %d has a Bloch wave vector", i);
    if (meshes[i]->has_quad)
      return fe_fail(FE_EUNSUPPORTED, "fe_batch_create: mesh %d has a quadrature potential", i);
  }
  for (int i = 1; i < n; ++i) {
    const fe_mesh* m = meshes[i];
    if (m->device != m0->device || m->stream != m0->stream)
      return fe_fail(FE_EINVAL, "fe_batch_create: mesh %d is on another device or stream", i);
    if (m->p != m0->p || std::memcmp(&m->coefH, &m0->coefH, sizeof(KronCoef)) != 0)
      return fe_fail(FE_EUNSUPPORTED,
                     "fe_batch_create: mesh %d differs in p or cell size from mesh 0", i);
  }
  fe_batch* b = new fe_batch;
  b->meshes.assign(meshes, meshes + n);
  b->p = m0->p;
  b->device = m0->device;
  b->stream = m0->stream;
  *out = b;
  return FE_OK;
}

extern "C" fe_status fe_batch_destroy(fe_batch* b) {
  if (!b) return FE_OK;
  fe_status st = FE_OK;
  if (b->d_desc || b->d_rr || b->d_counter) {
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess ||
        (b->d_desc && cudaFree(b->d_desc) != cudaSuccess) ||
        (b->d_rr && cudaFree(b->d_rr) != cudaSuccess) ||
        (b->d_counter && cudaFree(b->d_counter) != cudaSuccess)) {
      cudaGetLastError();
      st = fe_fail(FE_ECUDA, "fe_batch_destroy: could not release the batch work arrays");
    }
  }
  delete b;
  return st;
}

extern "C" fe_status fe_batch_tuning(const fe_batch* b, int* zseg, int* persistent,
                                     double* best_ms, int* ncand) {
  if (!b || !zseg || !persistent || !best_ms || !ncand)
    return fe_fail(FE_EINVAL, "fe_batch_tuning: null argument");
  *zseg = b->zseg;
  *persistent = b->persistent;
  *best_ms = b->tuned_ms;
  *ncand = b->ncand;
  return b->configured ? FE_OK
                       : fe_fail(FE_EINVAL, "fe_batch_tuning: no batched operator call yet");
}

extern "C" fe_status fe_batch_set_launch(fe_batch* b, int zseg, int persistent) {
  if (!b) return fe_fail(FE_EINVAL, "fe_batch_set_launch: null batch");
  if (zseg < 0 || (persistent != 0 && persistent != 1))
    return fe_fail(FE_EINVAL, "fe_batch_set_launch: need zseg >= 0 and persistent 0 or 1");
  b->zseg = zseg;
  b->persistent = persistent;
  b->configured = true;
  b->tuned_ms = 0.0;
  b->ncand = 0;
  return FE_OK;
}

extern "C" fe_status fe_batch_apply_H(fe_batch* b, const void* const* X, void* const* Y,
                                      const int64_t* nvec, const int64_t* ld,
                                      fe_precision prec) {
  if (!b) return fe_fail(FE_EINVAL, "fe_batch_apply_H: null batch");
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_batch_apply_H: FE_F64 and FE_F32 only");
  FE_TRY(check_blocks(b, X, nvec, ld, prec, "fe_batch_apply_H"));
  FE_TRY(check_blocks(b, (const void* const*)Y, nvec, ld, prec, "fe_batch_apply_H"));
  const int eb = elem_bytes(prec);
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    const size_t bytes = (size_t)b->meshes[i]->n_psi * ld[i] * eb;
    const char *xs = (const char*)X[i], *ys = (const char*)Y[i];
    if (xs < ys + bytes && ys < xs + bytes)
      return fe_fail(FE_EINVAL, "fe_batch_apply_H: instance %zu: X and Y overlap", i);
  }
  FE_TRY(fe_activate(b->meshes[0]));
  return prec == FE_F64 ? batch_apply<double>(b, X, Y, nvec, ld)
                        : batch_apply<float>(b, X, Y, nvec, ld);
}

extern "C" fe_status fe_batch_cheb_filter(fe_batch* b, void* const* X, const int64_t* nvec,
                                          const int64_t* ld, int degree, const double* a,
                                          const double* bnd, const double* a0,
                                          fe_precision prec) {
  if (!b) return fe_fail(FE_EINVAL, "fe_batch_cheb_filter: null batch");
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_batch_cheb_filter: FE_F64 and FE_F32 only");
  if (degree < 1 || degree > 1000)
    return fe_fail(FE_EINVAL, "fe_batch_cheb_filter: degree must be in [1, 1000]");
  if (!a || !bnd || !a0) return fe_fail(FE_EINVAL, "fe_batch_cheb_filter: null bounds");
  FE_TRY(check_blocks(b, (const void* const*)X, nvec, ld, prec, "fe_batch_cheb_filter"));
  for (size_t i = 0; i < b->meshes.size(); ++i)
    if (!(a0[i] < a[i] && a[i] < bnd[i]) || !std::isfinite(a0[i]) || !std::isfinite(bnd[i]))
      return fe_fail(FE_EINVAL, "fe_batch_cheb_filter: instance %zu: need a0 < a < b", i);
  FE_TRY(fe_activate(b->meshes[0]));
  return prec == FE_F64 ? batch_filter<double>(b, X, nvec, ld, degree, a, bnd, a0)
                        : batch_filter<float>(b, X, nvec, ld, degree, a, bnd, a0);
}

// ---- batched Rayleigh-Ritz ---------------------------------------------------------------------
// Per instance the same steps as fe_rayleigh_ritz's Gram path: S = X^T X, H = X^T (Ht X), the
// scaled Gram matrix D S D = R^T R (Cholesky), G = R^-T (D H D) R^-1 = Q diag(eig) Q^T, and
// X <- X D R^-1 Q.  Ht X is one batched operator launch; the n x n steps are batched cuBLAS /
// cuSOLVER calls over all instances; only the block products run per instance.
namespace {

__global__ void k_b_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void k_b_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
// d = 1/sqrt(diag S) per matrix
__global__ void k_b_invsqrt_diag(const double* __restrict__ S, int n, int nb, double* __restrict__ d) {
  const int64_t tot = (int64_t)n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / n, j = t % n;
    const double v = S[b * n * n + j * n + j];
    d[t] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  }
}
// S <- D S D and H <- D sym(H) D (column-major n x n, both triangles)
__global__ void k_b_scale(double* __restrict__ S, double* __restrict__ H, const double* __restrict__ d,
                          int n, int nb) {
  const int64_t tot = (int64_t)n * n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / ((int64_t)n * n), r = t % ((int64_t)n * n);
    const int i = (int)(r % n), j = (int)(r / n);
    if (i > j) continue;   // one thread per unordered pair
    const double di = d[b * n + i], dj = d[b * n + j];
    double* Sb = S + b * n * n;
    double* Hb = H + b * n * n;
    const double s = 0.5 * (Sb[i + (int64_t)j * n] + Sb[j + (int64_t)i * n]) * di * dj;
    const double h = 0.5 * (Hb[i + (int64_t)j * n] + Hb[j + (int64_t)i * n]) * di * dj;
    Sb[i + (int64_t)j * n] = s;
    Sb[j + (int64_t)i * n] = s;
    Hb[i + (int64_t)j * n] = h;
    Hb[j + (int64_t)i * n] = h;
  }
}
__global__ void k_b_symm(double* __restrict__ G, int n, int nb) {
  const int64_t tot = (int64_t)n * n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / ((int64_t)n * n), r = t % ((int64_t)n * n);
    const int i = (int)(r % n), j = (int)(r / n);
    if (i >= j) continue;
    double* Gb = G + b * n * n;
    const double v = 0.5 * (Gb[i + (int64_t)j * n] + Gb[j + (int64_t)i * n]);
    Gb[i + (int64_t)j * n] = v;
    Gb[j + (int64_t)i * n] = v;
  }
}
// row i of every C scaled by d_i; the diagonal of every R into rd
__global__ void k_b_rowscale(double* __restrict__ C, const double* __restrict__ d, int n, int nb) {
  const int64_t tot = (int64_t)n * n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / ((int64_t)n * n), r = t % ((int64_t)n * n);
    C[t] *= d[b * n + (r % n)];
  }
}
__global__ void k_b_diag(const double* __restrict__ R, int n, int nb, double* __restrict__ rd) {
  const int64_t tot = (int64_t)n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / n, j = t % n;
    rd[t] = R[b * n * n + j * n + j];
  }
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

extern "C" fe_status fe_batch_rayleigh_ritz(fe_batch* b, void* const* X, int64_t nvec,
                                            const int64_t* ld, double* const* eig,
                                            fe_precision prec) {
  if (!b || !eig) return fe_fail(FE_EINVAL, "fe_batch_rayleigh_ritz: null argument");
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED, "fe_batch_rayleigh_ritz: FE_F64 and FE_F32 only");
  const int nb = (int)b->meshes.size();
  if (prec == FE_F32)
    for (int i = 0; i < nb; ++i)
      if (b->meshes[i]->rr_products != FE_RR_PRODUCTS_TC32)
        return fe_fail(FE_EUNSUPPORTED, "fe_batch_rayleigh_ritz: float blocks need the tensor-core "
                       "block products (FE_OPT_RR_PRODUCTS = FE_RR_PRODUCTS_TC32) on every mesh");
  if (nvec < 1 || nvec > 4096) return fe_fail(FE_EINVAL, "fe_batch_rayleigh_ritz: need 1 <= nvec <= 4096");
  std::vector<int64_t> nv(nb, nvec);
  FE_TRY(check_blocks(b, (const void* const*)X, nv.data(), ld, prec, "fe_batch_rayleigh_ritz"));
  for (int i = 0; i < nb; ++i) {
    if (!eig[i]) return fe_fail(FE_EINVAL, "fe_batch_rayleigh_ritz: instance %d: null eig", i);
    if (nvec > b->meshes[i]->n_psi)
      return fe_fail(FE_EINVAL, "fe_batch_rayleigh_ritz: instance %d: nvec exceeds the node count", i);
  }
  FE_TRY(fe_activate(b->meshes[0]));
  fe_mesh* m0 = b->meshes[0];
  cudaStream_t st = b->stream;
  const int n = (int)nvec;
  const int64_t nn = (int64_t)n * n;
  const int eb = prec == FE_F64 ? 8 : 4;

  // Ht X of every instance (one launch), into each mesh's workspace: [HX | rotation tmp]
  std::vector<void*> hx(nb), tmp(nb);
  for (int i = 0; i < nb; ++i) {
    void* w;
    const size_t blk = (size_t)b->meshes[i]->n_psi * ld[i] * eb;
    FE_TRY(fe_ws(b->meshes[i], WS_RR_HX, 2 * blk, &w));
    hx[i] = w;
    tmp[i] = (char*)w + blk;
  }
  if (prec == FE_F64) FE_TRY(batch_apply<double>(b, X, hx.data(), nv.data(), ld));
  else FE_TRY(batch_apply<float>(b, X, hx.data(), nv.data(), ld));

  // batch work: S, H (double), Sf, Hf (float), d, W, R diagonals, pointer arrays, infos
  size_t bytes = sizeof(double) * (2 * nn * nb + 3 * (size_t)n * nb) + sizeof(float) * 2 * nn * nb +
                 sizeof(double*) * 2 * nb + sizeof(int) * 2 * nb + 1024;
  size_t dev_syev = 0, host_syev = 0;
  cusolverDnParams_t params = nullptr;
  FE_CUSOLVER(cusolverDnCreateParams(&params));
  struct ParamsGuard { cusolverDnParams_t p; ~ParamsGuard() { if (p) cusolverDnDestroyParams(p); } } pg{params};
  FE_CUSOLVER(cusolverDnXsyevBatched_bufferSize(m0->cusolver, params, CUSOLVER_EIG_MODE_VECTOR,
                                                CUBLAS_FILL_MODE_UPPER, n, CUDA_R_64F, nullptr, n,
                                                CUDA_R_64F, nullptr, CUDA_R_64F, &dev_syev,
                                                &host_syev, nb));
  bytes += dev_syev + 256;
  if (b->rr_bytes < bytes) {
    if (b->d_rr) {
      FE_CUDA(cudaStreamSynchronize(st));
      FE_CUDA(cudaFree(b->d_rr));
      b->d_rr = nullptr;
      b->rr_bytes = 0;
    }
    if (cudaMalloc(&b->d_rr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ENOMEM, "batched Rayleigh-Ritz work of %zu bytes could not be allocated", bytes);
    }
    b->rr_bytes = bytes;
  }
  if (b->h_rr.size() < host_syev + 1) b->h_rr.resize(host_syev + 1);
  double* S = (double*)b->d_rr;
  double* H = S + nn * nb;
  double* d = H + nn * nb;
  double* W = d + (size_t)n * nb;
  double* rd = W + (size_t)n * nb;
  float* Sf = (float*)(rd + (size_t)n * nb);
  float* Hf = Sf + nn * nb;
  double** pS = (double**)(((uintptr_t)(Hf + nn * nb) + 15) & ~(uintptr_t)15);
  double** pH = pS + nb;
  int* info = (int*)(pH + nb);
  void* syev_ws = (void*)(((uintptr_t)(info + 2 * nb) + 255) & ~(uintptr_t)255);
  std::vector<double*> hS(nb), hH(nb);
  for (int i = 0; i < nb; ++i) { hS[i] = S + nn * i; hH[i] = H + nn * i; }
  FE_CUDA(cudaMemcpyAsync(pS, hS.data(), sizeof(double*) * nb, cudaMemcpyHostToDevice, st));
  FE_CUDA(cudaMemcpyAsync(pH, hH.data(), sizeof(double*) * nb, cudaMemcpyHostToDevice, st));

  FiniteEmulationGuard finite(m0->cublas);
  // block products
  for (int i = 0; i < nb; ++i) {
    const int N = (int)b->meshes[i]->n_psi;
    if (prec == FE_F64) {
      const double one = 1.0, zero = 0.0;
      FE_CUBLAS(cublasDgemm(m0->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, (const double*)X[i],
                            (int)ld[i], (const double*)X[i], (int)ld[i], &zero, hS[i], n));
      FE_CUBLAS(cublasDgemm(m0->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, (const double*)X[i],
                            (int)ld[i], (const double*)hx[i], (int)ld[i], &zero, hH[i], n));
    } else {
      const float one = 1.0f, zero = 0.0f;
      const cublasComputeType_t ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
      FE_CUBLAS(cublasGemmEx(m0->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, X[i], CUDA_R_32F,
                             (int)ld[i], X[i], CUDA_R_32F, (int)ld[i], &zero, Sf + nn * i, CUDA_R_32F,
                             n, ct, CUBLAS_GEMM_DEFAULT));
      FE_CUBLAS(cublasGemmEx(m0->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, N, &one, X[i], CUDA_R_32F,
                             (int)ld[i], hx[i], CUDA_R_32F, (int)ld[i], &zero, Hf + nn * i, CUDA_R_32F,
                             n, ct, CUBLAS_GEMM_DEFAULT));
    }
  }
  const int64_t tot = nn * nb;
  if (prec == FE_F32) {
    k_b_f2d<<<grid_of(tot), 256, 0, st>>>(Sf, S, tot); fe_count_launch();
    k_b_f2d<<<grid_of(tot), 256, 0, st>>>(Hf, H, tot); fe_count_launch();
  }
  k_b_invsqrt_diag<<<grid_of((int64_t)n * nb), 256, 0, st>>>(S, n, nb, d); fe_count_launch();
  k_b_scale<<<grid_of(tot), 256, 0, st>>>(S, H, d, n, nb); fe_count_launch();
  FE_CUSOLVER(cusolverDnDpotrfBatched(m0->cusolver, CUBLAS_FILL_MODE_UPPER, n, pS, n, info, nb));
  k_b_diag<<<grid_of((int64_t)n * nb), 256, 0, st>>>(S, n, nb, rd); fe_count_launch();
  std::vector<int> hinfo(nb);
  std::vector<double> hrd((size_t)n * nb);
  FE_CUDA(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaMemcpyAsync(hrd.data(), rd, sizeof(double) * n * nb, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  // an instance whose scaled Gram matrix is not safely positive definite is redone alone
  std::vector<char> ill(nb, 0);
  for (int i = 0; i < nb; ++i) {
    double rmax = 0.0, rmin = 1e300;
    for (int j = 0; j < n; ++j) {
      rmax = std::fmax(rmax, std::fabs(hrd[(size_t)i * n + j]));
      rmin = std::fmin(rmin, std::fabs(hrd[(size_t)i * n + j]));
    }
    ill[i] = hinfo[i] != 0 || !(rmin > 0.0) ||
             (rmax / rmin) * (rmax / rmin) > (prec == FE_F32 ? kGramCondTC32 : kGramCondF64);
  }
  const double one = 1.0;
  // G = R^-T H R^-1
  FE_CUBLAS(cublasDtrsmBatched(m0->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                               CUBLAS_DIAG_NON_UNIT, n, n, &one, pS, n, pH, n, nb));
  FE_CUBLAS(cublasDtrsmBatched(m0->cublas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                               CUBLAS_DIAG_NON_UNIT, n, n, &one, pS, n, pH, n, nb));
  k_b_symm<<<grid_of(tot), 256, 0, st>>>(H, n, nb); fe_count_launch();
  FE_CUSOLVER(cusolverDnXsyevBatched(m0->cusolver, params, CUSOLVER_EIG_MODE_VECTOR,
                                     CUBLAS_FILL_MODE_UPPER, n, CUDA_R_64F, H, n, CUDA_R_64F, W,
                                     CUDA_R_64F, syev_ws, dev_syev, b->h_rr.data(), host_syev,
                                     info + nb, nb));
  // C = D R^-1 Q
  FE_CUBLAS(cublasDtrsmBatched(m0->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                               CUBLAS_DIAG_NON_UNIT, n, n, &one, pS, n, pH, n, nb));
  k_b_rowscale<<<grid_of(tot), 256, 0, st>>>(H, d, n, nb); fe_count_launch();
  if (prec == FE_F32) { k_b_d2f<<<grid_of(tot), 256, 0, st>>>(H, Hf, tot); fe_count_launch(); }
  FE_CUDA(cudaGetLastError());
  // X <- X C and the Ritz values, for the well-conditioned instances
  for (int i = 0; i < nb; ++i) {
    if (ill[i]) continue;
    const int N = (int)b->meshes[i]->n_psi;
    if (prec == FE_F64) {
      const double zero = 0.0;
      FE_CUBLAS(cublasDgemm(m0->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, N, n, &one, hH[i], n,
                            (const double*)X[i], (int)ld[i], &zero, (double*)tmp[i], (int)ld[i]));
    } else {
      const float onef = 1.0f, zerof = 0.0f;
      FE_CUBLAS(cublasGemmEx(m0->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, N, n, &onef, Hf + nn * i,
                             CUDA_R_32F, n, X[i], CUDA_R_32F, (int)ld[i], &zerof, tmp[i], CUDA_R_32F,
                             (int)ld[i], CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT));
    }
    FE_CUDA(cudaMemcpy2DAsync(X[i], ld[i] * eb, tmp[i], ld[i] * eb, (size_t)n * eb, N,
                              cudaMemcpyDeviceToDevice, st));
    FE_CUDA(cudaMemcpyAsync(eig[i], W + (size_t)i * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  }
  FE_CUDA(cudaMemcpyAsync(hinfo.data(), info + nb, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < nb; ++i)
    if (!ill[i] && hinfo[i] != 0)
      return fe_fail(FE_ECUDA, "fe_batch_rayleigh_ritz: instance %d: eigensolver info %d", i, hinfo[i]);
  for (int i = 0; i < nb; ++i)
    if (ill[i]) FE_TRY(fe_rayleigh_ritz(b->meshes[i], X[i], nvec, ld[i], eig[i], prec));
  return FE_OK;
}

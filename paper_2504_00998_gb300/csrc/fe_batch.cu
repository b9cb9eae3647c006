// Batched Hamiltonian application and Chebyshev filter over independent slabs.
//
// A bias sweep (Section 3: one slab geometry under a series of fields or potential
// differences, or slabs of several thicknesses) is a set of independent eigenproblems, each
// too small to fill the GPU alone.  A batch runs one operator kernel per Chebyshev step over
// every instance: the instances' CTA grids are concatenated into one 1D grid, and each
// instance keeps its own geometry, potential, block pointers and recurrence coefficients
// (alpha, beta, shift), read from a device array of per-instance descriptors.  The shared
// element coefficient table requires a common p and cell size.
#include <cmath>
#include <cstring>
#include <vector>

#include "fe_internal.h"

struct fe_batch {
  std::vector<fe_mesh*> meshes;
  int p = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  void* d_desc = nullptr;   // per-instance descriptors of the pending launches
  size_t desc_bytes = 0;
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
int64_t plan(const fe_batch* b, KronInst<T>* inst) {
  const int n = (int)b->meshes.size();
  for (int i = 0; i < n; ++i) inst[i].g = fe_geom(b->meshes[i], true);
  if constexpr (sizeof(T) == 8) return fe::kron_batch_plan_f64(b->p, inst, n);
  else return fe::kron_batch_plan_f32(b->p, inst, n);
}

template <typename T>
fe_status launch(const fe_batch* b, const KronInst<T>* d_inst, int64_t total, bool use_z) {
  const int n = (int)b->meshes.size();
  if constexpr (sizeof(T) == 8)
    return fe::kron_batch_f64(b->meshes[0]->coefH, b->p, d_inst, n, total, use_z, b->stream);
  else
    return fe::kron_batch_f32(b->meshes[0]->coefH, b->p, d_inst, n, total, use_z, b->stream);
}

template <typename T>
fe_status batch_apply(fe_batch* b, const void* const* X, void* const* Y, const int64_t* nvec,
                      const int64_t* ld) {
  const size_t n = b->meshes.size();
  std::vector<KronInst<T>> inst(n);
  std::vector<double> one(n, 1.0), zero(n, 0.0);
  for (size_t i = 0; i < n; ++i) inst[i].io.nvec = nvec[i];
  const int64_t total = plan(b, inst.data());
  fill_io(b, inst.data(), X, Y, nullptr, nvec, ld, one.data(), zero.data(), zero.data());
  FE_TRY(grow_desc(b, n * sizeof(KronInst<T>)));
  FE_CUDA(cudaMemcpyAsync(b->d_desc, inst.data(), n * sizeof(KronInst<T>),
                          cudaMemcpyHostToDevice, b->stream));
  return launch(b, (const KronInst<T>*)b->d_desc, total, false);
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
  for (int s = 0; s < degree; ++s) FE_TRY(launch(b, d + s * n, total, s > 0));
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
  if (b->d_desc) {
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess ||
        cudaFree(b->d_desc) != cudaSuccess) {
      cudaGetLastError();
      st = fe_fail(FE_ECUDA, "fe_batch_destroy: could not release the descriptors");
    }
  }
  delete b;
  return st;
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

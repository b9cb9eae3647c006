// Chebyshev filter variant that allocates no device memory.
//
// fe_cheb_filter needs one scratch block of X's size for the three-term recurrence and
// takes it from a workspace that the library allocates with cudaMalloc on first use.  Some
// callers cannot let a library allocate: a process whose framework allocator has already
// reserved the free device memory (a cudaMalloc would fail or fragment its pool), a
// service that must keep a fixed per-process memory budget after start-up, or a
// latency-sensitive loop where cudaMalloc's implicit device synchronisation would stall
// the other streams.  For them, fe_cheb_filter_static keeps the scratch in the file-scope
// array below instead.  The array is part of the module, so every device that loads this
// library holds it until the process exits.
#include <cmath>
#include <mutex>

#include "fe_internal.h"

#define FE_STATIC_SCRATCH_BYTES (64ull << 20)  // 64 MiB

// Device-side scratch of the allocation-free filter.  Host code must not pass this name to
// a kernel: on the host it is only a stand-in for the symbol, not a device address.
static __device__ __align__(256) unsigned char fe_static_scratch[FE_STATIC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// device address of the scratch array on the current device, looked up once per device and
// kept for the life of the process (like every other piece of this library's device state,
// it does not survive cudaDeviceReset)
fe_status scratch_address(int device, void** out) {
  if (device < 0 || device >= MAX_DEVICES)
    return fe_fail(FE_EINVAL, "fe_cheb_filter_static: device ordinal %d out of range", device);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, fe_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fe_fail(FE_ECUDA, "fe_cheb_filter_static: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return FE_OK;
}

}  // namespace

extern "C" fe_status fe_cheb_filter_static(fe_mesh* m, void* X, int64_t nvec, int64_t ld,
                                           int degree, double a, double b, double a0,
                                           fe_precision prec) {
  if (!m || !X) return fe_fail(FE_EINVAL, "fe_cheb_filter_static: null argument");
  if (m->has_k)
    return fe_fail(FE_EUNSUPPORTED, "fe_cheb_filter_static: Gamma-point blocks only");
  if (prec != FE_F64 && prec != FE_F32)
    return fe_fail(FE_EUNSUPPORTED,
                   "fe_cheb_filter_static: only FE_F64 and FE_F32 run without allocation");
  const int eb = prec == FE_F64 ? 8 : 4;
  if (nvec < 1 || ld < nvec) return fe_fail(FE_EINVAL, "fe_cheb_filter_static: need 1 <= nvec <= ld");
  if (((uintptr_t)X) % 16 != 0 || (ld * eb) % 16 != 0)
    return fe_fail(FE_EINVAL, "fe_cheb_filter_static: X must be 16-byte aligned and ld * %d a "
                   "multiple of 16", eb);
  if (degree < 1) return fe_fail(FE_EINVAL, "fe_cheb_filter_static: degree must be >= 1");
  if (!(a0 < a && a < b) || !std::isfinite(a0) || !std::isfinite(b))
    return fe_fail(FE_EINVAL, "fe_cheb_filter_static: need finite a0 < a < b");
  if (!m->has_potential)
    return fe_fail(FE_EINVAL, "fe_cheb_filter_static: call fe_set_potential first");
  if (m->nl.natoms > 0)
    return fe_fail(FE_EUNSUPPORTED, "fe_cheb_filter_static: the nonlocal term needs a workspace");
  const unsigned long long need = (unsigned long long)m->n_psi * (unsigned long long)ld * eb;
  if (need > FE_STATIC_SCRATCH_BYTES)
    return fe_fail(FE_EINVAL,
                   "fe_cheb_filter_static: block needs %llu bytes of scratch (n_psi * ld * %d), "
                   "above the %llu-byte static limit; use fe_cheb_filter",
                   need, eb, (unsigned long long)FE_STATIC_SCRATCH_BYTES);
  FE_TRY(fe_activate(m));
  void* W = nullptr;
  FE_TRY(scratch_address(m->device, &W));
  // same recurrence as fe_cheb_filter; the scratch is written by the first step before it
  // is read, so its previous contents never matter
  const double e = (b - a) / 2.0, c = (b + a) / 2.0;
  double sigma = e / (a0 - c);
  const double tau = 2.0 / sigma;
  FE_TRY(fe_hx_step(m, X, W, nullptr, nvec, ld, sigma / e, 0.0, c, prec));
  void* cur = W;
  void* prev = X;
  for (int i = 2; i <= degree; ++i) {
    const double sn = 1.0 / (tau - sigma);
    FE_TRY(fe_hx_step(m, cur, prev, prev, nvec, ld, 2.0 * sn / e, -sigma * sn, c, prec));
    void* t = cur;
    cur = prev;
    prev = t;
    sigma = sn;
  }
  if (cur != X)
    FE_CUDA(cudaMemcpy2DAsync(X, ld * eb, cur, ld * eb, nvec * eb, m->n_psi,
                              cudaMemcpyDeviceToDevice, m->stream));
  return FE_OK;
}

// Persistent float conjugate-gradient iteration of the Poisson solve (Section 2.3): the whole
// preconditioned iteration (cell-local stiffness product, node sums, the two dot products,
// the x / r update, the z-plane coarse correction, the Jacobi preconditioner and the
// direction update) runs in one cooperative launch, its steps separated by grid-wide
// barriers instead of kernel boundaries.  The vectors of one solve (a few tens of MB at the
// benchmark sizes) stay in L2 between the steps.
//
// Layout: two large blocks per SM.  A block is NG groups of CellStrip<P>::NTHR threads (as
// many as fit in 1024); in the cell step every group contracts its own strip of cells with
// its own shared arrays and a named barrier, and in the vector steps the block's threads
// share one contiguous range of nodes (groups of four; the range spans at most MAXSPAN phi
// planes).
//
// One iteration, three barriers:
//   1. cell products y_e = K_e p_e of the search direction into the discontinuous grid;
//      after the first iteration of a launch p is not yet stored: every staged node forms
//      p = z + beta p_old itself (the same single rounding its owner uses in step 2);
//   2. q = sum of the cell copies per node, the owners store the new p, p.q partials, and
//      the sums of q over the free nodes against each coarse function of the planes in the
//      block's range (the plane indicator; with the mode coarse space also the eight
//      in-plane modes); the block completing the barrier publishes alpha = r.z / p.q and
//      the coarse right-hand sides of the new residual r - alpha q, carried by recurrence:
//      b(r - alpha q) = b(r) - alpha b(q), with b(r) summed exactly from r in a launch's
//      first iteration (a launch starts after every reliable update, so the recurrence
//      never runs long); under the CEF projection it also publishes the new residual's
//      mean and subtracts mean * cnt_k from the indicator's right-hand side;
//   3. the coarse values of the block's planes (a row of the coarse inverse times the
//      right-hand side, one warp per plane and function), then in one pass x += alpha p,
//      r -= alpha q on free nodes, r -= mean (CEF), z = Dinv r plus the prolongation of the
//      coarse values on free nodes, r.z and r.r partials; the completing block publishes
//      beta, r.z, r.r, the iteration count and the convergence test.
// Every grid sum is taken over the block partials in index order by whichever block
// completes the barrier (the same code and order whichever it is), so results do not depend
// on scheduling.  Dot products keep the launch-per-step path's precision: a thread's terms
// in float, block and grid sums in double (float pairs within a warp).  The mode functions'
// sums and their coarse solves are in float: they only have to be a fixed linear map.
//
// The grid is co-resident by construction (cooperative launch sized from the occupancy
// calculator).  Every barrier wait is bounded (2 s): a block that gives up sets the state's
// fused_err and returns, and a block that sees the flag while waiting returns too, so a
// failure ends the launch with an error the host reads instead of a hang.
#include <algorithm>
#include <cstdint>

#include "fe_cg.cuh"
#include "fe_internal.h"
#include "fe_kcell.cuh"

namespace {

using fe_cg::CgState;
using fe_kc::CellCoef;
using fe_kc::CellStrip;

constexpr long long BAR_TIMEOUT_NS = 2000000000LL;
constexpr int BLOCKS_PER_SM = 2;
// planes that the nodes of one block may span (the host falls back to the launch-per-step
// iteration beyond this)
constexpr int MAXSPAN = 4;
// coarse functions per plane with the in-plane modes (the indicator and fe_cg::MODES_NM - 1
// modes)
constexpr int MODES_NM = fe_cg::MODES_NM;

// threads of a block: NG strip groups of GT threads
template <int P>
struct FusedShape {
  static constexpr int GT = CellStrip<P>::NTHR;
  static constexpr int NG = 1024 / GT;
  static constexpr int NT = NG * GT;
  // shared floats of one group (U, A, B), a multiple of four so every group stays 16-byte
  // aligned
  static constexpr int GROUP_FLOATS =
      (CellStrip<P>::U_FLOATS + 2 * CellStrip<P>::A_FLOATS + 3) / 4 * 4;
};

// dynamic shared memory of a block: the coarse right-hand side of the plane indicators [nzp]
// (doubles) and (NM > 1) of the modes [NM - 1][nzp] (floats), the mode tables (cos x, sin x
// [NX], cos y, sin y [NY], floats), then from byte offset group_offset() the strip groups'
// U, A, B
// (the tables start on a 16-byte boundary: they are read four entries at a time)
__host__ __device__ inline size_t table_offset(int NM, int nzp) {
  return (sizeof(double) * (size_t)nzp + sizeof(float) * (size_t)(NM - 1) * nzp + 15) / 16 * 16;
}
template <int NM>
inline size_t group_offset(int nzp, int NX, int NY) {
  size_t b = table_offset(NM, nzp);
  if (NM > 1) b += sizeof(float) * 2 * ((size_t)NX + NY);
  return (b + 15) / 16 * 16;
}
template <int P, int NM>
inline size_t fused_smem(int nzp, int NX, int NY) {
  return group_offset<NM>(nzp, NX, NY) + sizeof(float) * (size_t)FusedShape<P>::NG *
                                             FusedShape<P>::GROUP_FLOATS;
}

// grid-wide results published by the block that completes a barrier
struct __align__(16) Pub {
  double pq, alpha, mean, rz, rr, beta;
  int iters, done;
  float alphaf, meanf, betaf;   // the float values the vector steps use
  int stop;                     // the launch ends after this iteration
};
static_assert(sizeof(Pub) % 16 == 0 && sizeof(Pub) <= 32 * 16, "Pub is copied as 16-byte words");

struct FArgs {
  float *x, *r, *z, *p, *q, *ycell;
  const float* dinv;
  const unsigned char* mask;
  const double* Ainv;
  const double* cnt;
  double* part;               // [3][G]: p.q, r.z and r.r block partials
  double* seg;                // [G][MAXSPAN][NM]: sums of q against the coarse functions of
                              // the planes of each block's nodes (free nodes)
  double* seg_r;              // the same for r (a launch's first iteration)
  double* bprev;              // [NM][nzp]: the coarse right-hand sides of the current r
  double* cbg;                // [nzp]: the coarse right-hand side of the current iteration
  Pub* pub;
  unsigned int* bar;          // [0]: arrivals, [32]: barriers released (0 at launch)
  CgState* s;
  int nx, ny, nz, NX, NY, nzp;
  uint32_t chunk4;            // groups of four nodes per block
  int project;
  double inv_n;
  int nit, iters_stop;
  double rr_lo, rr_hi;
  int stall;                  // test aid: this block leaves before the first barrier (-1: none)
  const float* Amodes;        // (NM > 1) mode coarse inverses [NM - 1][nzp][nzp], float
  float* cbgf;                // (NM > 1) the modes' coarse right-hand sides [NM - 1][nzp]
  const float* mtab;          // (NM > 1) mode tables: cos x, sin x [NX]; cos y, sin y [NY]
  unsigned int grp_off;       // byte offset of the strip groups in dynamic shared memory
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* a, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* a, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier number k (1, 2, ... within the launch).  Each block's thread 0 adds the
// block's arrival; the block that arrives last runs fin() with all its threads (it sees every
// write made before the barrier), then releases the barrier by publishing k; the other
// blocks wait for the release.  Warp 0 then copies the published results into the block's
// shared copy (one read of that line per block, not per thread) unless the barrier
// publishes nothing (copy false).  Returns false in every
// thread of the block when the wait gave up (a peer failed, or 2 s passed).
template <class Fin>
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err, unsigned int k,
                                             const Pub* pub, Pub* spub, Fin fin,
                                             bool copy = true) {
  __shared__ int role;   // 1: completes the barrier, 0: waits, -1: gave up
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the block's writes before the barrier (ordered by the block barrier above);
    // acquire: the completing block then sees every block's writes
    const unsigned int old = atom_add_acq_rel_u32(bar, 1u);
    role = old == k * gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (role == 1) {
    fin();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_u32(bar + 32, k);
    }
  } else if (threadIdx.x == 0) {
    const long long t0 = global_ns();
    unsigned int spins = 0;
    while (ld_acquire_u32(bar + 32) < k) {
      if ((spins & 15u) == 15u && *(volatile int*)err != 0) { role = -1; break; }
      if (++spins > (1u << 26) || global_ns() - t0 > BAR_TIMEOUT_NS) {
        atomicExch(err, 1);
        role = -1;
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();   // the release has been seen (or the wait gave up)
  if (!copy) return role >= 0;
  if (threadIdx.x < (int)(sizeof(Pub) / 16) && role >= 0) {
    // 16-byte words, one per thread of warp 0, in one round trip
    reinterpret_cast<int4*>(spub)[threadIdx.x] = __ldcg(reinterpret_cast<const int4*>(pub) + threadIdx.x);
  }
  __syncthreads();
  return role >= 0;
}

// Reductions.  FP64 throughput is a small fraction of FP32 on this GPU, so a block-wide
// shuffle tree in double costs microseconds per value; these keep double arithmetic to one
// warp.  Every order is fixed, so results do not depend on scheduling.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// a float pair (hi + lo, |lo| <= ulp(hi) / 2) summed with Knuth's TwoSum and renormalised:
// about 48 significant bits
struct FPair {
  float hi, lo;
};
__device__ __forceinline__ FPair pair_add(FPair a, FPair b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float t = e + (a.lo + b.lo);
  const float h = s + t;
  return {h, t - (h - s)};
}
// block sums of float terms: float-pair sums within each warp (the warp's pair to shared
// memory), then warp 0 alone converts the pairs and adds them in double (the double
// instructions of one warp instead of every warp's).  The N totals land in out[0..N) of
// shared memory (read them after the trailing barrier).  sh holds N * 64 floats.
template <int N>
__device__ __forceinline__ void block_sum_f(const float (&v)[N], double* out, float* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    FPair d{v[j], 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const FPair t{__shfl_down_sync(0xffffffffu, d.hi, o), __shfl_down_sync(0xffffffffu, d.lo, o)};
      d = pair_add(d, t);
    }
    if (lane == 0) {
      sh[(j * 32 + w) * 2] = d.hi;
      sh[(j * 32 + w) * 2 + 1] = d.lo;
    }
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double t = 0.0;
      if (lane < nw) t = (double)sh[(j * 32 + lane) * 2] + (double)sh[(j * 32 + lane) * 2 + 1];
      t = warp_sum_d(t);
      if (lane == 0) out[j] = t;
    }
  }
  __syncthreads();
}
// block sums of float terms in float (every thread reads out[0..N) after the trailing
// barrier): a shuffle tree in each warp, then warp 0 adds the warp totals the same way; for
// sums that only have to be a fixed linear function of their terms.  sh holds N * 32 floats.
template <int N>
__device__ __forceinline__ void block_sum_plain(const float (&v)[N], float* out, float* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float d = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane == 0) sh[j * 32 + w] = d;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float t = lane < nw ? sh[j * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) out[j] = t;
    }
  }
  __syncthreads();
}

// sums of the n doubles part[j * stride + i] (i < n) for j < N, by warp 0 (lane l takes
// i = l, l + 32, ... in order, then a shuffle tree); every thread receives them.  part is
// global memory (read through L2: other blocks wrote it) unless SHARED.  sh holds N doubles.
template <int N, bool SHARED = false>
__device__ __forceinline__ void sum_parts(const double* part, int64_t stride, int n,
                                          double (&out)[N], double* sh) {
  if (threadIdx.x < 32) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double t = 0.0;
      for (int i = threadIdx.x; i < n; i += 32)
        t += SHARED ? part[j * stride + i] : __ldcg(part + j * stride + i);
      t = warp_sum_d(t);
      if (threadIdx.x == 0) sh[j] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) out[j] = sh[j];
  __syncthreads();
}

__device__ __forceinline__ float4 ldcg4(const float4* a) { return __ldcg(a); }
__device__ __forceinline__ float sum4(const float4& a) { return a.x + a.y + a.z + a.w; }

// v[s] += t for the register slot s (0 <= s < N) without local-memory indexing
template <int N>
__device__ __forceinline__ void add_slot(float (&v)[N], int s, float t) {
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j == s) v[j] += t;
}
template <int N>
__device__ __forceinline__ float pick_slot(const float (&v)[N], int s) {
  float r = v[0];
#pragma unroll
  for (int j = 1; j < N; ++j)
    if (j == s) r = v[j];
  return r;
}

// nodes (step 2) per thread and batch: independent loads in flight per thread
constexpr int UB2 = 2;

// NM: coarse functions per plane (1: the plane indicator; 5: with the in-plane modes cos x,
// sin x, cos y, sin y; 9: also their products cos x cos y, cos x sin y, sin x cos y,
// sin x sin y)
template <int P, int NM>
__global__ void __launch_bounds__(FusedShape<P>::NT, BLOCKS_PER_SM)
k_cg_fused(const CellCoef cf, const FArgs a) {
  using S = CellStrip<P>;
  using F = FusedShape<P>;
  constexpr int NT = F::NT, GT = F::GT, NG = F::NG;
  constexpr int NR = MAXSPAN > NM ? MAXSPAN : NM;   // values of one block reduction
  __shared__ double red[NR];
  __shared__ float redf[NR * 64];
  __shared__ float yv[MAXSPAN * NM];
  // the block's copy of the published results; at entry, the state
  __shared__ Pub sp;
  __shared__ int maxit;
  __shared__ double tol2;
  // dynamic: the coarse right-hand sides [NM][nzp] (doubles), the mode tables, then per
  // strip group its U, A, B
  extern __shared__ double dsm[];
  double* cb = dsm;
  float* mcx = reinterpret_cast<float*>(reinterpret_cast<char*>(dsm) + table_offset(NM, a.nzp));
  float* msx = mcx + a.NX;
  float* mcy = msx + a.NX;
  float* msy = mcy + a.NY;
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const uint32_t plane = (uint32_t)a.NX * (uint32_t)a.NY;
  const uint32_t plane4 = plane / 4;
  const uint32_t n4 = plane4 * (uint32_t)a.nzp;
  // the block's nodes: groups of four [c0, c1), spanning planes pl0 .. pl0 + nsp - 1
  const uint32_t c0 = min(n4, (uint32_t)bid * a.chunk4);
  const uint32_t c1 = min(n4, c0 + a.chunk4);
  const int pl0 = (int)(c0 / plane4);
  const int nsp = c1 > c0 ? (int)((c1 - 1) / plane4) - pl0 + 1 : 0;
  const int nstrip = (a.nx + S::CX - 1) / S::CX;
  const int ncs = nstrip * a.ny * a.nz;   // strips (fewer than the phi nodes)
  int* err = &a.s->fused_err;
  unsigned int nbar = 0;

  // The state at entry (read by every block before its first arrival; block 0 stores the
  // final state once the last barrier has been passed).  The scalars live in shared memory
  // and only warp 0 of a block does double arithmetic.
  if (tid == 0) {
    const CgState* st = a.s;
    sp.rz = st->rz; sp.rr = st->rr; sp.pq = st->pq; sp.alpha = st->alpha;
    sp.beta = st->beta; sp.mean = st->mean; sp.iters = st->iters; sp.done = st->done;
    sp.alphaf = (float)sp.alpha; sp.meanf = (float)sp.mean; sp.betaf = (float)sp.beta;
    sp.stop = 0;
    maxit = st->maxit;
    tol2 = st->tol2;
    // the published results start as the entry state (barriers 2 to 4 publish their part
    // of them; every block copies the whole after each)
    if (bid == 0) *a.pub = sp;
  }
  if constexpr (NM > 1) {
    for (int i = tid; i < 2 * (a.NX + a.NY); i += NT) mcx[i] = a.mtab[i];
  }
  __syncthreads();
  if (sp.done || bid == a.stall) return;

  float4* x4 = reinterpret_cast<float4*>(a.x);
  float4* r4 = reinterpret_cast<float4*>(a.r);
  float4* z4 = reinterpret_cast<float4*>(a.z);
  float4* p4 = reinterpret_cast<float4*>(a.p);
  const float4* q4 = reinterpret_cast<const float4*>(a.q);
  const float4* d4 = reinterpret_cast<const float4*>(a.dinv);
  const uchar4* m4 = reinterpret_cast<const uchar4*>(a.mask);

  // the block's sums of NM per-thread accumulators to out[(bid * MAXSPAN + sl) * NM + j]:
  // the indicator's in float pairs (it also carries the mean), the modes' in float
  auto store_sums = [&](const float (&ms)[NM], double* out, int sl) {
    const float m0[1] = {ms[0]};
    block_sum_f<1>(m0, red, redf);
    if constexpr (NM > 1) {
      float mm[NM - 1];
#pragma unroll
      for (int j = 1; j < NM; ++j) mm[j - 1] = ms[j];
      block_sum_plain<NM - 1>(mm, yv, redf);
    }
    if (tid < NM)
      out[((int64_t)bid * MAXSPAN + sl) * NM + tid] = tid == 0 ? red[0] : (double)yv[tid - 1];
  };
  // the sums of v over the free nodes of the block's range against the coarse functions of
  // each plane, plane by plane, into out (groups of four nodes; with the mode space a group
  // lies in one row)
  auto restrict4 = [&](const float4* v4, double* out) {
    for (int sl = 0; sl < nsp; ++sl) {
      const uint32_t pb = (uint32_t)(pl0 + sl) * plane4;
      const uint32_t lo = max(c0, pb), hi = min(c1, pb + plane4);
      float ms[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) ms[j] = 0.f;
      for (uint32_t k = lo + tid; k < hi; k += NT) {
        float4 v = ldcg4(v4 + k);
        const uchar4 mv = m4[k];
        if (mv.x) v.x = 0.f;
        if (mv.y) v.y = 0.f;
        if (mv.z) v.z = 0.f;
        if (mv.w) v.w = 0.f;
        const float s0 = sum4(v);
        ms[0] += s0;
        if constexpr (NM > 1) {
          const uint32_t i4 = (k - pb) * 4;
          const uint32_t gy = i4 / (uint32_t)a.NX, gx = i4 - gy * (uint32_t)a.NX;
          const float4 cx = *reinterpret_cast<const float4*>(mcx + gx);
          const float4 sx = *reinterpret_cast<const float4*>(msx + gx);
          const float vc = v.x * cx.x + v.y * cx.y + v.z * cx.z + v.w * cx.w;
          const float vs = v.x * sx.x + v.y * sx.y + v.z * sx.z + v.w * sx.w;
          const float cy = mcy[gy], sy = msy[gy];
          ms[1] += vc;
          ms[2] += vs;
          ms[3] += cy * s0;
          ms[4] += sy * s0;
          if constexpr (NM == 9) {
            ms[5] += cy * vc;
            ms[6] += sy * vc;
            ms[7] += cy * vs;
            ms[8] += sy * vs;
          }
        }
      }
      store_sums(ms, out, sl);
    }
  };

  bool pending = false;   // p = z + beta p not yet stored
  float bf = 0.f;
  for (int it = 0; it < a.nit; ++it) {
    // ---- 1. cell products of the search direction (a strip per thread group); in a
    // launch's first iteration also the exact sums of r against the coarse functions of the
    // block's planes (later iterations carry them by recurrence)
    if (it == 0) restrict4(r4, a.seg_r);
    {
      const int g = tid / GT, gt = tid - g * GT;
      float* Ug = reinterpret_cast<float*>(reinterpret_cast<char*>(dsm) + a.grp_off) +
                  (size_t)g * F::GROUP_FLOATS;
      float* Ag = Ug + S::U_FLOATS;
      float* Bg = Ag + S::A_FLOATS;
      auto sync = [g] { asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory"); };
      // (32-bit strip indices: the mesh has fewer than 2^31 phi nodes)
      for (int t = bid * NG + g; t < ncs; t += G * NG) {
        const int cs = t % nstrip;
        const int rest = t / nstrip;
        const int cy = rest % a.ny, cz = rest / a.ny;
        for (int e = gt; e < S::U_FLOATS; e += GT) {
          const int64_t gid = fe_kc::strip_node<P>(e, cs * S::CX, cy, cz, a.NX, a.NY);
          const float pv = __ldcg(a.p + gid);
          Ug[e] = pending ? __fmaf_rn(bf, pv, __ldcg(a.z + gid)) : pv;
        }
        fe_kc::strip_products<P>(cf, a.ycell, cs * S::CX, cy, cz, a.nx, a.ny, Ug, Ag, Bg, gt,
                                 sync);
      }
    }
    if (!grid_barrier(a.bar, err, ++nbar, a.pub, &sp, [] {}, false)) return;

    // ---- 2. q = K p (node sums), the stored direction, p.q, the sums of q over the free
    // nodes against the coarse functions; alpha and the coarse right-hand sides ----------
    {
      float acc = 0.f;
      const uint32_t n0 = c0 * 4, n1 = c1 * 4;
      for (uint32_t base = n0 + tid; base < n1; base += UB2 * NT) {
        float pv[UB2], qv[UB2];
#pragma unroll
        for (int u = 0; u < UB2; ++u) {
          const uint32_t id = base + u * NT;
          pv[u] = 0.f;
          qv[u] = 0.f;
          if (id < n1) {
            float pp = __ldcg(a.p + id);
            if (pending) pp = __fmaf_rn(bf, pp, __ldcg(a.z + id));
            pv[u] = pp;
            const uint32_t gz = id / plane, i = id - gz * plane;
            const uint32_t gy = i / (uint32_t)a.NX, gx = i - gy * (uint32_t)a.NX;
            int dx[2], dy[2];
            const int nxc = fe_kc::cell_copies_periodic<P>((int)gx, a.nx, dx);
            const int nyc = fe_kc::cell_copies_periodic<P>((int)gy, a.ny, dy);
            qv[u] = fe_kc::cell_gather_node<P>(a.ycell, dx, nxc, dy, nyc, (int)gz, a.nx, a.ny,
                                               a.nz);
          }
        }
#pragma unroll
        for (int u = 0; u < UB2; ++u) {
          const uint32_t id = base + u * NT;
          if (id < n1) {
            if (pending) a.p[id] = pv[u];
            a.q[id] = qv[u];
            acc = __fmaf_rn(pv[u], qv[u], acc);
          }
        }
      }
      const float f[1] = {acc};
      block_sum_f<1>(f, red, redf);   // (its barriers also order the q stores before restrict4)
      if (tid == 0) a.part[bid] = red[0];
      restrict4(q4, a.seg);
    }
    {
      // alpha; the coarse right-hand sides of r - alpha q: the sums of r (exact in a launch's
      // first iteration, else those of the previous iteration, bprev) minus alpha times the
      // sums of q, each over the blocks whose nodes meet the plane in block order; the CEF
      // mean of the new residual from the indicator sums, which it then leaves at zero (the
      // mode functions sum to zero over a plane)
      const bool first = it == 0;
      auto fin = [&] {
        double t[1];
        sum_parts<1>(a.part, 0, G, t, red);
        const double pq = t[0];
        const double alpha = pq == 0.0 ? 0.0 : sp.rz / pq;
        for (int e = tid; e < NM * a.nzp; e += NT) {
          const int md = e / a.nzp, k = e - md * a.nzp;
          const uint32_t g0 = (uint32_t)k * plane4, g1 = g0 + plane4 - 1;
          const int b0 = (int)(g0 / a.chunk4), b1 = (int)(g1 / a.chunk4);
          double sq = 0.0, sr = 0.0;
          for (int b = b0; b <= b1; ++b) {
            const int slot = k - (int)(((uint32_t)b * a.chunk4) / plane4);
            const int64_t at = ((int64_t)b * MAXSPAN + slot) * NM + md;
            sq += __ldcg(a.seg + at);
            if (first) sr += __ldcg(a.seg_r + at);
          }
          const double braw = (first ? sr : __ldcg(a.bprev + e)) - alpha * sq;
          if (md == 0) {
            cb[k] = braw;
          } else {
            a.bprev[e] = braw;
            a.cbgf[(md - 1) * a.nzp + k] = (float)braw;
          }
        }
        __syncthreads();
        double tt[1];
        sum_parts<1, true>(cb, 0, a.nzp, tt, red);
        const double mn = a.project ? tt[0] * a.inv_n : 0.0;
        for (int k = tid; k < a.nzp; k += NT) {
          const double b = cb[k] - mn * a.cnt[k];
          a.bprev[k] = b;
          a.cbg[k] = b;
        }
        if (tid == 0) {
          Pub* pb = a.pub;
          pb->pq = pq;
          pb->alpha = alpha;
          pb->alphaf = (float)alpha;
          pb->mean = mn;
          pb->meanf = (float)mn;
        }
      };
      if (!grid_barrier(a.bar, err, ++nbar, a.pub, &sp, fin)) return;
    }

    // ---- 3. the coarse values of the block's planes; x += alpha p, r -= alpha q, the CEF
    // mean, z = Dinv r + the coarse correction; r.z and r.r ---------------------------------
    {
      for (int k = tid; k < a.nzp; k += NT) cb[k] = __ldcg(a.cbg + k);
      float* cbf = reinterpret_cast<float*>(cb + a.nzp);   // (NM > 1) the modes' [NM - 1][nzp]
      for (int k = tid; k < (NM - 1) * a.nzp; k += NT) cbf[k] = __ldcg(a.cbgf + k);
      __syncthreads();
      // warp w for plane pl0 + w / NM and coarse function w % NM: y = sum_k Ainv[j][k] b_k
      // (lane l takes k = l, l + 32, ... in order, then a shuffle tree)
      const int lane = tid & 31;
      for (int w = tid >> 5; w < nsp * NM; w += NT / 32) {
        const int sl = w / NM, md = w - sl * NM;
        if (md == 0) {
          const double* row = a.Ainv + (int64_t)(pl0 + sl) * a.nzp;
          double y = 0.0;
          for (int k = lane; k < a.nzp; k += 32) y += row[k] * cb[k];
          y = warp_sum_d(y);
          if (lane == 0) yv[w] = (float)y;
        } else {
          // the mode inverses in float (single precision suffices for the coarse correction)
          const float* row = a.Amodes + ((size_t)(md - 1) * a.nzp + (pl0 + sl)) * a.nzp;
          const float* bk = cbf + (md - 1) * a.nzp;
          float y = 0.f;
          for (int k = lane; k < a.nzp; k += 32) y = __fmaf_rn(row[k], bk[k], y);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
          if (lane == 0) yv[w] = y;
        }
      }
      __syncthreads();
    }
    {
      const float af = sp.alphaf, meanf = sp.meanf;
      float a1 = 0.f, a2 = 0.f;
      for (uint32_t k = c0 + tid; k < c1; k += NT) {
        float4 xv = ldcg4(x4 + k), ri = ldcg4(r4 + k);
        const float4 pv = ldcg4(p4 + k), qv = ldcg4(q4 + k);
        const float4 dv = d4[k];
        const uchar4 mv = m4[k];
        if (!mv.x) { xv.x += af * pv.x; ri.x -= af * qv.x; }
        if (!mv.y) { xv.y += af * pv.y; ri.y -= af * qv.y; }
        if (!mv.z) { xv.z += af * pv.z; ri.z -= af * qv.z; }
        if (!mv.w) { xv.w += af * pv.w; ri.w -= af * qv.w; }
        x4[k] = xv;
        if (a.project) {
          ri.x -= meanf; ri.y -= meanf; ri.z -= meanf; ri.w -= meanf;
        }
        r4[k] = ri;
        const int sl = (int)(k / plane4) - pl0;
        float4 cv;
        if constexpr (NM == 1) {
          cv.x = cv.y = cv.z = cv.w = yv[sl];
        } else {
          const float* yy = yv + sl * NM;
          const uint32_t i4 = (k - (uint32_t)(pl0 + sl) * plane4) * 4;
          const uint32_t gy = i4 / (uint32_t)a.NX, gx = i4 - gy * (uint32_t)a.NX;
          const float4 cx = *reinterpret_cast<const float4*>(mcx + gx);
          const float4 sx = *reinterpret_cast<const float4*>(msx + gx);
          const float cy = mcy[gy], sy = msy[gy];
          // y0 + y1 cx + y2 sx + y3 cy + y4 sy (+ y5 cx cy + y6 cx sy + y7 sx cy + y8 sx sy)
          const float base = yy[0] + yy[3] * cy + yy[4] * sy;
          float fc = yy[1], fs = yy[2];
          if constexpr (NM == 9) {
            fc += yy[5] * cy + yy[6] * sy;
            fs += yy[7] * cy + yy[8] * sy;
          }
          cv.x = base + fc * cx.x + fs * sx.x;
          cv.y = base + fc * cx.y + fs * sx.y;
          cv.z = base + fc * cx.z + fs * sx.z;
          cv.w = base + fc * cx.w + fs * sx.w;
        }
        float4 zi;
        zi.x = mv.x ? 0.f : dv.x * ri.x + cv.x;
        zi.y = mv.y ? 0.f : dv.y * ri.y + cv.y;
        zi.z = mv.z ? 0.f : dv.z * ri.z + cv.z;
        zi.w = mv.w ? 0.f : dv.w * ri.w + cv.w;
        z4[k] = zi;
        a1 += ri.x * zi.x + ri.y * zi.y + ri.z * zi.z + ri.w * zi.w;
        a2 += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
      }
      const float f[2] = {a1, a2};
      block_sum_f<2>(f, red, redf);
      if (tid == 0) {
        a.part[G + bid] = red[0];
        a.part[2 * G + bid] = red[1];
      }
    }
    {
      // beta, r.z, r.r, the iteration count, the convergence test and the early stop
      auto fin = [&] {
        double t[2];
        sum_parts<2>(a.part + G, G, G, t, red);
        if (tid == 0) {
          Pub* pb = a.pub;
          const double rz0 = sp.rz;
          const double beta = rz0 == 0.0 ? 0.0 : t[0] / rz0;
          const int iters = sp.iters + 1;
          const int done = (t[1] <= tol2 || iters >= maxit) ? 1 : 0;
          pb->beta = beta;
          pb->betaf = (float)beta;
          pb->rz = t[0];
          pb->rr = t[1];
          pb->iters = iters;
          pb->done = done;
          pb->stop = (done || t[1] <= a.rr_lo || !(t[1] <= a.rr_hi) || iters >= a.iters_stop ||
                      it + 1 >= a.nit) ? 1 : 0;
        }
      };
      if (!grid_barrier(a.bar, err, ++nbar, a.pub, &sp, fin)) return;
    }
    pending = true;
    bf = sp.betaf;
    if (sp.stop) break;
  }

  // the direction update of the block's own nodes (no block reads p again in this launch)
  if (pending) {
    for (uint32_t k = c0 + tid; k < c1; k += NT) {
      const float4 zv = ldcg4(z4 + k);
      float4 pv = ldcg4(p4 + k);
      pv.x = __fmaf_rn(bf, pv.x, zv.x);
      pv.y = __fmaf_rn(bf, pv.y, zv.y);
      pv.z = __fmaf_rn(bf, pv.z, zv.z);
      pv.w = __fmaf_rn(bf, pv.w, zv.w);
      p4[k] = pv;
    }
  }
  if (bid == 0 && tid == 0) {
    CgState* st = a.s;
    st->rz = sp.rz;
    st->rr = sp.rr;
    st->pq = sp.pq;
    st->alpha = sp.alpha;
    st->beta = sp.beta;
    st->mean = sp.mean;
    st->iters = sp.iters;
    st->done = sp.done;
  }
}

struct Plan {
  int grid = 0;
  size_t smem = 0;
};

// the co-resident grid for the mesh (false, with nothing recorded as an error, when the
// persistent iteration cannot run: no cooperative launch, too many planes for the coarse
// right-hand sides in shared memory, no resident block)
template <int P, int NM>
bool plan_for(const fe_mesh* m, Plan* pl) {
  using F = FusedShape<P>;
  if (m->NZ > 8192) return false;
  const size_t smem = fused_smem<P, NM>(m->NZ, m->NX, m->NY);
  if (smem > 200 * 1024) return false;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
            coop != 0 && sms > 0;
  if (ok)
    ok = cudaFuncSetAttribute(k_cg_fused<P, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess;
  if (ok)
    ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_fused<P, NM>, F::NT, smem) ==
             cudaSuccess && per_sm >= 1;
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  pl->grid = std::min(per_sm, BLOCKS_PER_SM) * sms;
  pl->smem = smem;
  return true;
}

bool plan(const fe_mesh* m, Plan* pl) {
  switch (m->p) {
    case 1: return plan_for<1, 1>(m, pl);
    case 2: return plan_for<2, 1>(m, pl);
    case 3: return plan_for<3, 1>(m, pl);
    case 4: return plan_for<4, 1>(m, pl);
    case 5: return plan_for<5, 1>(m, pl);
    case 6: return plan_for<6, 1>(m, pl);
    default: return false;
  }
}

// groups of four nodes per block: an even share; false when a share would span more than
// MAXSPAN planes or the mesh has 2^31 or more phi nodes
bool chunk_for(const fe_mesh* m, int grid, uint32_t* chunk4) {
  const uint64_t plane4 = (uint64_t)m->NX * m->NY / 4;
  const uint64_t n4 = plane4 * (uint64_t)m->NZ;
  // (32-bit node indices with headroom for a batch past the end)
  if (plane4 == 0 || 4 * n4 >= (1ull << 31)) return false;
  const uint64_t c = (n4 + grid - 1) / grid;
  if ((c + plane4 - 2) / plane4 + 1 > (uint64_t)MAXSPAN) return false;
  *chunk4 = (uint32_t)c;
  return true;
}

template <int P, int NM>
fe_status launch(fe_mesh* m, const Plan& pl, const fe_cg::FusedCg& b, int nit,
                 const fe_cg::FusedStop& stop) {
  FArgs a;
  a.x = b.x; a.r = b.r; a.z = b.z; a.p = b.p;
  a.q = b.q;
  a.dinv = b.dinv;
  a.mask = b.mask;
  a.Ainv = b.Ainv;
  a.cnt = b.cnt;
  a.s = b.s;
  a.nx = m->nx; a.ny = m->ny; a.nz = m->nz;
  a.NX = m->NX; a.NY = m->NY; a.nzp = m->NZ;
  if (!chunk_for(m, pl.grid, &a.chunk4))
    return fe_fail(FE_EUNSUPPORTED, "persistent CG: a block's nodes would span too many planes");
  a.project = b.project;
  a.inv_n = 1.0 / (double)m->n_phi;
  a.nit = nit;
  a.iters_stop = stop.iters_stop;
  a.rr_lo = stop.rr_lo;
  a.rr_hi = stop.rr_hi;
  a.stall = m->cg_stall;
  a.Amodes = NM > 1 ? b.Amodes : nullptr;
  a.mtab = NM > 1 ? b.mtab : nullptr;
  a.grp_off = (unsigned int)group_offset<NM>(m->NZ, m->NX, m->NY);
  // workspace: partials, per-plane sums, the coarse right-hand sides, the published results
  // and the barrier words (each on its own 128-byte line); the cell grid is the two-pass
  // operator's scratch
  const size_t nsegs = (size_t)pl.grid * MAXSPAN * NM;
  const size_t nd = 3 * (size_t)pl.grid + 2 * nsegs + (size_t)a.nzp + (size_t)NM * a.nzp;
  const size_t off_cbgf = (sizeof(double) * nd + 127) / 128 * 128;
  const size_t off_pub = (off_cbgf + sizeof(float) * (size_t)(NM - 1) * a.nzp + 127) / 128 * 128;
  const size_t off_bar = off_pub + 256;
  const size_t bytes = off_bar + 256;
  void* w = nullptr;
  FE_TRY(fe_ws(m, WS_CGF, bytes, &w));
  char* wb = static_cast<char*>(w);
  a.part = reinterpret_cast<double*>(wb);
  a.seg = a.part + 3 * (size_t)pl.grid;
  a.seg_r = a.seg + nsegs;
  a.cbg = a.seg_r + nsegs;
  a.bprev = a.cbg + a.nzp;
  a.cbgf = reinterpret_cast<float*>(wb + off_cbgf);
  a.pub = reinterpret_cast<Pub*>(wb + off_pub);
  a.bar = reinterpret_cast<unsigned int*>(wb + off_bar);
  void* yc = nullptr;
  FE_TRY(fe_ws(m, WS_KCELL, fe_kcell_scratch_bytes(m), &yc));
  a.ycell = static_cast<float*>(yc);
  FE_CUDA(cudaMemsetAsync(a.bar, 0, 256, m->stream));
  const CellCoef cf = fe_kc::cell_coef(m);
  void* args[] = {(void*)&cf, (void*)&a};
  FE_CUDA(cudaLaunchCooperativeKernel((const void*)k_cg_fused<P, NM>, dim3(pl.grid),
                                      dim3(FusedShape<P>::NT), args, pl.smem, m->stream));
  fe_count_launch();
  return FE_OK;
}

// the mode coarse space needs planes whose groups of four nodes lie in one row
template <int P>
fe_status run_p(fe_mesh* m, const fe_cg::FusedCg& b, int nit, const fe_cg::FusedStop& stop) {
  Plan pl;
  if (b.Amodes && b.mtab && m->NX % 4 == 0 && plan_for<P, MODES_NM>(m, &pl))
    return launch<P, MODES_NM>(m, pl, b, nit, stop);
  if (!plan_for<P, 1>(m, &pl)) return fe_fail(FE_EUNSUPPORTED, "persistent CG: no co-resident grid");
  return launch<P, 1>(m, pl, b, nit, stop);
}

}  // namespace

namespace fe_cg {

bool fused_available(fe_mesh* m) {
  if (((int64_t)m->NX * m->NY) % 4 != 0) return false;
  Plan pl;
  uint32_t c = 0;
  return plan(m, &pl) && chunk_for(m, pl.grid, &c);
}

fe_status fused_run(fe_mesh* m, const FusedCg& b, int nit, const FusedStop& stop) {
  if (nit < 1) return fe_fail(FE_EINVAL, "persistent CG: nit < 1");
  switch (m->p) {
    case 1: return run_p<1>(m, b, nit, stop);
    case 2: return run_p<2>(m, b, nit, stop);
    case 3: return run_p<3>(m, b, nit, stop);
    case 4: return run_p<4>(m, b, nit, stop);
    case 5: return run_p<5>(m, b, nit, stop);
    case 6: return run_p<6>(m, b, nit, stop);
    default: return fe_fail(FE_EUNSUPPORTED, "persistent CG: p = %d", m->p);
  }
}

}  // namespace fe_cg

// Per-cell dense stiffness products on the tcgen05 tensor cores (FE_BF16_F32ACC).
//
// Section 2.3 FE discretization: the stiffness K = sum_e P_e^T K_e P_e with the exactly
// integrated cell matrix K_e (dense (p+1)^3 x (p+1)^3; identical for every cell of the
// uniform mesh).  Here the Hamiltonian part 1/2 M^-1/2 K M^-1/2 X is evaluated as
//   kernel 1 (tensor cores): for every cell e and 64-vector tile, y_e = K_e (S X)_e
//     with S = M^-1/2, as a 128-row (M) x 224 (K) x 64 (N) bf16 product per M tile on
//     tcgen05 with fp32 accumulation in tensor memory.  K_e lives in shared memory for
//     the whole persistent CTA (one cp.async.bulk copy of a pre-swizzled image); the cell
//     tile is gathered from the node-major block, scaled by S, rounded to bf16 and written
//     in the UMMA K-major 128-byte-swizzle layout; two stages alternate so the gather of
//     one cell overlaps the MMAs of the previous one and the tensor-memory read-out of
//     the one before.  y_e goes to a per-cell buffer (fp32).
//   kernel 2 (assembly): every stored node sums the y_e of its cells (at most 8), applies
//     the output scale, the potential and the fused Chebyshev update
//       Y = alpha (S sum_e y_e + (V - shift) X) + beta Z,
//     so each node is written once; no atomics.
// Every wait on an mbarrier is bounded; on expiry the kernel records an error flag,
// drains its own outstanding MMAs (bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fe_internal.h"

namespace {

constexpr int TC_N = 64;          // vectors per tile (MMA N)
constexpr int TC_THREADS = 256;   // 8 warps: all gather, warps 0-3 read tensor memory
constexpr int ATOM_ROWS_BYTES = 128;
constexpr unsigned WAIT_CAP = 1u << 22;

template <int P>
struct TcShape {
  static constexpr int N1 = P + 1;
  static constexpr int NE = N1 * N1 * N1;
  static constexpr int MT = (NE + 127) / 128;          // M tiles of 128 rows
  static constexpr int KP = (NE + 15) / 16 * 16;       // K padded to the MMA K of 16
  static constexpr int KS = KP / 16;                   // MMA K steps
  static constexpr int KA = (KP + 63) / 64;            // 128-byte swizzle atoms along K
  static constexpr int A_BYTES = MT * KA * 128 * ATOM_ROWS_BYTES;
  static constexpr int B_BYTES = KA * TC_N * ATOM_ROWS_BYTES;
  static constexpr int TMEM_COLS_NEEDED = 2 * MT * TC_N;
  static constexpr int TMEM_COLS = TMEM_COLS_NEEDED <= 32 ? 32 : TMEM_COLS_NEEDED <= 64 ? 64
                                   : TMEM_COLS_NEEDED <= 128 ? 128 : TMEM_COLS_NEEDED <= 256 ? 256 : 512;
  static constexpr int SMEM = 1024 + A_BYTES + 2 * B_BYTES + 64;
};

struct TcArgs {
  const float* X; int64_t ldx; int64_t nvec;
  float* Ycell;                 // [nvt][ncells][NE][64]
  const unsigned char* Aimg;    // pre-swizzled K_e image, A_BYTES
  int* err;
  int nx, ny, nz, NX, NY, gz_lo, NZs, nvt;
  int64_t ncells;
  float sig[FE_MAXN1], wz[FE_MAXN1];
  float zin;
};

struct AsmArgs {
  const float* X; int64_t ldx;
  float* Y; int64_t ldy;
  const float* Z; int64_t ldz;
  const float* V;
  const float* Ycell;
  int64_t nvec, npsi, ncells;
  int nx, ny, nz, NX, NY, gz_lo, NZs, nvt;
  float sig[FE_MAXN1], wz[FE_MAXN1];
  float zout;
  float alpha, beta, shift;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and raises the error flag) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, int* err) {
  for (unsigned i = 0; i < WAIT_CAP; ++i)
    if (mbar_try_wait(addr, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = TC_N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(mbar)
               : "memory");
}

#define FE_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), \
                 "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])

// 32 lanes x 32 columns of 32-bit values starting at taddr (lane bits 31:16, column 15:0)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : FE_R8(0), FE_R8(8), FE_R8(16), FE_R8(24)
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
#undef FE_R8

__device__ __forceinline__ float mz_of(const float* wz, int gz, int P, int nz) {
  int l = gz % P;
  if (l != 0) return wz[l];
  return (gz == 0 || gz == nz * P) ? wz[0] : 2.0f * wz[0];
}

template <int P>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_cells_kernel(const TcArgs a) {
  using S = TcShape<P>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB0 = sA + S::A_BYTES;
  uint64_t* mbar = (uint64_t*)(sB0 + 2 * S::B_BYTES);      // [0], [1]: MMA stages, [2]: A load
  uint32_t* tmem_slot = (uint32_t*)(mbar + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  __shared__ int s_abort;
  if (tid == 0) {
    s_abort = 0;
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    mbar_init(smem_u32(&mbar[2]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"((uint32_t)S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // the constant K_e image: one bulk copy, consumed only by the tensor core, so only the
  // issuing thread waits for it
  if (tid == 0) {
    mbar_expect_tx(smem_u32(&mbar[2]), (uint32_t)S::A_BYTES);
    bulk_g2s(smem_u32(sA), a.Aimg, (uint32_t)S::A_BYTES, smem_u32(&mbar[2]));
    if (!mbar_wait(smem_u32(&mbar[2]), 0, a.err)) s_abort = 1;
  }

  const int64_t nitems = (int64_t)a.nvt * a.ncells;
  const uint32_t idesc = idesc_bf16(128, TC_N);
  const float zin = a.zin;
  int committed[2] = {0, 0};   // commits issued per stage (uniform across the block)
  int drained[2] = {0, 0};     // completions this thread has observed per stage

  // wait until stage s has completed its first `upto` commits (parity of the last one)
  auto wait_stage = [&](int s, int upto) -> bool {
    while (drained[s] < upto) {
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(drained[s] & 1), a.err)) return false;
      ++drained[s];
    }
    return true;
  };

  // tensor memory -> per-cell output buffer for the item multiplied in stage s (warps 0-3)
  auto epilogue = [&](int64_t item, int s) -> bool {
    if (warp >= 4) return true;
    if (!wait_stage(s, committed[s])) return false;
    tc_fence_after();
    const int64_t vt = item / a.ncells, cell = item % a.ncells;
#pragma unroll
    for (int mt = 0; mt < S::MT; ++mt) {
      const int row = mt * 128 + warp * 32 + lane;
      float* dst = a.Ycell + (((vt * a.ncells + cell) * S::NE) + row) * TC_N;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) +
                               (uint32_t)(s * S::MT * TC_N + mt * TC_N + half * 32);
        tmem_ld32(taddr, r);
        if (row < S::NE) {
          float4* d4 = reinterpret_cast<float4*>(dst + half * 32);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            d4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
      }
    }
    tc_fence_before();
    return true;
  };

  int t = 0;
  int64_t prev_item = -1;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++t) {
    const int s = t & 1;
    unsigned char* sB = sB0 + s * S::B_BYTES;
    // stage s is free once the MMAs of item t-2 have completed
    bool mine_ok = wait_stage(s, committed[s]);
    const int64_t vt = item / a.ncells, cell = item % a.ncells;
    const int cx = (int)(cell % a.nx), cy = (int)((cell / a.nx) % a.ny);
    const int cz = (int)(cell / ((int64_t)a.nx * a.ny));
    // gather: (vector n, group g of 8 nodes) -> one 16-byte chunk of B row n
    constexpr int NG = S::KA * 8;
    for (int e = tid; mine_ok && e < TC_N * NG; e += TC_THREADS) {
      const int n = e % TC_N, g = e / TC_N;
      const int64_t v = vt * TC_N + n;
      uint32_t packed[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float f[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int mloc = g * 8 + h * 2 + u;
          float x = 0.0f;
          if (mloc < S::NE && v < a.nvec) {
            const int i = mloc % S::N1, j = (mloc / S::N1) % S::N1, k = mloc / (S::N1 * S::N1);
            const int gz = cz * P + k;
            const int zs = gz - a.gz_lo;
            if (zs >= 0 && zs < a.NZs) {
              const int gx = (cx * P + i) % a.NX, gy = (cy * P + j) % a.NY;
              const int64_t nid = gx + (int64_t)a.NX * (gy + (int64_t)a.NY * zs);
              const float sc =
                  zin * rsqrtf(mz_of(a.wz, gz, P, a.nz)) * a.sig[i % P] * a.sig[j % P];
              x = sc * __ldg(a.X + nid * a.ldx + v);
            }
          }
          f[u] = x;
        }
        __nv_bfloat162 b2 = __floats2bfloat162_rn(f[0], f[1]);
        packed[h] = *reinterpret_cast<uint32_t*>(&b2);
      }
      const int atom = g >> 3, cc = g & 7;
      uint4* dst = reinterpret_cast<uint4*>(sB + atom * (TC_N * ATOM_ROWS_BYTES) +
                                            n * ATOM_ROWS_BYTES + ((cc ^ (n & 7)) << 4));
      *dst = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
    if (!mine_ok) s_abort = 1;
    fence_proxy_async();
    __syncthreads();
    if (s_abort) break;   // block-uniform: read after the barrier
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
      for (int mt = 0; mt < S::MT; ++mt) {
        const uint32_t d = tmem + (uint32_t)(s * S::MT * TC_N + mt * TC_N);
#pragma unroll 1
        for (int ks = 0; ks < S::KS; ++ks) {
          const uint32_t koff = (uint32_t)((ks & 3) * 32);
          const uint64_t ad =
              sdesc(a0 + (uint32_t)((mt * S::KA + (ks >> 2)) * 128 * ATOM_ROWS_BYTES) + koff);
          const uint64_t bd = sdesc(b0 + (uint32_t)((ks >> 2) * TC_N * ATOM_ROWS_BYTES) + koff);
          umma_bf16(d, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
      }
      umma_commit(smem_u32(&mbar[s]));
    }
    committed[s] += 1;
    // read out the previous item while this one multiplies
    if (prev_item >= 0 && !epilogue(prev_item, (t - 1) & 1)) s_abort = 1;
    prev_item = item;
  }
  __syncthreads();
  if (!s_abort && prev_item >= 0) {
    if (!epilogue(prev_item, (t - 1) & 1)) s_abort = 1;
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    // drain the MMAs still in flight (bounded) before the tensor memory is released
    for (int s = 0; s < 2; ++s) {
      while (drained[s] < committed[s]) {
        bool done = false;
        for (unsigned i = 0; i < WAIT_CAP && !done; ++i)
          done = mbar_try_wait(smem_u32(&mbar[s]), (uint32_t)(drained[s] & 1));
        ++drained[s];
        if (!done) break;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)S::TMEM_COLS)
                 : "memory");
  }
}

template <int P>
__global__ void tc_assemble_kernel(const AsmArgs a) {
  using S = TcShape<P>;
  constexpr int CH = 4;                       // vectors per thread (one float4)
  constexpr int QPT = TC_N / CH;              // chunks per 64-vector tile
  const int64_t total = a.npsi * a.nvt * QPT;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % QPT);
    const int64_t r = e / QPT;
    const int vt = (int)(r % a.nvt);
    const int64_t node = r / a.nvt;
    const int64_t v0 = (int64_t)vt * TC_N + q * CH;
    if (v0 >= a.nvec) continue;
    const int gx = (int)(node % a.NX), gy = (int)((node / a.NX) % a.NY);
    const int zs = (int)(node / ((int64_t)a.NX * a.NY));
    const int gz = zs + a.gz_lo;
    int cxs[2], lxs[2], cys[2], lys[2], czs[2], lzs[2];
    int nxc = 0, nyc = 0, nzc = 0;
    if (gx % P == 0) {
      cxs[nxc] = (gx / P - 1 + a.nx) % a.nx; lxs[nxc++] = P;
      cxs[nxc] = (gx / P) % a.nx; lxs[nxc++] = 0;
    } else { cxs[nxc] = gx / P; lxs[nxc++] = gx % P; }
    if (gy % P == 0) {
      cys[nyc] = (gy / P - 1 + a.ny) % a.ny; lys[nyc++] = P;
      cys[nyc] = (gy / P) % a.ny; lys[nyc++] = 0;
    } else { cys[nyc] = gy / P; lys[nyc++] = gy % P; }
    if (gz % P == 0) {
      if (gz / P - 1 >= 0) { czs[nzc] = gz / P - 1; lzs[nzc++] = P; }
      if (gz / P < a.nz) { czs[nzc] = gz / P; lzs[nzc++] = 0; }
    } else { czs[nzc] = gz / P; lzs[nzc++] = gz % P; }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int iz = 0; iz < nzc; ++iz)
      for (int iy = 0; iy < nyc; ++iy)
        for (int ix = 0; ix < nxc; ++ix) {
          const int64_t cell = cxs[ix] + (int64_t)a.nx * (cys[iy] + (int64_t)a.ny * czs[iz]);
          const int loc = lxs[ix] + S::N1 * (lys[iy] + S::N1 * lzs[iz]);
          const float4 y = *reinterpret_cast<const float4*>(
              a.Ycell + (((int64_t)vt * a.ncells + cell) * S::NE + loc) * TC_N + q * CH);
          acc.x += y.x; acc.y += y.y; acc.z += y.z; acc.w += y.w;
        }
    const float so = a.zout * rsqrtf(mz_of(a.wz, gz, P, a.nz)) * a.sig[gx % P] * a.sig[gy % P];
    const float pv = a.V[node] - a.shift;
    float out[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int64_t v = v0 + c;
      if (v >= a.nvec) break;
      float val = a.alpha * (so * out[c] + pv * a.X[node * a.ldx + v]);
      if (a.Z != nullptr && a.beta != 0.0f) val += a.beta * a.Z[node * a.ldz + v];
      a.Y[node * a.ldy + v] = val;
    }
  }
}

// host image of K_e in the kernel's swizzled K-major layout (rows = output local node); the
// factor 1/2 of the kinetic term is applied with the output scale in the assembly kernel
template <int P>
std::vector<unsigned char> build_image(const fe_mesh* m) {
  using S = TcShape<P>;
  std::vector<unsigned char> img(S::A_BYTES, 0);
  const int n1 = S::N1;
  const double hx = m->h[0], hy = m->h[1], hz = m->h[2];
  const double ax = hy * hz / (2.0 * hx), ay = hx * hz / (2.0 * hy), az = hx * hy / (2.0 * hz);
  for (int I = 0; I < S::NE; ++I) {
    const int i = I % n1, j = (I / n1) % n1, k = I / (n1 * n1);
    for (int Jn = 0; Jn < S::NE; ++Jn) {
      const int i2 = Jn % n1, j2 = (Jn / n1) % n1, k2 = Jn / (n1 * n1);
      double v = ax * m->K1[i][i2] * m->M1[j][j2] * m->M1[k][k2] +
                 ay * m->M1[i][i2] * m->K1[j][j2] * m->M1[k][k2] +
                 az * m->M1[i][i2] * m->M1[j][j2] * m->K1[k][k2];
      __nv_bfloat16 b = __float2bfloat16_rn((float)v);
      const int mt = I / 128, row = I % 128;
      const int chunk = Jn / 8, within = Jn % 8;
      const int atom = chunk / 8, cc = chunk % 8;
      size_t off = (size_t)(mt * S::KA + atom) * 128 * ATOM_ROWS_BYTES + row * ATOM_ROWS_BYTES +
                   ((cc ^ (row & 7)) << 4) + within * 2;
      std::memcpy(&img[off], &b, 2);
    }
  }
  return img;
}

template <int P>
fe_status tc_run(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec, int64_t ld,
                 float alpha, float beta, float shift) {
  using S = TcShape<P>;
  static_assert(S::SMEM <= 227 * 1024, "shared memory");
  const int nvt = (int)((nvec + TC_N - 1) / TC_N);
  // workspaces: image + error flag, per-cell outputs
  void* wimg;
  FE_TRY(fe_ws(m, WS_TC_IMG, S::A_BYTES + 256, &wimg));
  int* err = (int*)((unsigned char*)wimg + S::A_BYTES);
  if (m->tc_img_p != P) {
    std::vector<unsigned char> img = build_image<P>(m);
    FE_CUDA(cudaMemcpyAsync(wimg, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    FE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
    m->tc_img_p = P;
  }
  void* yc;
  FE_TRY(fe_ws(m, WS_YCELL, sizeof(float) * (size_t)nvt * m->n_cells * S::NE * TC_N, &yc));
  TcArgs ta;
  ta.X = X; ta.ldx = ld; ta.nvec = nvec; ta.Ycell = (float*)yc;
  ta.Aimg = (const unsigned char*)wimg; ta.err = err;
  ta.nx = m->nx; ta.ny = m->ny; ta.nz = m->nz; ta.NX = m->NX; ta.NY = m->NY;
  ta.gz_lo = m->gz_lo; ta.NZs = m->NZs; ta.nvt = nvt; ta.ncells = m->n_cells;
  for (int k = 0; k < FE_MAXN1; ++k) {
    ta.sig[k] = (float)m->coefH.sig[k];
    ta.wz[k] = (float)m->coefH.wz[k];
  }
  ta.zin = (float)m->coefH.zin;
  auto kern = tc_cells_kernel<P>;
  FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, m->device);
  int64_t items = (int64_t)nvt * m->n_cells;
  int grid = (int)(items < dev_sms ? items : dev_sms);
  kern<<<grid, TC_THREADS, S::SMEM, m->stream>>>(ta); fe_count_launch();
  FE_CUDA(cudaGetLastError());

  AsmArgs aa;
  aa.X = X; aa.ldx = ld; aa.Y = Y; aa.ldy = ld; aa.Z = Z; aa.ldz = ld; aa.V = m->d_veff_f;
  aa.Ycell = (const float*)yc; aa.nvec = nvec; aa.npsi = m->n_psi; aa.ncells = m->n_cells;
  aa.nx = m->nx; aa.ny = m->ny; aa.nz = m->nz; aa.NX = m->NX; aa.NY = m->NY;
  aa.gz_lo = m->gz_lo; aa.NZs = m->NZs; aa.nvt = nvt;
  for (int k = 0; k < FE_MAXN1; ++k) { aa.sig[k] = ta.sig[k]; aa.wz[k] = ta.wz[k]; }
  aa.zout = (float)m->coefH.zout;
  aa.alpha = alpha; aa.beta = beta; aa.shift = shift;
  int64_t total = m->n_psi * nvt * (TC_N / 4);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  tc_assemble_kernel<P><<<(int)blocks, 256, 0, m->stream>>>(aa); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  // a raised wait-expiry flag is reported by the next call (no synchronisation here)
  if (!m->tc_err_pinned) {
    FE_CUDA(cudaHostAlloc((void**)&m->tc_err_pinned, sizeof(int), cudaHostAllocDefault));
    *m->tc_err_pinned = 0;
  }
  FE_CUDA(cudaMemcpyAsync(m->tc_err_pinned, err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  return FE_OK;
}

}  // namespace

fe_status fe_tc_apply(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec,
                      int64_t ld, float alpha, float beta, float shift, fe_precision prec) {
  if (prec != FE_BF16_F32ACC)
    return fe_fail(FE_EUNSUPPORTED, "tensor-core path: only FE_BF16_F32ACC is built");
  if (m->tc_err_pinned && *m->tc_err_pinned != 0)
    return fe_fail(FE_ETIMEOUT, "a tensor-core kernel's bounded wait expired earlier");
  switch (m->p) {
    case 2: return tc_run<2>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 3: return tc_run<3>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 4: return tc_run<4>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 5: return tc_run<5>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    default:
      return fe_fail(FE_EUNSUPPORTED, "tensor-core path supports p = 2..5 (p = %d)", m->p);
  }
}

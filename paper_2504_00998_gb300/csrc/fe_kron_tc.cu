// FP32-accurate Hamiltonian operator with the in-plane contractions on the tcgen05 tensor
// cores (FE_F32_F32ACC).
//
// Section 2.3 with Eq. Veff and Hloc: Ht = 1/2 M^-1/2 K M^-1/2 + diag(V_eff), with the
// exactly integrated stiffness of the uniform tensor-product mesh
//   K = ax K1 (x) M1 (x) M1 + ay M1 (x) K1 (x) M1 + az M1 (x) M1 (x) K1.
// The kernel evaluates the fused Chebyshev step Y = alpha (Ht - shift) X + beta Z with the
// same sum factorisation and z sweep as the CUDA-core operator (fe_kron.cuh): a CTA owns
// the nodes of an xy block of B x B cells and 8 vectors, stages each z plane with its
// p-node periodic halo, and accumulates the z contraction of the plane's in-plane results
// into the p + 1 output planes of the current cell layer, in registers.  What changes is
// how a plane's two in-plane contractions run:
//   (1) y contraction  D1[(xh, v)][n] = sum_yh U[yh][xh][v] B1[n][yh]
//       (n < 16: a = Ay_M U at the owned y; n >= 16: b = Ay_K U),
//   (2) x contraction  D2[(y, v)][n] = sum_k A2[(y, v)][k] B2[n][k], k = (part, xh)
//       (W1 = Ax_M a and W2 = Ax_K a + Ax_M b at the owned x, split into two halves),
// each one 128-row tcgen05.mma chain (kind::tf32, M = 128, N = 32, K = 8 per instruction)
// with the accumulator in tensor memory.  B1 and B2 are the assembled 1D operators of one
// block (the same for every block: the block size is a multiple of p), built on the host.
// Precision: every operand is split into a TF32 part and a TF32 remainder (hi = x rounded
// to 11 significant bits, lo = x - hi) and the product is hi*hi + lo*hi + hi*lo, which
// carries about 2^-22 of relative error per product -- the FP32 operator's accuracy class;
// accumulation is FP32.  The z contraction, the potential, the mass scalings and the
// Chebyshev combination run on the CUDA cores in FP32 as in the CUDA-core operator.
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises an error flag (reported
// by the next call as FE_ETIMEOUT), stops its sweep, waits (bounded) for its own MMAs and
// frees its tensor memory.
#include <cstring>
#include <vector>

#include "fe_kron.cuh"

namespace {

using fe::KronCoefT;

constexpr int KT_THREADS = 256;
constexpr int KT_TV = 8;               // vectors per CTA tile
constexpr unsigned KT_WAIT_CAP = 1u << 22;
constexpr int KT_IMG_BYTES = 4 * 4096; // B1 hi, B1 lo, B2 hi, B2 lo: 32 rows x 128 bytes each
constexpr int KT_TMEM_COLS = 64;       // D1 at column 0, D2 at column 32

template <int P>
struct KtShape {
  static constexpr int B = fe::KronBlock<P>::B;   // cells per block side
  static constexpr int BN = B * P;                // owned nodes per side
  static constexpr int BH = BN + P + 1;           // staged (halo) nodes per side
  static constexpr int XH = (BN + 1) / 2;         // owned x outputs per D2 column half
  static constexpr int NST = BH * BH * 2;         // 16-byte chunks per staged plane
  static constexpr int SPT = (NST + KT_THREADS - 1) / KT_THREADS;
  static constexpr int NSB = 3;                   // staging slots
  static_assert(BH <= 16 && XH <= 8 && BN * KT_TV <= 128, "block exceeds one MMA tile");
  static constexpr size_t STAGE_FLOATS = (size_t)NSB * BH * BH * KT_TV;
  static constexpr size_t VS_FLOATS = (size_t)NSB * BN * BN;
  // layout after the 1024-byte aligned base: A parts (32 KB), B images (16 KB), mbarriers and
  // the tensor-memory slot (64 bytes), stage ring, V ring
  static constexpr size_t SMEM = 1024 + 32768 + KT_IMG_BYTES + 64 + 4 * (STAGE_FLOATS + VS_FLOATS);
};

struct KtArgs {
  KronGeom g;
  const float* X; int64_t ldx;
  float* Y; int64_t ldy;
  const float* Z; int64_t ldz;
  const float* V;
  int64_t nvec;
  float alpha, beta, shift;
  const unsigned char* img;   // B operator images (KT_IMG_BYTES)
  int* err;
  int nvt;
};

// ---- tcgen05 / mbarrier helpers (inline PTX) ------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
__device__ __forceinline__ bool mb_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint32_t a, uint32_t parity) {
  for (unsigned i = 0; i < KT_WAIT_CAP; ++i)
    if (mb_try(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void tc_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor: tf32 x tf32 -> f32, both K-major, M = 128, N = 32
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(32 >> 3) << 17) |
                                ((uint32_t)(128 >> 4) << 24);
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d), "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(mbar)
               : "memory");
}
#define KT_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), \
                 "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : KT_R8(0), KT_R8(8)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : KT_R8(0)
               : "r"(taddr));
}
#undef KT_R8
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x = hi + lo with hi rounded to TF32 (11 significant bits; the tensor core reads the top 19
// bits of a 32-bit operand) and lo = x - hi exactly
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  // round to nearest (ties away from zero) at bit 13 of the finite value's bits
  const uint32_t h = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  hi = h;
  lo = __float_as_uint(x - __uint_as_float(h));
}

// byte offset of element (row, k) of a K-major, 128-byte-swizzled tile of 32-bit elements
__device__ __forceinline__ uint32_t swz(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ row) & 7) << 4) +
                    ((k & 3) << 2));
}

template <int P, bool FULL>
__global__ void __launch_bounds__(KT_THREADS, 2)
ktc_kernel(const KronCoefT<float> cf, const KtArgs a) {
  using S = KtShape<P>;
  constexpr int BN = S::BN, BH = S::BH, XH = S::XH, NSB = S::NSB, SPT = S::SPT, NST = S::NST;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // (pointer arithmetic on the shared array keeps the shared state space for the accesses)
  unsigned char* base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sAh = base;                 // A1 / A2 TF32 parts (aliased by the two stages)
  unsigned char* sAl = base + 16384;         // remainders
  unsigned char* sB = base + 32768;          // B1 hi, B1 lo, B2 hi, B2 lo
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + KT_IMG_BYTES);   // 8-byte aligned
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  float* stage = reinterpret_cast<float*>(sB + KT_IMG_BYTES + 64);   // [NSB][BH][BH][8]
  float* Vs = stage + S::STAGE_FLOATS;                                // [NSB][BN][BN]
  __shared__ int s_abort;

  const KronGeom& g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nxy = g.nbx * g.nby;
  const int rb = blockIdx.x / a.nvt;
  const int bxy = rb % nxy, vti = blockIdx.x % a.nvt, zsi = rb / nxy;
  const int x0 = (bxy % g.nbx) * BN, y0 = (bxy / g.nbx) * BN;
  const int64_t vt0 = (int64_t)vti * KT_TV;
  const int c0 = zsi * g.zseg;
  const int c1 = min(c0 + g.zseg, g.nz);
  const int cb = c0 > 0 ? c0 - 1 : 0;
  const int gbeg = cb * P, gend = c1 * P;
  const int64_t plane_nodes = (int64_t)g.NX * g.NY;

  if (tid == 0) {
    s_abort = 0;
    mb_init(su32(&mbar[0]), 1);
    mb_init(su32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(su32(tslot)), "r"((uint32_t)KT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_before();
  }
  // operator images into shared memory (read only by the tensor core)
  for (int i = tid; i < KT_IMG_BYTES / 16; i += KT_THREADS)
    reinterpret_cast<uint4*>(sB)[i] = __ldg(reinterpret_cast<const uint4*>(a.img) + i);
  proxy_fence();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  // ---- staging addresses (per thread, once) ----------------------------------------------
  int64_t s_goff[SPT];
  int s_bytes[SPT];
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    const int e = tid + i * KT_THREADS;
    const int ec = e < NST ? e : 0;
    const int ch = ec & 1, node = ec >> 1;
    const int xh = node % BH, yh = node / BH;
    const int gx = fe::pmod(x0 - P + xh, g.NX), gy = fe::pmod(y0 - P + yh, g.NY);
    const int64_t v0 = vt0 + ch * 4;
    const int64_t rem = a.nvec - v0;
    s_bytes[i] = e >= NST ? -1 : (FULL ? 16 : (rem <= 0 ? 0 : (rem >= 4 ? 16 : (int)(rem * 4))));
    s_goff[i] = (gx + (int64_t)g.NX * gy) * a.ldx + v0;
  }

  // ---- roles ------------------------------------------------------------------------------
  // conversion: row m = (xh, v) of A1, K half kh (8 y rows each)
  const int cm = tid & 127, ckh = tid >> 7;
  const int cxh = cm >> 3, cv = cm & 7;
  // D1 read-out / A2 write: TMEM lane r = (xh, v), part 0 (a) or 1 (b)
  const int r1 = lane + 32 * (warp & 3);
  const int dxh = r1 >> 3, dv = r1 & 7, dpart = warp >> 2;
  // D2 read-out / z contraction / output: TMEM lane r = (y, v), x half h
  const int r2 = r1;
  const int zy = r2 >> 3, zv = r2 & 7, zh = warp >> 2;
  const bool zrow = zy < BN;
  const int64_t zvec = vt0 + zv;
  bool zown[XH];
  float sxy[XH], isxy[XH];
  int64_t znode[XH];
  float acc[P + 1][XH];
#pragma unroll
  for (int q = 0; q < XH; ++q) {
    const int xq = zh * XH + q;
    zown[q] = zrow && xq < BN && (FULL || (x0 + xq < g.NX && y0 + zy < g.NY && zvec < a.nvec));
    znode[q] = (x0 + xq) + (int64_t)g.NX * (y0 + zy);
    sxy[q] = cf.mass_scale ? cf.sig[xq % P] * cf.sig[zy % P] : 1.0f;
    isxy[q] = 1.0f / sxy[q];
#pragma unroll
    for (int j = 0; j <= P; ++j) acc[j][q] = 0.0f;
  }

  auto stored = [&](int gz) { return gz - g.gz_lo >= 0 && gz - g.gz_lo < g.NZs; };
  auto rsq_of = [&](int gz) -> float {
    if (!cf.mass_scale) return 1.0f;
    const int l = gz % P;
    if (l != 0) return cf.rsq[l];
    return (gz == 0 || gz == g.nz * P) ? cf.rsq_face : cf.rsq[0];
  };
  auto sq_of = [&](int gz) -> float {
    if (!cf.mass_scale) return 1.0f;
    const int l = gz % P;
    if (l != 0) return cf.sq[l];
    return (gz == 0 || gz == g.nz * P) ? cf.sq_face : cf.sq[0];
  };
  auto owned_plane = [&](int gz) {
    return stored(gz) && ((gz >= c0 * P && gz < c1 * P) || (gz == g.nz * P && c1 == g.nz));
  };

  auto stage_plane = [&](int gz) {
    if (!stored(gz)) return;
    const int zs = gz - g.gz_lo;
    const int64_t pbase = (int64_t)zs * plane_nodes * a.ldx;
    float* dst = stage + (size_t)((gz - gbeg) % NSB) * BH * BH * KT_TV;
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      const int e = tid + i * KT_THREADS;
      if (s_bytes[i] > 0) fe::cp_async<16>(dst + e * 4, a.X + pbase + s_goff[i], s_bytes[i]);
      else if (s_bytes[i] == 0) fe::cp_async<16>(dst + e * 4, a.X, 0);
    }
    if (a.V != nullptr && tid < BN * BN) {
      const int x = tid % BN, y = tid / BN;
      float* vd = Vs + ((gz - gbeg) % NSB) * (BN * BN) + tid;
      const bool ok = FULL || (x0 + x < g.NX && y0 + y < g.NY);
      const int64_t nid = (int64_t)zs * plane_nodes + (x0 + x) + (int64_t)g.NX * (y0 + y);
      fe::cp_async<4>(vd, ok ? a.V + nid : a.V, ok ? 4 : 0);
    }
  };

  // The Chebyshev operand Z of output plane c P + j is loaded into zreg[j] when that plane is
  // swept (its latency hides behind the plane's work); Z may be Y itself -- the filter
  // overwrites Y_{k-1} -- and each entry is read by the thread that later writes it.
  float zreg[P][XH];
  auto load_z = [&](int gzo, int j) {
    if (a.Z == nullptr || !owned_plane(gzo) || !zrow) return;
    const int64_t pl = (int64_t)(gzo - g.gz_lo) * plane_nodes;
#pragma unroll
    for (int q = 0; q < XH; ++q)
      zreg[j][q] = zown[q] ? a.Z[(pl + znode[q]) * a.ldz + zvec] : 0.0f;
  };
  auto write_plane = [&](int gzo, int j) {
    if (!owned_plane(gzo) || !zrow) return;
    const int zs = gzo - g.gz_lo;
    const float ps = cf.zout * rsq_of(gzo);
    const int64_t pl = (int64_t)zs * plane_nodes;
#pragma unroll
    for (int q = 0; q < XH; ++q) {
      if (!zown[q]) continue;
      float out = a.alpha * ps * sxy[q] * acc[j][q];
      if (a.Z != nullptr) out = fmaf(a.beta, zreg[j][q], out);
      a.Y[(pl + znode[q]) * a.ldy + zvec] = out;
    }
  };

  // z contraction of the plane with local index K (compile time) into the layer accumulators
  auto plane_z = [&](auto kc, bool pot, bool face, float inv_ps, const float* vv, const float* st,
                     const float* w1, const float* w2) {
    constexpr int K = decltype(kc)::value;
    if constexpr (K <= P) {
#pragma unroll
      for (int q = 0; q < XH; ++q) {
        const int xq = zh * XH + q;
        if (pot && zown[q]) {
          const float pv = (vv[zy * BN + xq] - a.shift) * inv_ps * isxy[q];
          acc[K][q] = fmaf(pv, st[((zy + P) * BH + (xq + P)) * KT_TV + zv], acc[K][q]);
        }
        float u = w1[q], w = w2[q];
        if (face) { u *= cf.face_fix; w *= cf.face_fix; }
#pragma unroll
        for (int j = 0; j <= P; ++j)
          acc[j][q] = fmaf(cf.AzKs[j][K], u, fmaf(cf.AzMs[j][K], w, acc[j][q]));
      }
    }
  };
  auto dispatch_z = [&](int k, bool pot, bool face, float inv_ps, const float* vv,
                        const float* st, const float* w1, const float* w2) {
    switch (k) {
      case 0: plane_z(std::integral_constant<int, 0>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 1: plane_z(std::integral_constant<int, 1>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 2: plane_z(std::integral_constant<int, 2>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 3: plane_z(std::integral_constant<int, 3>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 4: plane_z(std::integral_constant<int, 4>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 5: plane_z(std::integral_constant<int, 5>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      default: break;
    }
  };
  auto shift_layer = [&]() {
#pragma unroll
    for (int q = 0; q < XH; ++q) {
      acc[0][q] = acc[P][q];
#pragma unroll
      for (int j = 1; j <= P; ++j) acc[j][q] = 0.0f;
    }
  };

  const uint32_t aH = su32(sAh), aL = su32(sAl);
  const uint32_t b1H = su32(sB), b1L = b1H + 4096, b2H = b1H + 8192, b2L = b1H + 12288;
  uint32_t n1 = 0, n2 = 0;            // phases of the two mbarriers seen complete (thread 0)
  uint32_t issued1 = 0, issued2 = 0;  // commits issued (thread 0)

  // ---- sweep --------------------------------------------------------------------------------
  stage_plane(gbeg);
  fe::cp_commit();
  int c = cb;
  for (int gz = gbeg; gz <= gend; ++gz) {
    const int k = gz - c * P;
    if (gz < gend) {
      stage_plane(gz + 1);
      fe::cp_commit();
      fe::cp_wait<1>();
    } else {
      fe::cp_wait<0>();
    }
    __syncthreads();
    if (s_abort) break;   // block-uniform: read after the barrier
    const float* st = stage + (size_t)((gz - gbeg) % NSB) * BH * BH * KT_TV;
    // the Chebyshev operand of this layer's output plane with local index k (only the sweep's
    // first plane has k = 0; a later layer's plane 0 is the previous layer's top plane and is
    // loaded after that layer's write-out below)
    if (k < P) {
      switch (k) {
        case 0: load_z(gz, 0); break;
        case 1: load_z(gz, 1); break;
        case 2: load_z(gz, 2); break;
        case 3: load_z(gz, 3); break;
        case 4: load_z(gz, 4); break;
        default: break;
      }
    }

    if (stored(gz)) {
      // (1) A1 = the staged plane as rows (xh, v), K = y halo row, split into TF32 parts
      {
        uint32_t hv[8], lv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int yh = ckh * 8 + i;
          const float x = (cxh < BH && yh < BH) ? st[(yh * BH + cxh) * KT_TV + cv] : 0.0f;
          split_tf32(x, hv[i], lv[i]);
        }
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const uint32_t off = swz(cm, ckh * 8 + hc * 4);
          *reinterpret_cast<uint4*>(sAh + off) = make_uint4(hv[4 * hc], hv[4 * hc + 1], hv[4 * hc + 2], hv[4 * hc + 3]);
          *reinterpret_cast<uint4*>(sAl + off) = make_uint4(lv[4 * hc], lv[4 * hc + 1], lv[4 * hc + 2], lv[4 * hc + 3]);
        }
      }
      proxy_fence();
      __syncthreads();
      if (tid == 0) {
        tc_after();
        // D1 = A1h B1h + A1l B1h + A1h B1l over K = 16 (two steps of 8)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ko = (uint32_t)ks * 32;
          mma_tf32(tmem, kdesc(aH + ko), kdesc(b1H + ko), ks > 0 ? 1u : 0u);
          mma_tf32(tmem, kdesc(aL + ko), kdesc(b1H + ko), 1u);
          mma_tf32(tmem, kdesc(aH + ko), kdesc(b1L + ko), 1u);
        }
        mma_commit(su32(&mbar[0]));
        ++issued1;
        if (mb_wait(su32(&mbar[0]), n1 & 1)) ++n1;
        else { atomicExch(a.err, 1); s_abort = 1; }
      }
      __syncthreads();   // the MMA's completion (seen by thread 0) releases the CTA
      tc_after();
      // (2) D1 read-out (rows (xh, v); part 0: a at columns 0-15, part 1: b at 16-31) and
      //     A2 = rows (y, v), K = part * 16 + xh, split into TF32 parts
      {
        uint32_t d[16];
        tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(dpart * 16), d);
        tmem_wait_ld();
        const int kk = dpart * 16 + dxh;
#pragma unroll
        for (int y = 0; y < BN; ++y) {
          const float x = dxh < BH ? __uint_as_float(d[y]) : 0.0f;
          uint32_t h, l;
          split_tf32(x, h, l);
          const uint32_t off = swz(y * KT_TV + dv, kk);
          *reinterpret_cast<uint32_t*>(sAh + off) = h;
          *reinterpret_cast<uint32_t*>(sAl + off) = l;
        }
      }
      tc_before();
      proxy_fence();
      __syncthreads();
      if (tid == 0) {
        tc_after();
        // D2 = A2h B2h + A2l B2h + A2h B2l over K = 32 (four steps of 8)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ko = (uint32_t)ks * 32;
          mma_tf32(tmem + 32, kdesc(aH + ko), kdesc(b2H + ko), ks > 0 ? 1u : 0u);
          mma_tf32(tmem + 32, kdesc(aL + ko), kdesc(b2H + ko), 1u);
          mma_tf32(tmem + 32, kdesc(aH + ko), kdesc(b2L + ko), 1u);
        }
        mma_commit(su32(&mbar[1]));
        ++issued2;
        if (mb_wait(su32(&mbar[1]), n2 & 1)) ++n2;
        else { atomicExch(a.err, 1); s_abort = 1; }
      }
      __syncthreads();
      tc_after();
      // (3) D2 read-out: W1 at columns 8 h + q, W2 at 16 + 8 h + q (q < XH), rows (y, v)
      float w1[8], w2[8];
      {
        uint32_t d[8];
        const uint32_t tl = tmem + 32 + ((uint32_t)(32 * (warp & 3)) << 16);
        tmem_ld8(tl + (uint32_t)(8 * zh), d);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) w1[q] = __uint_as_float(d[q]);
        tmem_ld8(tl + (uint32_t)(16 + 8 * zh), d);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) w2[q] = __uint_as_float(d[q]);
      }
      tc_before();
      const bool face = gz == 0 || gz == g.nz * P;
      const float inv_ps = sq_of(gz) * cf.izout;
      const float* vv = Vs + ((gz - gbeg) % NSB) * (BN * BN);
      if (zrow) dispatch_z(k, a.V != nullptr, face, inv_ps, vv, st, w1, w2);
      if (k == P) {
#pragma unroll
        for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
        shift_layer();
        ++c;
        load_z(gz, 0);
        if (c < c1 && zrow) dispatch_z(0, false, face, inv_ps, vv, st, w1, w2);
      }
    } else if (k == P) {
#pragma unroll
      for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
      shift_layer();
      ++c;
      load_z(gz, 0);
    }
  }
  if (!s_abort) write_plane(gend, 0);   // (its operand was loaded after the last layer)
  __syncthreads();
  if (s_abort && tid == 0) {
    // wait (bounded) for MMAs still in flight before the tensor memory is released
    if (issued1 > n1) mb_wait(su32(&mbar[0]), n1 & 1);
    if (issued2 > n2) mb_wait(su32(&mbar[1]), n2 & 1);
  }
  __syncthreads();
  if (warp == 0) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)KT_TMEM_COLS)
                 : "memory");
  }
}

// ---- host: operator images ---------------------------------------------------------------------
uint32_t tf32_rna(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u;   // (no infinities in the tables)
  u = (u + 0x1000u) & 0xffffe000u;
  return u;
}
void tf32_split(double c, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna((float)c);
  float h;
  std::memcpy(&h, &hi, 4);
  lo = tf32_rna((float)(c - (double)h));
}
size_t swz_host(int row, int k) {
  return (size_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ row) & 7) << 4) +
                  ((k & 3) << 2));
}

// Assembled 1D operator of one block: coefficient of halo input h (node base - P + h) in
// owned output o (node base + o), from the cell matrix A[j][k] (rows: output local index):
// output o = s P + j takes A[j][kk] from its own cell s (input halo s P + P + kk) and, at a
// cell's first node (j = 0), A[P][kk] from the previous cell (input halo s P + kk).
template <int P>
double block_coef(const double (*A)[FE_MAXN1], int o, int h) {
  const int s = o / P, j = o % P;
  double v = 0.0;
  const int kk = h - (s * P + P);
  if (kk >= 0 && kk <= P) v += A[j][kk];
  if (j == 0) {
    const int kp = h - s * P;
    if (kp >= 0 && kp <= P) v += A[P][kp];
  }
  return v;
}

template <int P>
std::vector<unsigned char> build_images(const KronCoef& cf) {
  using S = KtShape<P>;
  std::vector<unsigned char> img(KT_IMG_BYTES, 0);
  auto put = [&](int which, int n, int k, double c) {
    uint32_t hi, lo;
    tf32_split(c, hi, lo);
    std::memcpy(&img[(size_t)(2 * which) * 4096 + swz_host(n, k)], &hi, 4);
    std::memcpy(&img[(size_t)(2 * which + 1) * 4096 + swz_host(n, k)], &lo, 4);
  };
  // B1: rows n < 16 give a = Ay_M U at owned y = n, rows 16 + y give b = Ay_K U; K = y halo
  for (int y = 0; y < S::BN; ++y)
    for (int h = 0; h < S::BH; ++h) {
      put(0, y, h, block_coef<P>(cf.AyM, y, h));
      put(0, 16 + y, h, block_coef<P>(cf.AyK, y, h));
    }
  // B2: rows 8 hf + q give W1 at owned x = hf XH + q, rows 16 + 8 hf + q give W2; K = 16 part + xh
  for (int x = 0; x < S::BN; ++x) {
    const int hf = x / S::XH, q = x % S::XH;
    for (int h = 0; h < S::BH; ++h) {
      put(1, 8 * hf + q, h, block_coef<P>(cf.AxM, x, h));            // W1 from a
      put(1, 16 + 8 * hf + q, h, block_coef<P>(cf.AxK, x, h));       // W2 from a
      put(1, 16 + 8 * hf + q, 16 + h, block_coef<P>(cf.AxM, x, h));  // W2 from b
    }
  }
  return img;
}

template <int P>
fe_status ktc_run(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec, int64_t ld,
                  float alpha, float beta, float shift) {
  using S = KtShape<P>;
  void* w;
  FE_TRY(fe_ws(m, WS_KTC, KT_IMG_BYTES + 256, &w));
  int* err = (int*)((unsigned char*)w + KT_IMG_BYTES);
  if (!m->ktc_ready) {
    std::vector<unsigned char> img = build_images<P>(m->coefH);
    FE_CUDA(cudaMemcpyAsync(w, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    FE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
    if (!m->ktc_err_pinned) {
      FE_CUDA(cudaHostAlloc((void**)&m->ktc_err_pinned, sizeof(int), cudaHostAllocDefault));
      *m->ktc_err_pinned = 0;
    }
    m->ktc_ready = true;
  }
  KtArgs a;
  a.g = fe_geom(m, true);
  a.g.bx = a.g.by = S::B;
  a.g.nbx = (m->nx + S::B - 1) / S::B;
  a.g.nby = (m->ny + S::B - 1) / S::B;
  a.X = X; a.ldx = ld; a.Y = Y; a.ldy = ld; a.Z = (beta != 0.0f) ? Z : nullptr; a.ldz = ld;
  a.V = m->d_veff_f; a.nvec = nvec; a.alpha = alpha; a.beta = beta; a.shift = shift;
  a.img = (const unsigned char*)w; a.err = err;
  const int64_t nvt = (nvec + KT_TV - 1) / KT_TV;
  a.nvt = (int)nvt;
  const int64_t baseg = (int64_t)a.g.nbx * a.g.nby * nvt;
  const int64_t want = 4 * (int64_t)fe::device_sms();
  int zseg = a.g.nz;
  while (zseg > 2 && baseg * ((a.g.nz + zseg - 1) / zseg) < want) zseg = (zseg + 1) / 2;
  a.g.zseg = zseg;
  const int64_t total = baseg * ((a.g.nz + zseg - 1) / zseg);
  if (total > 0x7fffffffLL) return fe_fail(FE_EINVAL, "tensor-core operator: grid too large");
  const bool full = a.g.NX % S::BN == 0 && a.g.NY % S::BN == 0 && nvec % KT_TV == 0;
  auto kern = full ? ktc_kernel<P, true> : ktc_kernel<P, false>;
  FE_TRY(fe::kron_func_setup(kern, S::SMEM));
  KronCoefT<float> cft = fe::convert_coef<float>(m->coefH);
  kern<<<(unsigned)total, KT_THREADS, S::SMEM, m->stream>>>(cft, a); fe_count_launch();
  FE_CUDA(cudaGetLastError());
  // a raised wait-expiry flag is reported by the next call (no synchronisation here)
  FE_CUDA(cudaMemcpyAsync(m->ktc_err_pinned, err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  return FE_OK;
}

}  // namespace

fe_status fe_ktc_apply(fe_mesh* m, const float* X, float* Y, const float* Z, int64_t nvec,
                       int64_t ld, float alpha, float beta, float shift) {
  if (m->has_k)
    return fe_fail(FE_EUNSUPPORTED, "FE_F32_F32ACC: Gamma-point (real) blocks only");
  if (m->ktc_err_pinned && *m->ktc_err_pinned != 0)
    return fe_fail(FE_ETIMEOUT, "a tensor-core operator kernel's bounded wait expired earlier");
  switch (m->p) {
    case 1: return ktc_run<1>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 2: return ktc_run<2>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 3: return ktc_run<3>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 4: return ktc_run<4>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    case 5: return ktc_run<5>(m, X, Y, Z, nvec, ld, alpha, beta, shift);
    default:
      return fe_fail(FE_EUNSUPPORTED, "FE_F32_F32ACC supports p = 1..5 (p = %d)", m->p);
  }
}

// Matrix-free application of the finite-element operators of Section 2.3 on the uniform
// tensor-product slab mesh.
//
// For a uniform hexahedral mesh the assembled stiffness K_IJ = int grad N_I . grad N_J is a
// sum of Kronecker products of the exactly integrated 1D element matrices,
//   K = ax K1 (x) M1 (x) M1 + ay M1 (x) K1 (x) M1 + az M1 (x) M1 (x) K1,
// (ax = hy hz / (2 hx), ...) and the GLL-lumped overlap is M = J mx (x) my (x) mz.  The
// kernel evaluates, output-stationary,
//   Y = alpha * ( oscale * K (S X) + (V - shift) X ) + beta * Z
// which is the Hamiltonian Ht = 1/2 M^-1/2 K M^-1/2 + V (Eq. Veff and Hloc) with the
// three-term Chebyshev update fused (S = M^-1/2, oscale = 1/2 M^-1/2), or the Poisson
// operator K (S = I, oscale = 1, no potential).
//
// Work decomposition: one CTA owns the nodes of an xy block of BX x BY cells (half-open),
// a tile of NCH vector chunks, and a range of z layers.  It sweeps the z planes in order.
// Each plane (with a p-node periodic halo in x and y), the potential and the previous
// Chebyshev iterate of the owned nodes are staged into shared memory with cp.async one
// plane ahead; the plane is contracted in y then in x (cell by cell, the shared boundary
// node taking the previous cell's last row), and the two in-plane results are accumulated
// into the p+1 output planes of the current z layer held in registers.  A layer's first p
// planes are final once its top plane is processed; the top plane's sum carries into the
// next layer.  No scatter, no atomics: every output node is written once by the thread that
// owns it, so results are bitwise reproducible.
//
// All tile dimensions are compile-time constants; each thread's staging addresses are
// computed once per launch.  CTAs are small (a few hundred threads, ~50 KB of shared
// memory) so that several share an SM and one CTA's barriers overlap another's work.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fe_gll_tables.h"
#include "fe_internal.h"

namespace fe {

// Device copy of the coefficient tables.  Rows have a stride of 8 entries, 16-byte aligned,
// so that the compiler can fetch four coefficients per constant load.
constexpr int KCS = 8;

template <typename T>
struct KronCoefT {
  alignas(16) T AyM[FE_MAXN1][KCS];
  alignas(16) T AyK[FE_MAXN1][KCS];
  alignas(16) T AxM[FE_MAXN1][KCS];
  alignas(16) T AxK[FE_MAXN1][KCS];
  // z tables with the plane's input scale folded in: AzKs[j][k] = AzK[j][k] zin / sqrt(mz_k),
  // mz_k the z mass factor of an interior plane with local index k (k = 0 and k = p: a plane
  // shared by two cells); a face plane multiplies its inputs by face_fix first
  alignas(16) T AzKs[FE_MAXN1][KCS];
  alignas(16) T AzMs[FE_MAXN1][KCS];
  T sig[FE_MAXN1];
  // 1/sqrt and sqrt of the z mass factor of a plane by local index (index 0: a plane shared
  // by two cells; *_face: the bottom or top face), so that no plane pays a division
  T rsq[FE_MAXN1], sq[FE_MAXN1];
  T rsq_face, sq_face, face_fix;
  T zout, izout;
  T ax, ay;   // in-plane stiffness scales (used with the compile-time shape tables)
  int mass_scale;
  int cplx;   // write -i (operator X) on interleaved (re, im) lanes
};

template <typename T>
inline KronCoefT<T> convert_coef(const KronCoef& c) {
  KronCoefT<T> o = {};
  double rsq[FE_MAXN1];
  for (int i = 0; i < FE_MAXN1; ++i) {
    const double mz = i == 0 ? 2.0 * c.wz[0] : c.wz[i];
    rsq[i] = c.mass_scale ? (mz > 0.0 ? 1.0 / std::sqrt(mz) : 0.0) : 1.0;
  }
  int p = 0;   // degree: the last local index with a nonzero GLL weight
  for (int i = 1; i < FE_MAXN1; ++i)
    if (c.wz[i] > 0.0) p = i;
  for (int i = 0; i < FE_MAXN1; ++i) {
    for (int j = 0; j < FE_MAXN1; ++j) {
      o.AyM[i][j] = (T)c.AyM[i][j];
      o.AyK[i][j] = (T)c.AyK[i][j];
      o.AxM[i][j] = (T)c.AxM[i][j];
      o.AxK[i][j] = (T)c.AxK[i][j];
      const double sz = c.zin * rsq[(j == p) ? 0 : j];
      o.AzKs[i][j] = (T)(c.AzK[i][j] * sz);
      o.AzMs[i][j] = (T)(c.AzM[i][j] * sz);
    }
    o.sig[i] = (T)c.sig[i];
    const double mz = i == 0 ? 2.0 * c.wz[0] : c.wz[i];
    o.rsq[i] = mz > 0.0 ? (T)(1.0 / std::sqrt(mz)) : T(0);
    o.sq[i] = (T)std::sqrt(mz > 0.0 ? mz : 0.0);
  }
  o.rsq_face = c.wz[0] > 0.0 ? (T)(1.0 / std::sqrt(c.wz[0])) : T(0);
  o.sq_face = (T)std::sqrt(c.wz[0] > 0.0 ? c.wz[0] : 0.0);
  o.face_fix = c.mass_scale ? (T)std::sqrt(2.0) : T(1);
  o.zout = (T)c.zout;
  o.izout = (T)(1.0 / c.zout);
  o.ax = (T)c.ax;
  o.ay = (T)c.ay;
  o.mass_scale = c.mass_scale;
  o.cplx = c.cplx;
  return o;
}

// A chunk is CH consecutive vector entries of one node: 16 bytes (float4 / double2) or,
// for single-vector operators, one element.  Aligned to its size so that every shared- and
// global-memory access of a chunk is one vector instruction (the block layouts guarantee
// it: 16-byte aligned blocks whose rows are a multiple of 16 bytes).
template <typename T, int CH>
struct alignas(sizeof(T) * CH) Chunk {
  T v[CH];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < CH; ++e) v[e] = T(0);
  }
  __device__ __forceinline__ void fma(T a, const Chunk& x) {
#pragma unroll
    for (int e = 0; e < CH; ++e) v[e] = fma_t(a, x.v[e], v[e]);
  }
  __device__ __forceinline__ static T fma_t(T a, T b, T c) { return a * b + c; }
};

template <>
__device__ __forceinline__ float Chunk<float, 4>::fma_t(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
// d0,d1 += c * (b0,b1): one paired FP32 FMA (the same correctly rounded fma in each lane)
__device__ __forceinline__ void ffma2(float& d0, float& d1, float c, float b0, float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %2};\n\tmov.b64 rb, {%3, %4};\n\t"
      "mov.b64 rd, {%0, %1};\n\tfma.rn.f32x2 rd, ra, rb, rd;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "+f"(d0), "+f"(d1) : "f"(c), "f"(b0), "f"(b1));
}
// float chunks accumulate two lanes per instruction
template <>
__device__ __forceinline__ void Chunk<float, 4>::fma(float a, const Chunk& x) {
  ffma2(v[0], v[1], a, x.v[0], x.v[1]);
  ffma2(v[2], v[3], a, x.v[2], x.v[3]);
}
template <>
__device__ __forceinline__ double Chunk<double, 2>::fma_t(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ double Chunk<double, 1>::fma_t(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ float Chunk<float, 1>::fma_t(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int nbytes_valid) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(nbytes_valid));
  } else if constexpr (BYTES == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(nbytes_valid));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(nbytes_valid));
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// compile-time tile shape
template <int P_, int BX_, int BY_, int NCH_, int NTHR_>
struct KronTileT {
  static constexpr int P = P_, BX = BX_, BY = BY_, NCH = NCH_, NTHR = NTHR_;
  static constexpr int BXn = BX * P, BYn = BY * P;
  static constexpr int BXH = BXn + P + 1, BYH = BYn + P + 1;
  static constexpr int NZI = BXn * BYn * NCH;            // output items (node, chunk)
  static constexpr int IPT = (NZI + NTHR - 1) / NTHR;    // output items per thread
  static constexpr int NST = BYH * BXH * NCH;            // staged chunks per plane
  static constexpr int SPT = (NST + NTHR - 1) / NTHR;    // staged chunks per thread
  static constexpr int NYI = BXH * NCH * BY;             // y-phase items (cell segments)
  static constexpr int NXI = BYn * NCH * BX;             // x-phase items (cell segments)
  static constexpr int ZR = P + 2;                       // ring of staged Chebyshev planes
  // stage (and V) slots: plane gz + 2 is staged while other threads may still read plane gz
  // after the plane's last barrier, so three slots keep those reads race-free
  static constexpr int NSB = 3;
  // row strides (in nodes) of the in-plane intermediates, odd so that the x phase's
  // column-wise accesses (consecutive threads on consecutive rows) fall in distinct banks
  static constexpr int ARS = BXH | 1;
  static constexpr int WRS = BXn | 1;
};

// One CTA's work: xy block bxy (x fastest), vector tile vti, z segment zsi.
// FULL: every xy block is complete and every vector tile full, so no ownership, edge or
// ragged-vector test is needed anywhere in the sweep.
// CT (float Hamiltonian): the in-plane contractions take the shape-only tables M1 sig and
// K1 sig as compile-time constants (FFMA immediates instead of constant-bank loads) and apply
// the mesh scales ay, ax as one multiply per y output and one FMA per x output.
template <typename T, int CH, class TL, bool FULL, bool CT>
__device__ __forceinline__ void kron_body(const KronCoefT<T>& cf, const KronGeom& g,
                                          const KronIO<T>& io, int bxy, int vti, int zsi) {
  using C = Chunk<T, CH>;
  constexpr int P = TL::P, NCH = TL::NCH, BXn = TL::BXn, BYn = TL::BYn;
  constexpr int BXH = TL::BXH, NTHR = TL::NTHR, IPT = TL::IPT;
  constexpr int ARS = TL::ARS, WRS = TL::WRS;
  constexpr int NZI = TL::NZI, NST = TL::NST, SPT = TL::SPT;
  constexpr int CHB = CH * (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* stage0 = reinterpret_cast<C*>(smem_raw);                  // [NSB][BYH][BXH][NCH]
  C* A = stage0 + TL::NSB * NST;                               // [BYn][ARS][NCH]
  C* B = A + BYn * ARS * NCH;
  C* W1 = B + BYn * ARS * NCH;                                 // [BYn][WRS][NCH]
  C* W2 = W1 + BYn * WRS * NCH;
  C* Zr = W2 + BYn * WRS * NCH;                                // [ZR][BYn][BXn][NCH]
  // the shape-table variants are launched for the mass-scaled Hamiltonian only
  const bool mass_scale = CT || cf.mass_scale;
  const bool use_z = io.Z != nullptr;                          // (beta != 0 by launch)
  const bool use_v = io.V != nullptr;
  T* Vs = reinterpret_cast<T*>(Zr + (use_z ? TL::ZR * NZI : 0));   // [NSB][BYn][BXn]

  const int tid = threadIdx.x;
  const int bxi = bxy % g.nbx, byi = bxy / g.nbx;
  const int x0 = bxi * BXn, y0 = byi * BYn;
  const int64_t vt0 = (int64_t)vti * NCH * CH;
  const int c0 = zsi * g.zseg;
  const int c1 = min(c0 + g.zseg, g.nz);
  const int cb = c0 > 0 ? c0 - 1 : 0;
  const int gbeg = cb * P, gend = c1 * P;
  const int64_t plane_nodes = (int64_t)g.NX * g.NY;

  // ---- staging addresses (per thread, once) ---------------------------------------------
  int64_t s_goff[SPT];
  int s_bytes[SPT];
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    const int e = tid + i * NTHR;
    const int ec = e < NST ? e : 0;
    const int ch = ec % NCH, node = ec / NCH;
    const int xh = node % BXH, yh = node / BXH;
    const int gx = pmod(x0 - P + xh, g.NX), gy = pmod(y0 - P + yh, g.NY);
    const int64_t v0 = vt0 + (int64_t)ch * CH;
    const int64_t rem = io.nvec - v0;
    s_bytes[i] = e >= NST ? -1
                          : (FULL ? CHB : (rem <= 0 ? 0 : (rem >= CH ? CHB : (int)(rem * sizeof(T)))));
    s_goff[i] = (gx + (int64_t)g.NX * gy) * io.ldx + v0;
  }

  // ---- the thread's output items ---------------------------------------------------------
  int it_x[IPT], it_y[IPT], it_ch[IPT];
  bool it_own[IPT];
  int64_t it_node[IPT];     // in-plane node index of the output
  int64_t it_yo[IPT];       // offset of the item's entries in a plane of Y
  T it_sxy[IPT], it_isxy[IPT];
  int it_w[IPT], it_v[IPT], it_s[IPT];   // the item's offsets in W1 / W2, a V plane, a stage
  C acc[IPT][P + 1];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int item = tid + i * NTHR;
    const bool valid = item < NZI;
    const int itc = valid ? item : 0;
    it_ch[i] = itc % NCH;
    const int node = itc / NCH;
    it_x[i] = node % BXn;
    it_y[i] = node / BXn;
    const int64_t v0 = vt0 + (int64_t)it_ch[i] * CH;
    it_own[i] = valid && (FULL || ((x0 + it_x[i] < g.NX) && (y0 + it_y[i] < g.NY) && (v0 < io.nvec)));
    it_node[i] = (x0 + it_x[i]) + (int64_t)g.NX * (y0 + it_y[i]);
    it_yo[i] = it_node[i] * io.ldy + v0;
    it_sxy[i] = mass_scale ? cf.sig[it_x[i] % P] * cf.sig[it_y[i] % P] : T(1);
    it_isxy[i] = T(1) / it_sxy[i];
    it_w[i] = (it_y[i] * TL::WRS + it_x[i]) * NCH + it_ch[i];
    it_v[i] = it_y[i] * BXn + it_x[i];
    it_s[i] = ((it_y[i] + P) * BXH + (it_x[i] + P)) * NCH + it_ch[i];
#pragma unroll
    for (int j = 0; j <= P; ++j) acc[i][j].zero();
  }

  auto stored = [&](int gz) { return gz - g.gz_lo >= 0 && gz - g.gz_lo < g.NZs; };
  auto owned_plane = [&](int gz) {   // planes this segment writes
    return stored(gz) && ((gz >= c0 * P && gz < c1 * P) || (gz == g.nz * P && c1 == g.nz));
  };

  // stage plane gz: the halo block of X into the stage buffer, V and the Chebyshev operand
  // of the owned nodes into their rings
  // (called for gz = gbeg, gbeg + 1, ... in order: offsets and ring slots advance by one plane)
  int64_t st_xoff = (int64_t)(gbeg - g.gz_lo) * plane_nodes * io.ldx;
  const int64_t st_xstride = plane_nodes * io.ldx;
  int st_slot = 0;                   // (gz - gbeg) % NSB of the plane to stage
  int st_zslot = gbeg % TL::ZR;      // gz % ZR of the plane to stage
  // the thread's V node and Z chunk offsets within a plane, and their plane offsets
  int64_t st_voff = (int64_t)(gbeg - g.gz_lo) * plane_nodes;
  int64_t st_zoff = st_voff * io.ldz;
  const int64_t st_zstride = plane_nodes * io.ldz;
  int64_t v_in = 0;
  bool v_ok = false;
  if (tid < BXn * BYn) {
    const int x = tid % BXn, y = tid / BXn;
    v_ok = FULL || (x0 + x < g.NX && y0 + y < g.NY);
    v_in = (x0 + x) + (int64_t)g.NX * (y0 + y);
  }
  int64_t z_in[IPT];
  int z_nb[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int64_t v0 = vt0 + (int64_t)it_ch[i] * CH;
    const int64_t rem = io.nvec - v0;
    z_nb[i] = !it_own[i] ? 0 : (FULL ? CHB : (rem <= 0 ? 0 : (rem >= CH ? CHB : (int)(rem * sizeof(T)))));
    z_in[i] = it_node[i] * io.ldz + v0;
  }
  auto stage_plane = [&](int gz) {
    const int64_t pbase = st_xoff, vbase = st_voff, zbase = st_zoff;
    const int sslot = st_slot, zslot = st_zslot;
    st_xoff += st_xstride;
    st_voff += plane_nodes;
    st_zoff += st_zstride;
    st_slot = st_slot + 1 == TL::NSB ? 0 : st_slot + 1;
    st_zslot = st_zslot + 1 == TL::ZR ? 0 : st_zslot + 1;
    if (!stored(gz)) return;
    C* dst = stage0 + sslot * NST;
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      const int e = tid + i * NTHR;
      if constexpr (FULL && NST % NTHR == 0) {
        // full tile, every thread stages SPT whole chunks
        cp_async<CHB>(dst + e, io.X + pbase + s_goff[i], CHB);
      } else {
        if (s_bytes[i] > 0) cp_async<CHB>(dst + e, io.X + pbase + s_goff[i], s_bytes[i]);
        else if (s_bytes[i] == 0) cp_async<CHB>(dst + e, io.X, 0);
      }
    }
    if (use_v && tid < BXn * BYn) {
      T* vd = Vs + sslot * (BXn * BYn) + tid;
      if constexpr (FULL)
        cp_async<(int)sizeof(T)>(vd, io.V + vbase + v_in, (int)sizeof(T));
      else
        cp_async<(int)sizeof(T)>(vd, v_ok ? io.V + vbase + v_in : io.V, v_ok ? (int)sizeof(T) : 0);
    }
    if (use_z && owned_plane(gz)) {
      C* zd = Zr + zslot * NZI;
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const int item = tid + i * NTHR;
        if (item >= NZI) continue;
        if constexpr (FULL) {
          cp_async<CHB>(zd + item, io.Z + zbase + z_in[i], CHB);
        } else {
          const int nb = z_nb[i];
          const T* src = nb ? io.Z + zbase + z_in[i] : io.Z;
          cp_async<CHB>(zd + item, src, nb);
        }
      }
    }
  };

  // write the final value of output plane gzo held in acc[i][j]
  // layer c's bottom plane c P: its Z ring slot (c P) % ZR
  int wr_zbase = (cb * P) % TL::ZR;
  auto write_plane = [&](int gzo, int j) {
    if (!owned_plane(gzo)) return;
    const int zs = gzo - g.gz_lo;
    T rs = T(1);   // 1 / sqrt(mz) of the plane (local index j; 1 for the plain stiffness)
    if (mass_scale)
      rs = j != 0 ? cf.rsq[j] : ((gzo == 0 || gzo == g.nz * P) ? cf.rsq_face : cf.rsq[0]);
    const T ps = cf.zout * rs;
    int zsl = wr_zbase + j;
    zsl -= zsl >= TL::ZR ? TL::ZR : 0;
    const C* zsrc = Zr + zsl * NZI;
    T* yplane = io.Y + (int64_t)zs * plane_nodes * io.ldy;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (!it_own[i]) continue;
      const int64_t v0 = vt0 + (int64_t)it_ch[i] * CH;
      const T sc = io.alpha * ps * it_sxy[i];
      C out;
      // (the shape-table variants are launched for the real operator only)
      if (!CT && cf.cplx) {
        // -i (a + i b) = b - i a on each (re, im) lane pair (even chunk widths only)
        out.zero();
#pragma unroll
        for (int e = 0; e + 1 < CH; e += 2) {
          out.v[e] = sc * acc[i][j].v[e + 1];
          out.v[e + 1] = -sc * acc[i][j].v[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e) out.v[e] = sc * acc[i][j].v[e];
      }
      if (use_z) {
        const C zc = zsrc[tid + i * NTHR];
#pragma unroll
        for (int e = 0; e < CH; ++e) out.v[e] = C::fma_t(io.beta, zc.v[e], out.v[e]);
      }
      T* yp = yplane + it_yo[i];
      if (FULL || v0 + CH <= io.nvec) {
        *reinterpret_cast<C*>(yp) = out;
      } else {
        for (int e = 0; e < CH; ++e)
          if (v0 + e < io.nvec) yp[e] = out.v[e];
      }
    }
  };

  // Plane with local index K (compile time, so every coefficient is an immediate operand):
  // the potential term of the plane's own nodes (when pot) and the z contraction of its
  // in-plane results into the layer accumulators.
  auto plane_z = [&](auto kc, bool pot, bool face, T inv_ps, const T* vv, const C* st,
                     const C* w1, const C* w2) {
    constexpr int K = decltype(kc)::value;
    if constexpr (K <= P) {
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        if (pot && it_own[i]) {
          const T pv = (vv[it_v[i]] - io.shift) * inv_ps * it_isxy[i];
          const C xs = st[it_s[i]];
          acc[i][K].fma(pv, xs);
        }
        C a = w1[i], b = w2[i];
#pragma unroll
        if (face) {
#pragma unroll
          for (int e = 0; e < CH; ++e) { a.v[e] *= cf.face_fix; b.v[e] *= cf.face_fix; }
        }
#pragma unroll
        for (int j = 0; j <= P; ++j) {
          acc[i][j].fma(cf.AzKs[j][K], a);
          acc[i][j].fma(cf.AzMs[j][K], b);
        }
      }
    }
  };
  auto dispatch_z = [&](int k, bool pot, bool face, T inv_ps, const T* vv, const C* st,
                        const C* w1, const C* w2) {
    switch (k) {
      case 0: plane_z(std::integral_constant<int, 0>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 1: plane_z(std::integral_constant<int, 1>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 2: plane_z(std::integral_constant<int, 2>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 3: plane_z(std::integral_constant<int, 3>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 4: plane_z(std::integral_constant<int, 4>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 5: plane_z(std::integral_constant<int, 5>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      case 6: plane_z(std::integral_constant<int, 6>{}, pot, face, inv_ps, vv, st, w1, w2); break;
      default: break;
    }
  };

  auto shift_layer = [&]() {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      acc[i][0] = acc[i][P];
#pragma unroll
      for (int j = 1; j <= P; ++j) acc[i][j].zero();
    }
  };

  // in-plane 1D coefficients: the mesh's tables, or (CT) the compile-time shape tables
  auto cYM = [&](int j, int k) -> T {
    if constexpr (CT) return (T)gll_ms<P>(j, k); else return cf.AyM[j][k];
  };
  auto cYK = [&](int j, int k) -> T {
    if constexpr (CT) return (T)gll_ks<P>(j, k); else return cf.AyK[j][k];
  };
  auto cXM = [&](int j, int k) -> T {
    if constexpr (CT) return (T)gll_ms<P>(j, k); else return cf.AxM[j][k];
  };
  auto cXK = [&](int j, int k) -> T {
    if constexpr (CT) return (T)gll_ks<P>(j, k); else return cf.AxK[j][k];
  };

  // scalar-lane items of the in-plane phases (used when each thread has at most one)
  constexpr int NL = NCH * CH;
  int y_ibase = 0, y_obase = 0, x_ibase = 0, x_obase = 0;
  {
    const int l = tid % NL, r = tid / NL;
    const int xh = r % BXH, yb = (r / BXH) * P;
    y_ibase = (yb * BXH + xh) * NL + l;
    y_obase = (yb * ARS + xh) * NL + l;
    const int y = r % BYn, xb = (r / BYn) * P;
    x_ibase = y * ARS * NL + xb * NL + l;
    x_obase = (y * WRS + xb) * NL + l;
  }

  // ---- sweep -----------------------------------------------------------------------------
  stage_plane(gbeg);
  cp_commit();
  int c = cb;
  int cur_slot = 0;   // (gz - gbeg) % NSB
  for (int gz = gbeg; gz <= gend; ++gz, cur_slot = cur_slot + 1 == TL::NSB ? 0 : cur_slot + 1) {
    const int k = gz - c * P;
    if (gz < gend) {
      stage_plane(gz + 1);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const C* st = stage0 + cur_slot * NST;

    if (stored(gz)) {
      // The two in-plane phases run on scalar lanes: an item is one cell segment of one
      // vector entry, so that every thread has work (a chunk-wide item would leave most of
      // the CTA idle at the following barrier).  NL scalars per node, lane-fastest indexing
      // keeps consecutive threads on consecutive words.
      using S1 = Chunk<T, 1>;
      const S1* sts = reinterpret_cast<const S1*>(st);
      S1* As = reinterpret_cast<S1*>(A);
      S1* Bs = reinterpret_cast<S1*>(B);
      // phase Y: a = AyM U, b = AyK U along y for every halo x
      auto phase_y = [&](int ibase, int obase) {
        S1 own[P + 1], prv[P];
#pragma unroll
        for (int kk = 0; kk <= P; ++kk) own[kk] = sts[ibase + (P + kk) * BXH * NL];
#pragma unroll
        for (int kk = 0; kk < P; ++kk) prv[kk] = sts[ibase + kk * BXH * NL];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          S1 a, b;
          a.zero();
          b.zero();
#pragma unroll
          for (int kk = 0; kk <= P; ++kk) {
            a.fma(cYM(j, kk), own[kk]);
            b.fma(cYK(j, kk), own[kk]);
          }
          if (j == 0) {
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
              a.fma(cYM(P, kk), prv[kk]);
              b.fma(cYK(P, kk), prv[kk]);
            }
            a.fma(cYM(P, P), own[0]);
            b.fma(cYK(P, P), own[0]);
          }
          if constexpr (CT) b.v[0] *= cf.ay;
          As[obase + j * ARS * NL] = a;
          Bs[obase + j * ARS * NL] = b;
        }
      };
      if constexpr (TL::NYI * CH == NTHR) {
        phase_y(y_ibase, y_obase);
      } else if constexpr (TL::NYI * CH <= NTHR) {
        if (tid < TL::NYI * CH) phase_y(y_ibase, y_obase);
      } else {
#pragma unroll 1
        for (int e = tid; e < TL::NYI * CH; e += NTHR) {
          const int l = e % NL, r = e / NL, xh = r % BXH, yb = (r / BXH) * P;
          phase_y((yb * BXH + xh) * NL + l, (yb * ARS + xh) * NL + l);
        }
      }
      __syncthreads();
      // phase X: W1 = AxM a, W2 = AxK a + AxM b along x for every owned y
      {
        S1* W1s = reinterpret_cast<S1*>(W1);
        S1* W2s = reinterpret_cast<S1*>(W2);
        auto phase_x = [&](int ibase, int obase) {
          const S1* arow = As + ibase;
          const S1* brow = Bs + ibase;
          S1 ao[P + 1], bo[P + 1];
#pragma unroll
          for (int kk = 0; kk <= P; ++kk) {
            ao[kk] = arow[(P + kk) * NL];
            bo[kk] = brow[(P + kk) * NL];
          }
#pragma unroll
          for (int j = 0; j < P; ++j) {
            S1 u, v, vk;   // (CT: v gathers M1 sig b, vk gathers K1 sig a, scaled by ax)
            u.zero();
            v.zero();
            vk.zero();
            S1& vka = CT ? vk : v;
#pragma unroll
            for (int kk = 0; kk <= P; ++kk) {
              u.fma(cXM(j, kk), ao[kk]);
              vka.fma(cXK(j, kk), ao[kk]);
              v.fma(cXM(j, kk), bo[kk]);
            }
            if (j == 0) {
#pragma unroll
              for (int kk = 0; kk < P; ++kk) {
                const S1 ap = arow[kk * NL];
                const S1 bp = brow[kk * NL];
                u.fma(cXM(P, kk), ap);
                vka.fma(cXK(P, kk), ap);
                v.fma(cXM(P, kk), bp);
              }
              u.fma(cXM(P, P), ao[0]);
              vka.fma(cXK(P, P), ao[0]);
              v.fma(cXM(P, P), bo[0]);
            }
            if constexpr (CT) v.fma(cf.ax, vk);
            W1s[obase + j * NL] = u;
            W2s[obase + j * NL] = v;
          }
        };
        if constexpr (TL::NXI * CH <= NTHR) {
          if (tid < TL::NXI * CH) phase_x(x_ibase, x_obase);
        } else {
#pragma unroll 1
          for (int e = tid; e < TL::NXI * CH; e += NTHR) {
            const int l = e % NL, r = e / NL, y = r % BYn, xb = (r / BYn) * P;
            phase_x(y * ARS * NL + xb * NL + l, (y * WRS + xb) * NL + l);
          }
        }
      }
      __syncthreads();
      C w1[IPT], w2[IPT];
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const int item = it_w[i];
        w1[i] = W1[item];
        w2[i] = W2[item];
      }
      const bool face = gz == 0 || gz == g.nz * P;
      T sqz = T(1);   // sqrt(mz) of the plane (1 for the plain stiffness)
      if (mass_scale) {
        const int l = k == P ? 0 : k;   // gz % P
        sqz = l != 0 ? cf.sq[l] : (face ? cf.sq_face : cf.sq[0]);
      }
      const T inv_ps = sqz * cf.izout;
      const T* vv = Vs + cur_slot * (BXn * BYn);
      dispatch_z(k, use_v, face, inv_ps, vv, st, w1, w2);
      if (k == P) {
        // the layer is complete: its first P planes are final; the top plane's sum
        // becomes the bottom accumulator of the next layer
#pragma unroll
        for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
        shift_layer();
        ++c;
        wr_zbase += P;
        wr_zbase -= wr_zbase >= TL::ZR ? TL::ZR : 0;
        if (c < c1) dispatch_z(0, false, face, inv_ps, vv, st, w1, w2);
      }
    } else if (k == P) {
      // an unstored (homogeneous Dirichlet) plane contributes nothing
#pragma unroll
      for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
      shift_layer();
      ++c;
      wr_zbase += P;
      wr_zbase -= wr_zbase >= TL::ZR ? TL::ZR : 0;
    }
  }
  // the last processed plane (gend = c1 P) is final only if it is the top face
  write_plane(gend, 0);
}

// 1D grid, vector tile fastest: the CTAs that read the other halves of a node's DRAM
// bursts (neighbouring vector tiles of the same xy block) run side by side, so a burst is
// fetched once; neighbouring xy blocks (halo sharing) follow within the resident window.
// the float block operator (four-lane chunks) takes the compile-time shape tables
template <typename T, int CH>
struct KronShapeTables {
  static constexpr bool value = std::is_same<T, float>::value && CH == 4;
};

// Residency bound: the float operator's tiles of up to 256 threads are held to three CTAs per
// SM (at most 85 registers), where the per-plane barriers of one CTA overlap two others' work.
template <typename T, int CH, class TL>
struct KronMinBlocks {
  static constexpr int value = (std::is_same<T, float>::value && CH == 4 && TL::NTHR <= 256) ? 3 : 1;
};

template <typename T, int CH, class TL, bool FULL, bool CT>
__global__ void __launch_bounds__(TL::NTHR, (KronMinBlocks<T, CH, TL>::value))
kron_kernel(const KronCoefT<T> cf, const KronGeom g, const KronIO<T> io, int nvt) {
  const int b = blockIdx.x;
  const int nxy = g.nbx * g.nby;
  const int r = b / nvt;
  kron_body<T, CH, TL, FULL, CT>(cf, g, io, r % nxy, b % nvt, r / nxy);
}

// Batched form: many independent meshes that share p and the cell size (so one coefficient
// table) in one launch.  The 1D grid concatenates the instances' CTA grids; a CTA finds its
// instance by binary search over the ascending first-CTA offsets.
template <typename T, int CH, class TL, bool FULL, bool CT>
__global__ void __launch_bounds__(TL::NTHR, (KronMinBlocks<T, CH, TL>::value))
kron_batch_kernel(const KronCoefT<T> cf, const KronInst<T>* __restrict__ inst, int ninst) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].cta0 <= b) lo = mid; else hi = mid - 1;
  }
  const KronGeom g = inst[lo].g;
  const KronIO<T> io = inst[lo].io;
  const int64_t local = b - inst[lo].cta0;
  const int nxy = g.nbx * g.nby;
  const int64_t nvt = inst[lo].nvt;
  const int64_t r = local / nvt;
  kron_body<T, CH, TL, FULL, CT>(cf, g, io, (int)(r % nxy), (int)(local % nvt), (int)(r / nxy));
}

// Persistent batched form: a grid of resident CTAs takes the batch's work items (the CTAs of
// the one-CTA-per-item grid above) from a device counter, so that the items of tall and
// short instances spread over the SMs as they finish (dynamic load balance for uneven slab
// heights).  The counter starts at zero for each launch.
template <typename T, int CH, class TL, bool FULL, bool CT>
__global__ void __launch_bounds__(TL::NTHR, (KronMinBlocks<T, CH, TL>::value))
kron_batch_persist_kernel(const KronCoefT<T> cf, const KronInst<T>* __restrict__ inst, int ninst,
                          int64_t total, unsigned long long* __restrict__ counter) {
  __shared__ long long s_item;
  for (;;) {
    __syncthreads();   // every thread is done with the previous item's shared memory
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t b = s_item;
    if (b >= total) break;
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (inst[mid].cta0 <= b) lo = mid; else hi = mid - 1;
    }
    const KronGeom g = inst[lo].g;
    const KronIO<T> io = inst[lo].io;
    const int64_t local = b - inst[lo].cta0;
    const int nxy = g.nbx * g.nby;
    const int64_t nvt = inst[lo].nvt;
    const int64_t r = local / nvt;
    kron_body<T, CH, TL, FULL, CT>(cf, g, io, (int)(r % nxy), (int)(local % nvt), (int)(r / nxy));
  }
}

// Dynamic shared memory limit, and the largest shared-memory carveout so that the residency
// of these kernels is set by registers and their own shared memory, not by the L1 split.
template <typename K>
inline fe_status kron_func_setup(K kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fe_fail(FE_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  }
  return FE_OK;
}

// shared memory of one CTA
template <typename T, int CH, class TL>
inline size_t kron_smem(bool use_z, bool use_v) {
  const size_t cb = sizeof(Chunk<T, CH>);
  size_t s = cb * (TL::NSB * (size_t)TL::NST + 2 * (size_t)TL::BYn * TL::ARS * TL::NCH +
                   2 * (size_t)TL::BYn * TL::WRS * TL::NCH);
  if (use_z) s += cb * TL::ZR * (size_t)TL::NZI;
  if (use_v) s += sizeof(T) * TL::NSB * (size_t)TL::BXn * TL::BYn;
  return s;
}

template <typename T, int CH, class TL>
fe_status kron_launch_t(const KronCoef& cf, const KronGeom& g, const KronIO<T>& io,
                        cudaStream_t st) {
  if (g.bx != TL::BX || g.by != TL::BY) return fe_fail(FE_EINVAL, "tile shape mismatch");
  KronIO<T> io2 = io;
  if (io2.Z != nullptr && io2.beta == T(0)) io2.Z = nullptr;
  const size_t smem = kron_smem<T, CH, TL>(io2.Z != nullptr, io2.V != nullptr);
  if (smem > 227 * 1024) return fe_fail(FE_EINVAL, "tile needs %zu bytes of shared memory", smem);
  const int64_t vtile = (int64_t)TL::NCH * CH;
  const bool full = g.NX % TL::BXn == 0 && g.NY % TL::BYn == 0 && io.nvec % vtile == 0;
  auto kern = full ? kron_kernel<T, CH, TL, true, false> : kron_kernel<T, CH, TL, false, false>;
  if constexpr (KronShapeTables<T, CH>::value) {
    if (cf.mass_scale && !cf.cplx)
      kern = full ? kron_kernel<T, CH, TL, true, true> : kron_kernel<T, CH, TL, false, true>;
  }
  if (cf.cplx && (CH % 2 != 0 || io.nvec % 2 != 0))
    return fe_fail(FE_EINVAL, "complex operator needs interleaved (re, im) lane pairs");
  FE_TRY(kron_func_setup(kern, smem));
  const int64_t nvt = (io.nvec + vtile - 1) / vtile;
  const int64_t total = (int64_t)g.nbx * g.nby * nvt * ((g.nz + g.zseg - 1) / g.zseg);
  if (total > 0x7fffffffLL || nvt > 0x7fffffffLL) return fe_fail(FE_EINVAL, "grid too large");
  KronCoefT<T> cft = convert_coef<T>(cf);
  kern<<<(unsigned)total, TL::NTHR, smem, st>>>(cft, g, io2, (int)nvt); fe_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "kron kernel launch: %s", cudaGetErrorString(e));
  return FE_OK;
}

// cells per block side for each p: about ten nodes per side
template <int P>
struct KronBlock {
  static constexpr int B = P == 1 ? 8 : P == 2 ? 5 : P == 3 ? 3 : 2;
};

// threads: enough for one output item (node, chunk) and one y-phase scalar item each
template <int P, int NCH, int CH>
struct KronTileFor {
  static constexpr int B = KronBlock<P>::B;
  static constexpr int NZ_ITEMS = B * P * B * P * NCH;
  static constexpr int NY_ITEMS = (B * P + P + 1) * B * NCH * CH;
  static constexpr int N = NZ_ITEMS > NY_ITEMS ? NZ_ITEMS : NY_ITEMS;
  static constexpr int NTHR = (N + 31) / 32 * 32 > 512 ? 512 : (N + 31) / 32 * 32;
  using type = KronTileT<P, B, B, NCH, NTHR>;
};

}  // namespace fe

namespace fe {

inline int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// fill the block grid and the z segmentation for tile TL, then launch
template <typename T, int CH, class TL>
fe_status kron_go(const KronCoef& cf, KronGeom g, const KronIO<T>& io, cudaStream_t st) {
  g.bx = TL::BX;
  g.by = TL::BY;
  const int nx = g.NX / g.p, ny = g.NY / g.p;
  g.nbx = (nx + TL::BX - 1) / TL::BX;
  g.nby = (ny + TL::BY - 1) / TL::BY;
  const int64_t vt = (io.nvec + (int64_t)TL::NCH * CH - 1) / ((int64_t)TL::NCH * CH);
  const int64_t base = (int64_t)g.nbx * g.nby * vt;
  const int64_t want = 4 * (int64_t)device_sms();
  int zseg = g.nz;
  while (zseg > 2 && base * ((g.nz + zseg - 1) / zseg) < want) zseg = (zseg + 1) / 2;
  g.zseg = zseg;
  return kron_launch_t<T, CH, TL>(cf, g, io, st);
}

// batched plan: every instance gets tile TL; z segments are split (uniformly) only while the
// whole batch has fewer than four CTAs per SM, or have the requested length zseg_req > 0
template <typename T, int CH, class TL>
int64_t kron_batch_plan_t(KronInst<T>* inst, int n, int zseg_req) {
  int nzmax = 1;
  for (int i = 0; i < n; ++i) {
    KronGeom& g = inst[i].g;
    g.bx = TL::BX;
    g.by = TL::BY;
    g.nbx = (g.NX / g.p + TL::BX - 1) / TL::BX;
    g.nby = (g.NY / g.p + TL::BY - 1) / TL::BY;
    inst[i].nvt = (inst[i].io.nvec + (int64_t)TL::NCH * CH - 1) / ((int64_t)TL::NCH * CH);
    inst[i].full = g.NX % TL::BXn == 0 && g.NY % TL::BYn == 0 &&
                   inst[i].io.nvec % ((int64_t)TL::NCH * CH) == 0;
    nzmax = g.nz > nzmax ? g.nz : nzmax;
  }
  const int64_t want = 4 * (int64_t)device_sms();
  auto total_for = [&](int zseg) {
    int64_t t = 0;
    for (int i = 0; i < n; ++i) {
      const KronGeom& g = inst[i].g;
      t += (int64_t)g.nbx * g.nby * inst[i].nvt * ((g.nz + zseg - 1) / zseg);
    }
    return t;
  };
  int zseg = nzmax;
  if (zseg_req > 0) zseg = zseg_req < nzmax ? zseg_req : nzmax;
  else
    while (zseg > 2 && total_for(zseg) < want) zseg = (zseg + 1) / 2;
  int64_t cta = 0;
  for (int i = 0; i < n; ++i) {
    KronGeom& g = inst[i].g;
    g.zseg = zseg;
    inst[i].cta0 = cta;
    cta += (int64_t)g.nbx * g.nby * inst[i].nvt * ((g.nz + zseg - 1) / zseg);
  }
  return cta;
}

template <typename T, int CH, class TL>
fe_status kron_batch_launch_t(const KronCoef& cf, const KronInst<T>* d_inst, int n,
                              int64_t total, bool use_z, bool full, cudaStream_t st,
                              unsigned long long* counter) {
  const size_t smem = kron_smem<T, CH, TL>(use_z, true);
  if (smem > 227 * 1024) return fe_fail(FE_EINVAL, "tile needs %zu bytes of shared memory", smem);
  if (total < 1 || total > 0x7fffffffLL) return fe_fail(FE_EINVAL, "batched grid of %lld CTAs", (long long)total);
  const bool ct = KronShapeTables<T, CH>::value && cf.mass_scale && !cf.cplx;
  KronCoefT<T> cft = convert_coef<T>(cf);
  if (counter) {
    // persistent grid: as many CTAs as stay resident, each taking items from the counter
    auto kern = full ? kron_batch_persist_kernel<T, CH, TL, true, false>
                     : kron_batch_persist_kernel<T, CH, TL, false, false>;
    if constexpr (KronShapeTables<T, CH>::value) {
      if (ct) kern = full ? kron_batch_persist_kernel<T, CH, TL, true, true>
                          : kron_batch_persist_kernel<T, CH, TL, false, true>;
    }
    FE_TRY(kron_func_setup(kern, smem));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TL::NTHR, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    const int64_t grid = std::min<int64_t>(total, (int64_t)per_sm * device_sms());
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st) != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ECUDA, "batched kron: counter reset failed");
    }
    kern<<<(unsigned)grid, TL::NTHR, smem, st>>>(cft, d_inst, n, total, counter); fe_count_launch();
  } else {
    auto kern = full ? kron_batch_kernel<T, CH, TL, true, false> : kron_batch_kernel<T, CH, TL, false, false>;
    if constexpr (KronShapeTables<T, CH>::value) {
      if (ct) kern = full ? kron_batch_kernel<T, CH, TL, true, true> : kron_batch_kernel<T, CH, TL, false, true>;
    }
    FE_TRY(kron_func_setup(kern, smem));
    kern<<<(unsigned)total, TL::NTHR, smem, st>>>(cft, d_inst, n); fe_count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "batched kron launch: %s", cudaGetErrorString(e));
  return FE_OK;
}

template <typename T, int CH, int NCH>
int64_t kron_batch_plan_dispatch(int p, KronInst<T>* inst, int n, int zseg_req) {
  switch (p) {
    case 1: return kron_batch_plan_t<T, CH, typename KronTileFor<1, NCH, CH>::type>(inst, n, zseg_req);
    case 2: return kron_batch_plan_t<T, CH, typename KronTileFor<2, NCH, CH>::type>(inst, n, zseg_req);
    case 3: return kron_batch_plan_t<T, CH, typename KronTileFor<3, NCH, CH>::type>(inst, n, zseg_req);
    case 4: return kron_batch_plan_t<T, CH, typename KronTileFor<4, NCH, CH>::type>(inst, n, zseg_req);
    case 5: return kron_batch_plan_t<T, CH, typename KronTileFor<5, NCH, CH>::type>(inst, n, zseg_req);
    case 6: return kron_batch_plan_t<T, CH, typename KronTileFor<6, NCH, CH>::type>(inst, n, zseg_req);
    default: return -1;
  }
}

template <typename T, int CH, int NCH>
fe_status kron_batch_dispatch(const KronCoef& cf, int p, const KronInst<T>* d_inst, int n,
                              int64_t total, bool use_z, bool full, cudaStream_t st,
                              unsigned long long* counter) {
  switch (p) {
#define FE_BCASE(pp)                                                                      \
  case pp:                                                                                \
    return kron_batch_launch_t<T, CH, typename KronTileFor<pp, NCH, CH>::type>(cf, d_inst, n, \
                                                                          total, use_z, full, st, counter);
    FE_BCASE(1) FE_BCASE(2) FE_BCASE(3) FE_BCASE(4) FE_BCASE(5) FE_BCASE(6)
#undef FE_BCASE
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", p);
  }
}

template <typename T, int CH, int NCH>
fe_status kron_dispatch(const KronCoef& cf, const KronGeom& g, const KronIO<T>& io,
                        cudaStream_t st) {
  switch (g.p) {
    case 1: return kron_go<T, CH, typename KronTileFor<1, NCH, CH>::type>(cf, g, io, st);
    case 2: return kron_go<T, CH, typename KronTileFor<2, NCH, CH>::type>(cf, g, io, st);
    case 3: return kron_go<T, CH, typename KronTileFor<3, NCH, CH>::type>(cf, g, io, st);
    case 4: return kron_go<T, CH, typename KronTileFor<4, NCH, CH>::type>(cf, g, io, st);
    case 5: return kron_go<T, CH, typename KronTileFor<5, NCH, CH>::type>(cf, g, io, st);
    case 6: return kron_go<T, CH, typename KronTileFor<6, NCH, CH>::type>(cf, g, io, st);
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", g.p);
  }
}

}  // namespace fe

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
// Work decomposition: one CTA owns an xy block of bx x by cells' nodes (half-open), a tile
// of vectors, and a range of z layers.  It sweeps the z planes in order; each plane (with a
// p-node halo in x and y, periodic wrap) is staged into shared memory with cp.async one
// plane ahead, contracted in y then in x in shared memory (cell by cell, the shared
// boundary node taking the previous cell's last row), and the two in-plane results are
// accumulated into the p+1 output planes of the current z layer held in registers.  A
// layer's first p planes are final once its top plane is processed; the top plane's sum
// carries into the next layer.  No scatter, no atomics: every output node is written once
// by the thread that owns it, so results are bitwise reproducible.
#pragma once

#include "fe_internal.h"

namespace fe {

template <typename T>
struct KronCoefT {
  T AyM[FE_MAXN1][FE_MAXN1], AyK[FE_MAXN1][FE_MAXN1];
  T AxM[FE_MAXN1][FE_MAXN1], AxK[FE_MAXN1][FE_MAXN1];
  T AzK[FE_MAXN1][FE_MAXN1], AzM[FE_MAXN1][FE_MAXN1];
  T sig[FE_MAXN1];
  T wz[FE_MAXN1];
  T zin, zout;
  int mass_scale;
};

template <typename T>
inline KronCoefT<T> convert_coef(const KronCoef& c) {
  KronCoefT<T> o;
  for (int i = 0; i < FE_MAXN1; ++i) {
    for (int j = 0; j < FE_MAXN1; ++j) {
      o.AyM[i][j] = (T)c.AyM[i][j];
      o.AyK[i][j] = (T)c.AyK[i][j];
      o.AxM[i][j] = (T)c.AxM[i][j];
      o.AxK[i][j] = (T)c.AxK[i][j];
      o.AzK[i][j] = (T)c.AzK[i][j];
      o.AzM[i][j] = (T)c.AzM[i][j];
    }
    o.sig[i] = (T)c.sig[i];
    o.wz[i] = (T)c.wz[i];
  }
  o.zin = (T)c.zin;
  o.zout = (T)c.zout;
  o.mass_scale = c.mass_scale;
  return o;
}

// A chunk is CH consecutive vector entries of one node: 16 bytes (float4 / double2) or,
// for single-vector operators, one double.
template <typename T, int CH>
struct Chunk {
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
template <>
__device__ __forceinline__ double Chunk<double, 2>::fma_t(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ double Chunk<double, 1>::fma_t(double a, double b, double c) {
  return __fma_rn(a, b, c);
}

template <typename T, int CH>
__device__ __forceinline__ Chunk<T, CH> lds(const Chunk<T, CH>* p) {
  return *p;
}

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int nbytes_valid,
                                         int chunk_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (chunk_bytes == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(nbytes_valid));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
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

template <typename T, int P, int CH, int IPT>
__global__ void __launch_bounds__(512)
kron_kernel(const KronCoefT<T> cf, const KronGeom g, const KronIO<T> io, const int nch) {
  using C = Chunk<T, CH>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int BXn = g.bx * P, BYn = g.by * P;
  const int BXH = BXn + P + 1, BYH = BYn + P + 1;
  C* stage0 = reinterpret_cast<C*>(smem_raw);
  const int stage_sz = BYH * BXH * nch;
  C* A = stage0 + 2 * stage_sz;
  C* B = A + BYn * BXH * nch;
  C* W1 = B + BYn * BXH * nch;
  C* W2 = W1 + BYn * BXn * nch;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bxi = blockIdx.x % g.nbx, byi = blockIdx.x / g.nbx;
  const int x0 = bxi * BXn, y0 = byi * BYn;
  const int64_t vt0 = (int64_t)blockIdx.y * nch * CH;
  const int c0 = blockIdx.z * g.zseg;
  const int c1 = min(c0 + g.zseg, g.nz);
  const int cb = c0 > 0 ? c0 - 1 : 0;
  const int gbeg = cb * P, gend = c1 * P;
  const int nitemsZ = BXn * BYn * nch;

  // ---- the thread's output items --------------------------------------------------------
  int it_x[IPT], it_y[IPT], it_ch[IPT];
  bool it_own[IPT];
  T it_sxy[IPT];
  C acc[IPT][P + 1];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    int item = tid + i * nthr;
    bool valid = item < nitemsZ;
    int itc = valid ? item : 0;
    it_ch[i] = itc % nch;
    int node = itc / nch;
    it_x[i] = node % BXn;
    it_y[i] = node / BXn;
    int64_t v0 = vt0 + (int64_t)it_ch[i] * CH;
    it_own[i] = valid && (x0 + it_x[i] < g.NX) && (y0 + it_y[i] < g.NY) && (v0 < io.nvec);
    it_sxy[i] = cf.mass_scale ? cf.sig[it_x[i] % P] * cf.sig[it_y[i] % P] : T(1);
#pragma unroll
    for (int j = 0; j <= P; ++j) acc[i][j].zero();
  }

  const int chunk_bytes = (int)(CH * sizeof(T));
  auto stage_plane = [&](int gz, C* dst) {
    int zs = gz - g.gz_lo;
    if (zs < 0 || zs >= g.NZs) return;
    const int total = BYH * BXH * nch;
    for (int e = tid; e < total; e += nthr) {
      int ch = e % nch;
      int node = e / nch;
      int xh = node % BXH, yh = node / BXH;
      int gx = pmod(x0 - P + xh, g.NX);
      int gy = pmod(y0 - P + yh, g.NY);
      int64_t nid = gx + (int64_t)g.NX * (gy + (int64_t)g.NY * zs);
      int64_t v0 = vt0 + (int64_t)ch * CH;
      int64_t rem = io.nvec - v0;
      int valid = rem <= 0 ? 0 : (rem >= CH ? chunk_bytes : (int)(rem * sizeof(T)));
      const T* src = valid ? io.X + nid * io.ldx + v0 : io.X;
      cp_async(dst + e, src, valid, chunk_bytes);
    }
  };

  auto mz_of = [&](int gz) -> T {
    int l = gz % P;
    if (l != 0) return cf.wz[l];
    return (gz == 0 || gz == g.nz * P) ? cf.wz[0] : T(2) * cf.wz[0];
  };

  // write the final value of output plane gzo held in acc[i][j]
  auto write_plane = [&](int gzo, int j) {
    int zs = gzo - g.gz_lo;
    if (zs < 0 || zs >= g.NZs) return;
    T ps = cf.mass_scale ? cf.zout / sqrt(mz_of(gzo)) : cf.zout;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (!it_own[i]) continue;
      int64_t nid = (x0 + it_x[i]) + (int64_t)g.NX * ((y0 + it_y[i]) + (int64_t)g.NY * zs);
      int64_t v0 = vt0 + (int64_t)it_ch[i] * CH;
      T sc = io.alpha * ps * it_sxy[i];
      C out;
#pragma unroll
      for (int e = 0; e < CH; ++e) out.v[e] = sc * acc[i][j].v[e];
      if (io.Z != nullptr && io.beta != T(0)) {
        const T* zp = io.Z + nid * io.ldz + v0;
        if (v0 + CH <= io.nvec) {
          C zc = *reinterpret_cast<const C*>(zp);
#pragma unroll
          for (int e = 0; e < CH; ++e) out.v[e] = C::fma_t(io.beta, zc.v[e], out.v[e]);
        } else {
          for (int e = 0; e < CH; ++e)
            if (v0 + e < io.nvec) out.v[e] = C::fma_t(io.beta, zp[e], out.v[e]);
        }
      }
      T* yp = io.Y + nid * io.ldy + v0;
      if (v0 + CH <= io.nvec) {
        *reinterpret_cast<C*>(yp) = out;
      } else {
        for (int e = 0; e < CH; ++e)
          if (v0 + e < io.nvec) yp[e] = out.v[e];
      }
    }
  };

  // z contraction of the current plane's in-plane results into the layer accumulators
  auto phase_z = [&](int k, T s_in, const C* w1, const C* w2) {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      C a = w1[i], b = w2[i];
#pragma unroll
      for (int e = 0; e < CH; ++e) { a.v[e] *= s_in; b.v[e] *= s_in; }
#pragma unroll
      for (int j = 0; j <= P; ++j) {
        // k is uniform across the block; the table lookups are constant-bank reads
        T ck, cm;
        switch (k) {
#define FE_ZCASE(kk) \
  case kk:           \
    if (kk <= P) { ck = cf.AzK[j][kk]; cm = cf.AzM[j][kk]; } else { ck = cm = T(0); } break;
          FE_ZCASE(0) FE_ZCASE(1) FE_ZCASE(2) FE_ZCASE(3) FE_ZCASE(4) FE_ZCASE(5) FE_ZCASE(6)
#undef FE_ZCASE
          default: ck = cm = T(0);
        }
        acc[i][j].fma(ck, a);
        acc[i][j].fma(cm, b);
      }
    }
  };

  // ---- sweep -----------------------------------------------------------------------------
  stage_plane(gbeg, stage0);
  cp_commit();
  int c = cb;
  for (int gz = gbeg; gz <= gend; ++gz) {
    const int k = gz - c * P;
    C* st = stage0 + ((gz - gbeg) & 1) * stage_sz;
    if (gz < gend) {
      stage_plane(gz + 1, stage0 + ((gz + 1 - gbeg) & 1) * stage_sz);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();

    const int zs = gz - g.gz_lo;
    const bool stored = zs >= 0 && zs < g.NZs;
    C w1[IPT], w2[IPT];
    if (stored) {
      const T pscale = cf.mass_scale ? cf.zout / sqrt(mz_of(gz)) : cf.zout;
      // potential term folded into the accumulator of this plane (k = 0..P of layer c)
      if (io.V != nullptr) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          if (!it_own[i]) continue;
          int64_t nid = (x0 + it_x[i]) + (int64_t)g.NX * ((y0 + it_y[i]) + (int64_t)g.NY * zs);
          T vv = (io.V[nid] - io.shift) / (pscale * it_sxy[i]);
          const C xs = st[((it_y[i] + P) * BXH + (it_x[i] + P)) * nch + it_ch[i]];
          switch (k) {
#define FE_PCASE(kk) \
  case kk:           \
    if (kk <= P) acc[i][kk].fma(vv, xs); break;
            FE_PCASE(0) FE_PCASE(1) FE_PCASE(2) FE_PCASE(3) FE_PCASE(4) FE_PCASE(5) FE_PCASE(6)
#undef FE_PCASE
            default: break;
          }
        }
      }
      // phase Y: a = AyM U, b = AyK U along y at every halo x, cell by cell
      {
        const int cnt = BXH * nch * g.by;
        for (int e = tid; e < cnt; e += nthr) {
          int ch = e % nch;
          int r = e / nch;
          int xh = r % BXH;
          int cyl = r / BXH;
          int yb = cyl * P;
          C own[P + 1], prv[P];
#pragma unroll
          for (int kk = 0; kk <= P; ++kk) own[kk] = st[((yb + P + kk) * BXH + xh) * nch + ch];
#pragma unroll
          for (int kk = 0; kk < P; ++kk) prv[kk] = st[((yb + kk) * BXH + xh) * nch + ch];
#pragma unroll
          for (int j = 0; j < P; ++j) {
            C a, b;
            a.zero();
            b.zero();
#pragma unroll
            for (int kk = 0; kk <= P; ++kk) {
              a.fma(cf.AyM[j][kk], own[kk]);
              b.fma(cf.AyK[j][kk], own[kk]);
            }
            if (j == 0) {
#pragma unroll
              for (int kk = 0; kk < P; ++kk) {
                a.fma(cf.AyM[P][kk], prv[kk]);
                b.fma(cf.AyK[P][kk], prv[kk]);
              }
              a.fma(cf.AyM[P][P], own[0]);
              b.fma(cf.AyK[P][P], own[0]);
            }
            A[((yb + j) * BXH + xh) * nch + ch] = a;
            B[((yb + j) * BXH + xh) * nch + ch] = b;
          }
        }
      }
      __syncthreads();
      // phase X: W1 = AxM a, W2 = AxK a + AxM b along x at every owned y
      {
        const int cnt = BYn * nch * g.bx;
        for (int e = tid; e < cnt; e += nthr) {
          int ch = e % nch;
          int r = e / nch;
          int y = r % BYn;
          int cxl = r / BYn;
          int xb = cxl * P;
          const C* arow = A + (size_t)y * BXH * nch;
          const C* brow = B + (size_t)y * BXH * nch;
          C ao[P + 1], bo[P + 1];
#pragma unroll
          for (int kk = 0; kk <= P; ++kk) {
            ao[kk] = arow[(xb + P + kk) * nch + ch];
            bo[kk] = brow[(xb + P + kk) * nch + ch];
          }
#pragma unroll
          for (int j = 0; j < P; ++j) {
            C u, v;
            u.zero();
            v.zero();
#pragma unroll
            for (int kk = 0; kk <= P; ++kk) {
              u.fma(cf.AxM[j][kk], ao[kk]);
              v.fma(cf.AxK[j][kk], ao[kk]);
              v.fma(cf.AxM[j][kk], bo[kk]);
            }
            if (j == 0) {
#pragma unroll
              for (int kk = 0; kk < P; ++kk) {
                C ap = arow[(xb + kk) * nch + ch];
                C bp = brow[(xb + kk) * nch + ch];
                u.fma(cf.AxM[P][kk], ap);
                v.fma(cf.AxK[P][kk], ap);
                v.fma(cf.AxM[P][kk], bp);
              }
              u.fma(cf.AxM[P][P], ao[0]);
              v.fma(cf.AxK[P][P], ao[0]);
              v.fma(cf.AxM[P][P], bo[0]);
            }
            W1[(y * BXn + xb + j) * nch + ch] = u;
            W2[(y * BXn + xb + j) * nch + ch] = v;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        int item = (it_y[i] * BXn + it_x[i]) * nch + it_ch[i];
        w1[i] = W1[item];
        w2[i] = W2[item];
      }
      const T s_in = cf.mass_scale ? cf.zin / sqrt(mz_of(gz)) : cf.zin;
      phase_z(k, s_in, w1, w2);
      if (k == P) {
        // the layer is complete: its first P planes are final; the top plane's sum
        // becomes the bottom accumulator of the next layer
        if (c >= c0) {
#pragma unroll
          for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
        }
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          acc[i][0] = acc[i][P];
#pragma unroll
          for (int j = 1; j <= P; ++j) acc[i][j].zero();
        }
        ++c;
        if (c < c1) phase_z(0, s_in, w1, w2);
      }
    } else {
      // an unstored (homogeneous Dirichlet) plane contributes nothing
      if (k == P) {
        if (c >= c0) {
#pragma unroll
          for (int j = 0; j < P; ++j) write_plane(c * P + j, j);
        }
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          acc[i][0] = acc[i][P];
#pragma unroll
          for (int j = 1; j <= P; ++j) acc[i][j].zero();
        }
        ++c;
      }
    }
  }
  // the last processed plane (gend = c1 P) is final only if it is the top face
  if (c1 == g.nz) write_plane(gend, 0);
}

template <typename T, int P, int CH, int IPT>
fe_status kron_launch_t(const KronCoef& cf, const KronGeom& g, const KronIO<T>& io, int nch,
                        cudaStream_t st) {
  const int BXn = g.bx * P, BYn = g.by * P;
  const int BXH = BXn + P + 1, BYH = BYn + P + 1;
  const int nitemsZ = BXn * BYn * nch;
  int nthr = ((nitemsZ + IPT - 1) / IPT + 31) / 32 * 32;
  if (nthr > 512) return fe_fail(FE_EINVAL, "tile too large for one CTA");
  size_t smem = sizeof(Chunk<T, CH>) * (size_t)nch *
                (2 * (size_t)BYH * BXH + 2 * (size_t)BYn * BXH + 2 * (size_t)BYn * BXn);
  if (smem > 227 * 1024) return fe_fail(FE_EINVAL, "tile needs %zu bytes of shared memory", smem);
  auto kern = kron_kernel<T, P, CH, IPT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fe_fail(FE_ECUDA, "smem attribute: %s", cudaGetErrorString(e));
  }
  int64_t vtile = (int64_t)nch * CH;
  dim3 grid(g.nbx * g.nby, (unsigned)((io.nvec + vtile - 1) / vtile),
            (unsigned)((g.nz + g.zseg - 1) / g.zseg));
  if (grid.y > 65535 || grid.z > 65535) return fe_fail(FE_EINVAL, "grid too large");
  KronCoefT<T> cft = convert_coef<T>(cf);
  kern<<<grid, nthr, smem, st>>>(cft, g, io, nch); fe_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_fail(FE_ECUDA, "kron kernel launch: %s", cudaGetErrorString(e));
  return FE_OK;
}

}  // namespace fe

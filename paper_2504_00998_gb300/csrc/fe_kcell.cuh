// Cell-local float stiffness product of the Poisson iterations (Section 2.3), shared by the
// two-pass operator (fe_kcell.cu) and the persistent CG kernel (fe_cg_fused.cu).
//
// K is the assembly of the cell matrices K_e = az K1 (x) M1 (x) M1 + M1 (x) (ax K1 (x) M1 +
// M1 (x) ay K1) (z (x) x (x) y order, exactly integrated 1D matrices).  A strip of CX cells
// along x is staged in shared memory and every cell's y_e = K_e x_e is formed by three line
// contractions (y, then x, then z), each a dense (p+1) x (p+1) product on one line of the
// cell per thread.  The unassembled cell results go to a discontinuous node grid (every cell
// keeps its own copy of a shared node): index ((cz n1 + lz) ny n1 + cy n1 + ly) nx n1 +
// cx n1 + lx, n1 = p + 1.  A node's value is then the sum of its one to eight copies, lower
// cells first, so the result does not depend on scheduling.
#pragma once

#include <cstdint>

#include "fe_internal.h"

namespace fe_kc {

// cells per strip: about 256 to 400 lines of p + 1 nodes per phase
template <int P>
struct CellStrip {
  static constexpr int N1 = P + 1;
  static constexpr int CX = P == 1 ? 32 : P <= 3 ? 16 : P <= 5 ? 8 : 4;   // static smem < 48 KB
  static constexpr int LINES = CX * N1 * N1;
  static constexpr int NTHR = (LINES + 31) / 32 * 32;
  static constexpr int UW = CX * P + 1;          // staged nodes along x
  static constexpr int U_FLOATS = N1 * N1 * UW;  // [lz][ly][xl]
  static constexpr int A_FLOATS = N1 * N1 * CX * N1;
  static constexpr int SPT = (U_FLOATS + NTHR - 1) / NTHR;   // staged values per thread
};

struct CellCoef {
  float M1[FE_MAXN1][FE_MAXN1];   // AyM = AxM = AzM (the 1D mass)
  float Ky[FE_MAXN1][FE_MAXN1];   // ay K1
  float Kx[FE_MAXN1][FE_MAXN1];   // ax K1
  float Kz[FE_MAXN1][FE_MAXN1];   // az K1
};

// the float coefficients of the mesh's Poisson operator
inline CellCoef cell_coef(const fe_mesh* m) {
  CellCoef cf;
  const KronCoef& k = m->coefK;
  for (int j = 0; j < FE_MAXN1; ++j)
    for (int i = 0; i < FE_MAXN1; ++i) {
      cf.M1[j][i] = (float)k.AzM[j][i];
      cf.Ky[j][i] = (float)k.AyK[j][i];
      cf.Kx[j][i] = (float)k.AxK[j][i];
      cf.Kz[j][i] = (float)k.AzK[j][i];
    }
  return cf;
}

// global node of staged element e (< U_FLOATS) of the strip (cx0, cy, cz): x periodic (a
// partial last strip wraps), y periodic, z inside the slab
template <int P>
__device__ __forceinline__ int64_t strip_node(int e, int cx0, int cy, int cz, int NX, int NY) {
  using S = CellStrip<P>;
  constexpr int N1 = S::N1, UW = S::UW;
  const int xl = e % UW, ly = (e / UW) % N1, lz = e / (UW * N1);
  int gx = cx0 * P + xl;
  gx -= (gx >= NX) ? NX * (gx / NX) : 0;
  int gy = cy * P + ly;
  gy -= (gy >= NY) ? NY : 0;
  const int64_t gz = (int64_t)cz * P + lz;
  return (gz * NY + gy) * NX + gx;
}

// y_e of the strip of cells (cx0 .. cx0 + CX - 1, cy, cz) into the discontinuous grid, from
// the strip's nodes already written to U (element e = strip_node's).  U, A, B are shared
// arrays (U_FLOATS, A_FLOATS, A_FLOATS floats) of the NTHR threads that call it together
// (thread index tid < NTHR), and sync() is their barrier.  U is read only before the second
// of the three barriers, so once every thread has returned from a call (the third barrier
// passed) U may be refilled for the next strip without a further barrier.
template <int P, class Sync>
__device__ __forceinline__ void strip_products(const CellCoef& cf, float* __restrict__ ycell,
                                               int cx0, int cy, int cz, int nx, int ny,
                                               const float* U, float* A, float* B, int tid,
                                               Sync sync) {
  using S = CellStrip<P>;
  constexpr int N1 = S::N1, CX = S::CX, UW = S::UW;
  sync();
  // [lz][ly][c][lx]: the y contractions with M1 (A) and ay K1 (B), then in place the x
  // contractions W1 = M1 A (in A) and W2 = ax K1 A + M1 B (in B): an x line is read whole by
  // the one thread that overwrites it
  float* W1 = A;
  float* W2 = B;
  const bool active = tid < S::LINES;
  // y lines (lz, c, lx): A, B = (M1, ay K1) along y
  if (active) {
    const int lx = tid % N1, c = (tid / N1) % CX, lz = tid / (N1 * CX);
    float in[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) in[k] = U[(lz * N1 + k) * UW + c * P + lx];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        a = __fmaf_rn(cf.M1[j][k], in[k], a);
        b = __fmaf_rn(cf.Ky[j][k], in[k], b);
      }
      const int o = ((lz * N1 + j) * CX + c) * N1 + lx;
      A[o] = a;
      B[o] = b;
    }
  }
  sync();
  // x lines (c, ly, lz): W1 = M1 A, W2 = ax K1 A + M1 B along x
  if (active) {
    const int c = tid % CX, ly = (tid / CX) % N1, lz = tid / (CX * N1);
    const int base = ((lz * N1 + ly) * CX + c) * N1;
    float a[N1], b[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) { a[k] = A[base + k]; b[k] = B[base + k]; }
#pragma unroll
    for (int j = 0; j < N1; ++j) {
      float u = 0.f, v = 0.f;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        u = __fmaf_rn(cf.M1[j][k], a[k], u);
        v = __fmaf_rn(cf.Kx[j][k], a[k], v);
        v = __fmaf_rn(cf.M1[j][k], b[k], v);
      }
      W1[base + j] = u;
      W2[base + j] = v;
    }
  }
  sync();
  // z lines (lx, c, ly): y_e = az K1 W1 + M1 W2 along z, to the discontinuous grid
  if (active) {
    const int lx = tid % N1, c = (tid / N1) % CX, ly = tid / (N1 * CX);
    const int cx = cx0 + c;
    if (cx < nx) {
      float w1[N1], w2[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int o = ((k * N1 + ly) * CX + c) * N1 + lx;
        w1[k] = W1[o];
        w2[k] = W2[o];
      }
      const int64_t dnx = (int64_t)nx * N1, dny = (int64_t)ny * N1;
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          s = __fmaf_rn(cf.Kz[j][k], w1[k], s);
          s = __fmaf_rn(cf.M1[j][k], w2[k], s);
        }
        ycell[(((int64_t)cz * N1 + j) * dny + (int64_t)cy * N1 + ly) * dnx + (int64_t)cx * N1 + lx] = s;
      }
    }
  }
}

// stage the strip from load(gid) (the input at global node gid), then strip_products (the
// whole block of NTHR threads)
template <int P, class Load>
__device__ __forceinline__ void cell_strip(const CellCoef& cf, Load load, float* __restrict__ ycell,
                                           int cx0, int cy, int cz, int nx, int ny, int NX,
                                           int NY, float* U, float* A, float* B) {
  using S = CellStrip<P>;
  for (int e = threadIdx.x; e < S::U_FLOATS; e += S::NTHR)
    U[e] = load(strip_node<P>(e, cx0, cy, cz, NX, NY));
  strip_products<P>(cf, ycell, cx0, cy, cz, nx, ny, U, A, B, (int)threadIdx.x,
                    [] { __syncthreads(); });
}

// the one or two (cell, local index) copies of global index g along a periodic direction of
// nc cells, lower cell first (d[0], and d[1] when there are two); returns their number
template <int P>
__device__ __forceinline__ int cell_copies_periodic(int g, int nc, int* d) {
  constexpr int N1 = P + 1;
  const int c = g / P, l = g - c * P;
  const int cur = c * N1 + l;
  d[0] = l == 0 ? (c == 0 ? nc - 1 : c - 1) * N1 + P : cur;
  d[1] = cur;
  return l == 0 ? 2 : 1;
}

// the assembled value at node (gx, gy, gz): the sum of its copies, lower cells first (loads
// through L2: the grid may have been written by other blocks of the same kernel).  dx, dy
// and their counts come from cell_copies_periodic; the loops have constant trip counts so
// that the copy indices stay in registers.
template <int P>
__device__ __forceinline__ float cell_gather_node(const float* ycell, const int* dx, int nxc,
                                                  const int* dy, int nyc, int gz, int nx, int ny,
                                                  int nz) {
  constexpr int N1 = P + 1;
  const int c = gz / P, l = gz - c * P;
  const bool below = l == 0 && c > 0, own = c < nz;
  int dz[2];
  dz[0] = below ? (c - 1) * N1 + P : c * N1 + l;
  dz[1] = c * N1 + l;
  const int nzc = (below ? 1 : 0) + (own ? 1 : 0);
  const int64_t dnx = (int64_t)nx * N1, dny = (int64_t)ny * N1;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (a >= nzc) break;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (b >= nyc) break;
      const float* row = ycell + ((int64_t)dz[a] * dny + dy[b]) * dnx;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (e >= nxc) break;
        s += __ldcg(row + dx[e]);
      }
    }
  }
  return s;
}

}  // namespace fe_kc

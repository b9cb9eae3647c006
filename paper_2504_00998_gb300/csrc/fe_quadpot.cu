// Potential term integrated by Gauss quadrature: the consistent (cell-matrix) form of the
// potential in the discretised Kohn-Sham operator of Section 2.3,
//   V_IJ = int N_I V_eff N_J dx = sum_cells sum_q w_q |J| V_e(x_q) N_I(x_q) N_J(x_q),
// with V_eff given at the (p+1)^3 Gauss-Legendre points of every cell.  Each cell's matrix
// is V_e = B^T diag(W_e) B with B = B1 (x) B1 (x) B1 the interpolation from the cell's GLL
// nodes to its Gauss points, so it is applied without being stored: per cell and vector,
// three line contractions to the Gauss points, the pointwise weight W_e = w |J| V_e, and
// three transposed contractions back (6 (p+1)^4 FMAs instead of (p+1)^6 for a stored
// matrix, and no matrix traffic).  The scaled operator adds
//   Y += alpha M^-1/2 V M^-1/2 X
// to the output of the sum-factorised kinetic operator (which then runs with a zero
// collocated potential and only the Chebyshev shift on its diagonal).
//
// Assembly is deterministic: the cells are processed in colour passes such that no two cells
// of one pass share a node (parity of cx, cy, cz; a third x (y) class holds the last cell when
// nx (ny) is odd, since the periodic wrap joins it to cell 0), and a cell that meets itself
// across the periodic wrap (nx or ny = 1) folds its two copies of a node before writing.
#include <cmath>
#include <vector>

#include <type_traits>

#include "fe_blas.cuh"
#include "fe_gll_tables.h"
#include "fe_internal.h"

namespace {

template <typename T>
struct QuadLanes;
template <>
struct QuadLanes<float> {
  static constexpr int v = 32;   // vector lanes per CTA
  using V16 = float4;            // one 16-byte access
};
template <>
struct QuadLanes<double> {
  static constexpr int v = 16;
  using V16 = double2;
};

// thread layout of one cell: a thread per 16-byte lane group of a line (N1^2 lines per
// direction), rounded up to whole warps
template <typename T, int P>
struct QuadShape {
  static constexpr int N1 = P + 1, NN = N1 * N1 * N1;
  static constexpr int VC = QuadLanes<T>::v;
  static constexpr int VW = 16 / (int)sizeof(T);   // lanes per 16-byte access
  static constexpr int G = VC / VW;                // lane groups per node
  static constexpr int LINES = N1 * N1 * G;
  static constexpr int NT = (LINES + 31) / 32 * 32;
};

template <typename T>
struct QuadB {
  T B[FE_MAXN1][FE_MAXN1];   // B[q][i] = l_i(gauss point q), reference interval
};

struct QuadPass {
  int nx, ny, NX, NY, gz_lo, gz_hi;
  int ox, oy, oz;         // colour class per direction (2: the last cell of an odd row)
  int cntx, cnty, cntz;   // cells of the class per direction
  int foldx, foldy;       // a single cell along x (y): local nodes 0 and p coincide
};

__device__ __forceinline__ int class_cell(int t, int cls, int n) {
  return cls == 2 ? n - 1 : 2 * t + cls;
}

template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <>
__device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ float4 vfma(float a, const float4& x, const float4& y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 vfma(double a, const double2& x, const double2& y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float4 vscale(float a, const float4& x) {
  return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}
__device__ __forceinline__ double2 vscale(double a, const double2& x) {
  return make_double2(a * x.x, a * x.y);
}
// keep the first k lanes (k < lanes of the access), zero the rest
__device__ __forceinline__ float4 vkeep(float4 x, int k) {
  if (k < 4) x.w = 0.f;
  if (k < 3) x.z = 0.f;
  if (k < 2) x.y = 0.f;
  return x;
}
__device__ __forceinline__ double2 vkeep(double2 x, int k) {
  if (k < 2) x.y = 0.0;
  return x;
}
__device__ __forceinline__ void vstore_first(float* p, const float4& x, int k) {
  p[0] = x.x;
  if (k > 1) p[1] = x.y;
  if (k > 2) p[2] = x.z;
}
__device__ __forceinline__ void vstore_first(double* p, const double2& x, int) { p[0] = x.x; }

// one line contraction along direction D of the cell block in shared memory ([node][lane],
// 16-byte groups): forward dst(q) = sum_e B[q][e] src(e) (times the quadrature weight of
// point q when WEIGH), transposed dst(e) = sum_q B[q][e] src(q).  Line (a, b, group) of the
// calling thread: a, b the two other local indices.
template <typename T, int P, int D, bool TR, bool WEIGH>
__device__ __forceinline__ void contract(const QuadB<T>& cb, const T* __restrict__ src,
                                         T* __restrict__ dst, const T* __restrict__ Ws, int a,
                                         int b, int grp) {
  using S = QuadShape<T, P>;
  using V = typename QuadLanes<T>::V16;
  constexpr int N1 = S::N1, G = S::G;
  constexpr int STRIDE = D == 0 ? 1 : D == 1 ? N1 : N1 * N1;
  const int base = D == 0 ? (b * N1 + a) * N1 : D == 1 ? b * N1 * N1 + a : b * N1 + a;
  const V* s = reinterpret_cast<const V*>(src);
  V* d = reinterpret_cast<V*>(dst);
  V in[N1];
#pragma unroll
  for (int e = 0; e < N1; ++e) in[e] = s[(base + e * STRIDE) * G + grp];
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    V acc = vzero<V>();
#pragma unroll
    for (int e = 0; e < N1; ++e) {
      // float: the interpolation table as compile-time constants (immediate operands)
      T c;
      if constexpr (std::is_same<T, float>::value)
        c = TR ? fe::gauss_b<P>(e, q) : fe::gauss_b<P>(q, e);
      else
        c = TR ? cb.B[e][q] : cb.B[q][e];
      acc = vfma(c, in[e], acc);
    }
    if constexpr (WEIGH) acc = vscale(Ws[base + q * STRIDE], acc);
    d[(base + q * STRIDE) * G + grp] = acc;
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(QuadShape<T, P>::NT)
k_quad_apply(const QuadB<T> cb, const QuadPass g, const T* __restrict__ X, T* __restrict__ Y,
             int64_t ld, int64_t nvec, const T* __restrict__ W, const T* __restrict__ rsq,
             T alpha) {
  using S = QuadShape<T, P>;
  using V = typename QuadLanes<T>::V16;
  constexpr int N1 = S::N1, NN = S::NN, VC = S::VC, VW = S::VW, G = S::G, NT = S::NT;
  constexpr int SLOTS = NN * G;                      // 16-byte slots of the cell block
  constexpr int IT = (SLOTS + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + NN * VC;
  constexpr int NNE = (NN + 1) & ~1;                 // even: keeps node[] 8-byte aligned
  T* Ws = bufB + NN * VC;                            // w |J| V at the Gauss points
  T* rs = Ws + NNE;                                  // M^-1/2 at the cell's nodes
  int64_t* node = reinterpret_cast<int64_t*>(rs + NNE);

  int t = blockIdx.x;
  const int tx = t % g.cntx;
  t /= g.cntx;
  const int ty = t % g.cnty, tz = t / g.cnty;
  const int cx = class_cell(tx, g.ox, g.nx), cy = class_cell(ty, g.oy, g.ny);
  const int cz = 2 * tz + g.oz;
  const int64_t cell = ((int64_t)cz * g.ny + cy) * g.nx + cx;
  const int64_t v0 = (int64_t)blockIdx.y * VC;
  const int64_t plane = (int64_t)g.NX * g.NY;
  const int tid = threadIdx.x;

  for (int e = tid; e < NN; e += NT) {
    const int i = e % N1, j = (e / N1) % N1, k = e / (N1 * N1);
    int gx = cx * P + i, gy = cy * P + j;
    gx -= gx >= g.NX ? g.NX : 0;
    gy -= gy >= g.NY ? g.NY : 0;
    const int gz = cz * P + k;
    const bool in = gz >= g.gz_lo && gz <= g.gz_hi;
    const int64_t n = in ? (gz - g.gz_lo) * plane + (int64_t)gy * g.NX + gx : -1;
    node[e] = n;
    rs[e] = in ? rsq[n] : T(0);
    Ws[e] = W[cell * NN + e];
  }
  __syncthreads();
  const bool act = tid < S::LINES;
  const int grp = tid % G, ab = tid / G;
  const int la = ab % N1, lb = ab / N1;     // (j, k) of the thread's x line
  const int xbase = (lb * N1 + la) * N1;
  const int64_t vv = v0 + (int64_t)grp * VW;
  const int64_t left = nvec - vv;           // lanes of the group that are vectors
  // x lines straight from global memory: u = M^-1/2 X on the line's nodes (every load of
  // the thread in flight before the first use; zero on Dirichlet faces and past the last
  // vector; a row holds ld >= the group's end, so the whole group is in bounds), then the
  // forward x contraction
  if (act) {
    V in[N1];
#pragma unroll
    for (int e = 0; e < N1; ++e) {
      const int64_t n = node[xbase + e];
      in[e] = vzero<V>();
      if (n >= 0 && left > 0) in[e] = *reinterpret_cast<const V*>(X + n * ld + vv);
    }
    V* d = reinterpret_cast<V*>(bufB);
#pragma unroll
    for (int e = 0; e < N1; ++e) {
      in[e] = vscale(rs[xbase + e], in[e]);
      if (left < VW) in[e] = vkeep(in[e], left > 0 ? (int)left : 0);
    }
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      V acc = vzero<V>();
#pragma unroll
      for (int e = 0; e < N1; ++e) {
        T c;
        if constexpr (std::is_same<T, float>::value) c = fe::gauss_b<P>(q, e);
        else c = cb.B[q][e];
        acc = vfma(c, in[e], acc);
      }
      d[(xbase + q) * G + grp] = acc;
    }
  }
  __syncthreads();
  if (act) contract<T, P, 1, false, false>(cb, bufB, bufA, Ws, la, lb, grp);
  __syncthreads();
  if (act) contract<T, P, 2, false, true>(cb, bufA, bufB, Ws, la, lb, grp);
  __syncthreads();
  if (act) contract<T, P, 2, true, false>(cb, bufB, bufA, Ws, la, lb, grp);
  __syncthreads();
  if (act) contract<T, P, 1, true, false>(cb, bufA, bufB, Ws, la, lb, grp);
  __syncthreads();
  if (!g.foldy) {
    // transposed x contraction in registers and Y += alpha M^-1/2 (.) along the line; a
    // single cell along x (foldx) adds its two copies of node 0 before writing it once
    if (act) {
      const V* sv = reinterpret_cast<const V*>(bufB);
      V in[N1], out[N1];
#pragma unroll
      for (int q = 0; q < N1; ++q) in[q] = sv[(xbase + q) * G + grp];
#pragma unroll
      for (int e = 0; e < N1; ++e) {
        V acc = vzero<V>();
#pragma unroll
        for (int q = 0; q < N1; ++q) {
          T c;
          if constexpr (std::is_same<T, float>::value) c = fe::gauss_b<P>(q, e);
          else c = cb.B[q][e];
          acc = vfma(c, in[q], acc);
        }
        out[e] = acc;
      }
      if (g.foldx) out[0] = vfma(T(1), out[P], out[0]);
      V yv[N1];
#pragma unroll
      for (int e = 0; e < N1; ++e) {
        const int64_t n = node[xbase + e];
        yv[e] = vzero<V>();
        if (n >= 0 && left > 0 && !(g.foldx && e == P))
          yv[e] = *reinterpret_cast<const V*>(Y + n * ld + vv);
      }
#pragma unroll
      for (int e = 0; e < N1; ++e) {
        const int64_t n = node[xbase + e];
        if (n < 0 || left <= 0 || (g.foldx && e == P)) continue;
        const V o = vfma(alpha * rs[xbase + e], out[e], yv[e]);
        T* yp = Y + n * ld + vv;
        if (left >= VW)
          *reinterpret_cast<V*>(yp) = o;
        else
          vstore_first(yp, o, (int)left);
      }
    }
    return;
  }
  // a single cell along y: the two copies of each j = 0 node are in different x lines, so
  // the block goes back to the nodes in shared memory and is folded there
  if (act) contract<T, P, 0, true, false>(cb, bufB, bufA, Ws, la, lb, grp);
  __syncthreads();
  V* A = reinterpret_cast<V*>(bufA);
  if (g.foldx) {
    for (int idx = tid; idx < N1 * N1 * G; idx += NT) {
      const int gg = idx % G, r = idx / G;   // r = (k, j)
      V x = A[(r * N1) * G + gg];
      const V y = A[(r * N1 + P) * G + gg];
      A[(r * N1) * G + gg] = vfma(T(1), y, x);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < N1 * N1 * G; idx += NT) {
    const int gg = idx % G, r = idx / G;
    const int i = r % N1, k = r / N1;
    V x = A[(k * N1 * N1 + i) * G + gg];
    const V y = A[(k * N1 * N1 + P * N1 + i) * G + gg];
    A[(k * N1 * N1 + i) * G + gg] = vfma(T(1), y, x);
  }
  __syncthreads();
  // Y += alpha M^-1/2 (V u): all loads of Y first, then the updates
  {
    V yv[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int sl = tid + it * NT;
      yv[it] = vzero<V>();
      if (sl < SLOTS) {
        const int e = sl / G, ww = (sl % G) * VW;
        const int64_t n = node[e];
        if (n >= 0 && v0 + ww < nvec) yv[it] = *reinterpret_cast<const V*>(Y + n * ld + v0 + ww);
      }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int sl = tid + it * NT;
      if (sl >= SLOTS) continue;
      const int e = sl / G, ww = (sl % G) * VW;
      const int i = e % N1, j = (e / N1) % N1;
      if ((g.foldx && i == P) || j == P) continue;
      const int64_t n = node[e];
      if (n < 0 || v0 + ww >= nvec) continue;
      const V o = vfma(alpha * rs[e], A[sl], yv[it]);
      T* yp = Y + n * ld + v0 + ww;
      const int64_t rem = nvec - (v0 + ww);
      if (rem >= VW)
        *reinterpret_cast<V*>(yp) = o;
      else
        vstore_first(yp, o, (int)rem);
    }
  }
}

template <typename T, int P>
size_t quad_smem() {
  using S = QuadShape<T, P>;
  return sizeof(T) * (2 * (size_t)S::NN * S::VC + 2 * (size_t)((S::NN + 1) & ~1)) +
         sizeof(int64_t) * S::NN;
}

template <typename T, int P>
fe_status quad_apply_p(fe_mesh* m, const QuadB<T>& cb, const T* X, T* Y, int64_t ld,
                       int64_t nvec, const T* W, const T* rsq, T alpha) {
  using S = QuadShape<T, P>;
  constexpr int VC = S::VC;
  const size_t smem = quad_smem<T, P>();
  cudaError_t e = cudaFuncSetAttribute(k_quad_apply<T, P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_quad_apply<T, P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fe_fail(FE_ECUDA, "quadrature potential: %s", cudaGetErrorString(e));
  }
  if (((uintptr_t)X) % 16 || ((uintptr_t)Y) % 16 || (ld * (int64_t)sizeof(T)) % 16)
    return fe_fail(FE_EINVAL, "quadrature potential: blocks need 16-byte aligned rows");
  const int64_t nchunk = (nvec + VC - 1) / VC;
  if (nchunk > 65535) return fe_fail(FE_EINVAL, "quadrature potential: too many vectors");
  // colour classes per direction: {class, cells}
  auto classes = [](int n, bool periodic, int* cls, int* cnt) {
    if (!periodic) {
      cls[0] = 0; cnt[0] = (n + 1) / 2;
      cls[1] = 1; cnt[1] = n / 2;
      return 2;
    }
    if (n == 1) { cls[0] = 0; cnt[0] = 1; return 1; }
    if (n % 2 == 0) {
      cls[0] = 0; cnt[0] = n / 2;
      cls[1] = 1; cnt[1] = n / 2;
      return 2;
    }
    cls[0] = 0; cnt[0] = (n - 1) / 2;
    cls[1] = 1; cnt[1] = (n - 1) / 2;
    cls[2] = 2; cnt[2] = 1;
    return 3;
  };
  int clx[3], cnx[3], cly[3], cny[3], clz[3], cnz[3];
  const int ncx = classes(m->nx, true, clx, cnx);
  const int ncy = classes(m->ny, true, cly, cny);
  const int ncz = classes(m->nz, false, clz, cnz);
  QuadPass g;
  g.nx = m->nx; g.ny = m->ny; g.NX = m->NX; g.NY = m->NY;
  g.gz_lo = m->gz_lo; g.gz_hi = m->gz_hi;
  g.foldx = m->nx == 1; g.foldy = m->ny == 1;
  for (int a = 0; a < ncz; ++a)
    for (int b = 0; b < ncy; ++b)
      for (int c = 0; c < ncx; ++c) {
        const int64_t cells = (int64_t)cnx[c] * cny[b] * cnz[a];
        if (cells == 0) continue;
        if (cells > 0x7fffffffLL) return fe_fail(FE_EINVAL, "quadrature potential: mesh too large");
        g.ox = clx[c]; g.oy = cly[b]; g.oz = clz[a];
        g.cntx = cnx[c]; g.cnty = cny[b]; g.cntz = cnz[a];
        k_quad_apply<T, P><<<dim3((unsigned)cells, (unsigned)nchunk), S::NT, smem, m->stream>>>(
            cb, g, X, Y, ld, nvec, W, rsq, alpha);
        fe_count_launch();
      }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

template <typename T>
fe_status quad_apply_t(fe_mesh* m, const T* X, T* Y, int64_t ld, int64_t nvec, const T* W,
                       const T* rsq, T alpha) {
  QuadB<T> cb;
  for (int q = 0; q < FE_MAXN1; ++q)
    for (int i = 0; i < FE_MAXN1; ++i) cb.B[q][i] = (T)m->Bq[q][i];
  switch (m->p) {
    case 1: return quad_apply_p<T, 1>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    case 2: return quad_apply_p<T, 2>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    case 3: return quad_apply_p<T, 3>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    case 4: return quad_apply_p<T, 4>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    case 5: return quad_apply_p<T, 5>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    case 6: return quad_apply_p<T, 6>(m, cb, X, Y, ld, nvec, W, rsq, alpha);
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", m->p);
  }
}

// n-point Gauss-Legendre rule on [-1, 1]: Newton's method on P_n from the Chebyshev-like
// first guesses cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' from the three-term recurrence;
// weights 2 / ((1 - x^2) P_n'(x)^2).  Ascending order.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static_assert(FE_MAXN1 == 7, "the weight kernel takes seven Gauss weights");

// W[e][q] = w_a w_b w_c |J| Vq[e][q], q = a + nq (b + nq c); float copy alongside
__global__ void k_quad_weights(const double* __restrict__ Vq, int64_t n, int nq, double detJ,
                               double w0, double w1, double w2, double w3, double w4, double w5,
                               double w6, double* __restrict__ W, float* __restrict__ Wf) {
  const double wq[7] = {w0, w1, w2, w3, w4, w5, w6};
  const int nn = nq * nq * nq;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % nn);
    const int a = q % nq, b = (q / nq) % nq, c = q / (nq * nq);
    const double v = wq[a] * wq[b] * wq[c] * detJ * Vq[i];
    W[i] = v;
    Wf[i] = (float)v;
  }
}

// M^-1/2 at psi nodes from the lumped mass at phi nodes
__global__ void k_psi_rsq(const double* __restrict__ mass, int64_t off, int64_t n,
                          double* __restrict__ r, float* __restrict__ rf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = 1.0 / sqrt(mass[i + off]);
    r[i] = s;
    rf[i] = (float)s;
  }
}

__global__ void k_zero2(double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = 0.0;
    b[i] = 0.0f;
  }
}

struct InterpB {
  double B[FE_MAXN1][FE_MAXN1];
};

// f at every cell's Gauss points from its nodal values on phi nodes
__global__ void k_interp_quad(const InterpB cb, const double* __restrict__ f, int p, int nx,
                              int ny, int NX, int NY, int64_t ncells, double* __restrict__ out) {
  const int n1 = p + 1, nn = n1 * n1 * n1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells * nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = i / nn;
    const int q = (int)(i % nn);
    const int a = q % n1, b = (q / n1) % n1, c = q / (n1 * n1);
    const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny);
    const int cz = (int)(cell / ((int64_t)nx * ny));
    double s = 0.0;
    for (int k = 0; k < n1; ++k) {
      const int64_t gz = (int64_t)cz * p + k;
      double sy = 0.0;
      for (int j = 0; j < n1; ++j) {
        int gy = cy * p + j;
        gy -= gy >= NY ? NY : 0;
        const double* row = f + (gz * NY + gy) * NX;
        double sx = 0.0;
        for (int l = 0; l < n1; ++l) {
          int gx = cx * p + l;
          gx -= gx >= NX ? NX : 0;
          sx = fma(cb.B[a][l], row[gx], sx);
        }
        sy = fma(cb.B[b][j], sx, sy);
      }
      s = fma(cb.B[c][k], sy, s);
    }
    out[i] = s;
  }
}

}  // namespace

void fe_quad_setup_basis(fe_mesh* m) {
  const int n1 = m->p + 1;
  double x[FE_MAXN1], w[FE_MAXN1];
  gauss_legendre(n1, x, w);
  for (int q = 0; q < FE_MAXN1; ++q) {
    m->wq[q] = q < n1 ? w[q] : 0.0;
    for (int i = 0; i < FE_MAXN1; ++i) {
      double l = 0.0;
      if (q < n1 && i < n1) {
        l = 1.0;
        for (int j = 0; j < n1; ++j)
          if (j != i) l *= (x[q] - m->xi[j]) / (m->xi[i] - m->xi[j]);
      }
      m->Bq[q][i] = l;
    }
  }
}

void fe_quad_free(fe_mesh* m) {
  cudaFree(m->d_qW);
  cudaFree(m->d_qW_f);
  cudaFree(m->d_rsq);
  cudaFree(m->d_rsq_f);
  m->d_qW = nullptr;
  m->d_qW_f = nullptr;
  m->d_rsq = nullptr;
  m->d_rsq_f = nullptr;
  m->has_quad = false;
}

fe_status fe_quad_apply(fe_mesh* m, const void* X, void* Y, int64_t nvec, int64_t ld,
                        double alpha, bool dbl) {
  if (!m->has_quad) return FE_OK;
  if (dbl)
    return quad_apply_t<double>(m, (const double*)X, (double*)Y, ld, nvec, m->d_qW, m->d_rsq,
                                alpha);
  return quad_apply_t<float>(m, (const float*)X, (float*)Y, ld, nvec, m->d_qW_f, m->d_rsq_f,
                             (float)alpha);
}

extern "C" fe_status fe_set_potential_quad(fe_mesh* m, const double* vq) {
  if (!m || !vq) return fe_fail(FE_EINVAL, "fe_set_potential_quad: null argument");
  if (m->p > 6) return fe_fail(FE_EUNSUPPORTED, "fe_set_potential_quad: p = %d", m->p);
  FE_TRY(fe_activate(m));
  const int n1 = m->p + 1;
  const int64_t nq = m->n_cells * (int64_t)n1 * n1 * n1;
  if (!m->d_veff) {
    if (cudaMalloc(&m->d_veff, m->n_psi * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_veff_f, m->n_psi * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fe_fail(FE_ENOMEM, "potential allocation failed");
    }
  }
  if (!m->d_qW) {
    if (cudaMalloc(&m->d_qW, nq * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_qW_f, nq * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->d_rsq, m->n_psi * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_rsq_f, m->n_psi * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      fe_quad_free(m);
      return fe_fail(FE_ENOMEM, "quadrature potential allocation failed");
    }
  }
  cudaStream_t st = m->stream;
  // the collocated potential is zero: the kinetic kernel keeps only the Chebyshev shift
  k_zero2<<<fe::grid_for(m->n_psi), 256, 0, st>>>(m->d_veff, m->d_veff_f, m->n_psi);
  fe_count_launch();
  const double* w = m->wq;
  k_quad_weights<<<fe::grid_for(nq), 256, 0, st>>>(vq, nq, n1, m->J, w[0], w[1], w[2], w[3],
                                                   w[4], w[5], w[6], m->d_qW, m->d_qW_f);
  fe_count_launch();
  k_psi_rsq<<<fe::grid_for(m->n_psi), 256, 0, st>>>(
      m->d_mass, (int64_t)m->gz_lo * m->NX * m->NY, m->n_psi, m->d_rsq, m->d_rsq_f);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  m->has_potential = true;
  m->has_quad = true;
  return FE_OK;
}

extern "C" fe_status fe_interp_quad(fe_mesh* m, const double* f_phi, double* out) {
  if (!m || !f_phi || !out) return fe_fail(FE_EINVAL, "fe_interp_quad: null argument");
  FE_TRY(fe_activate(m));
  InterpB cb;
  for (int q = 0; q < FE_MAXN1; ++q)
    for (int i = 0; i < FE_MAXN1; ++i) cb.B[q][i] = m->Bq[q][i];
  const int n1 = m->p + 1;
  const int64_t total = m->n_cells * (int64_t)n1 * n1 * n1;
  k_interp_quad<<<fe::grid_for(total), 256, 0, m->stream>>>(cb, f_phi, m->p, m->nx, m->ny, m->NX,
                                                           m->NY, m->n_cells, out);
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// Single-vector stiffness product y = K x (float) for the Poisson iterations of Section 2.3,
// cell by cell.
//
// K is the assembly of the cell matrices K_e = az K1 (x) M1 (x) M1 + M1 (x) (ax K1 (x) M1 +
// M1 (x) ay K1) (z (x) x (x) y order, exactly integrated 1D matrices).  With one vector the
// plane sweep of the block operator leaves most of a CTA idle between its per-plane barriers,
// so this path has two short passes instead:
//   1. k_cell_apply: a CTA takes a strip of CX cells along x, stages the strip's nodes, and
//      forms y_e = K_e x_e of every cell by three line contractions (y, then x, then z), each
//      a dense (p+1) x (p+1) product on one line of the cell per thread.  The unassembled
//      cell results go to a discontinuous node grid (every cell keeps its own copy of a shared
//      node): index ((cz n1 + lz) ny n1 + cy n1 + ly) nx n1 + cx n1 + lx, n1 = p + 1.
//   2. k_cell_gather: every node sums its one to eight cell copies, lower cells first, so the
//      result does not depend on scheduling.
#include <cstdint>

#include "fe_internal.h"

namespace {

// cells per CTA strip: about 256 to 400 lines of p + 1 nodes per phase
template <int P>
struct CellStrip {
  static constexpr int N1 = P + 1;
  static constexpr int CX = P == 1 ? 32 : P <= 3 ? 16 : P <= 5 ? 8 : 4;   // static smem < 48 KB
  static constexpr int LINES = CX * N1 * N1;
  static constexpr int NTHR = (LINES + 31) / 32 * 32;
  static constexpr int UW = CX * P + 1;          // staged nodes along x
};

struct CellCoef {
  float M1[FE_MAXN1][FE_MAXN1];   // AyM = AxM = AzM (the 1D mass)
  float Ky[FE_MAXN1][FE_MAXN1];   // ay K1
  float Kx[FE_MAXN1][FE_MAXN1];   // ax K1
  float Kz[FE_MAXN1][FE_MAXN1];   // az K1
};

template <int P>
__global__ void __launch_bounds__(CellStrip<P>::NTHR)
k_cell_apply(const CellCoef cf, const float* __restrict__ x, float* __restrict__ ycell, int nx,
             int ny, int NX, int NY) {
  fe_pdl_enter();
  using S = CellStrip<P>;
  constexpr int N1 = S::N1, CX = S::CX, UW = S::UW;
  __shared__ float U[N1 * N1 * UW];               // [lz][ly][xl]
  // [lz][ly][c][lx]: the y contractions with M1 (A) and ay K1 (B), then in place the x
  // contractions W1 = M1 A (in A) and W2 = ax K1 A + M1 B (in B): an x line is read whole by
  // the one thread that overwrites it
  __shared__ float A[N1 * N1 * CX * N1];
  __shared__ float B[N1 * N1 * CX * N1];
  float* W1 = A;
  float* W2 = B;
  const int cy = blockIdx.y, cz = blockIdx.z;
  const int cx0 = blockIdx.x * CX;
  const int tid = threadIdx.x;
  const int64_t plane = (int64_t)NX * NY;

  // stage the strip (x periodic, so gx wraps; y periodic; z inside the slab)
  for (int e = tid; e < N1 * N1 * UW; e += S::NTHR) {
    const int xl = e % UW, ly = (e / UW) % N1, lz = e / (UW * N1);
    int gx = cx0 * P + xl;
    gx -= (gx >= NX) ? NX * (gx / NX) : 0;
    int gy = cy * P + ly;
    gy -= (gy >= NY) ? NY : 0;
    const int64_t gz = (int64_t)cz * P + lz;
    U[e] = x[gz * plane + (int64_t)gy * NX + gx];
  }
  __syncthreads();

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
  __syncthreads();
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
  __syncthreads();
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

// y at node (gx, gy, gz) = sum of its copies in the discontinuous grid; blocks of 32 x 8
// nodes of one plane (blockIdx.z strides over the planes)
template <int P>
__global__ void __launch_bounds__(256)
k_cell_gather(const float* __restrict__ ycell, float* __restrict__ y, int nx, int ny, int nz,
              int NX, int NY) {
  fe_pdl_enter();
  constexpr int N1 = P + 1;
  const int gx = blockIdx.x * 32 + threadIdx.x;
  const int gy = blockIdx.y * 8 + threadIdx.y;
  if (gx >= NX || gy >= NY) return;
  // the (cell, local index) copies of the node per direction, lower cell first
  int dx[2], dy[2], nxc = 0, nyc = 0;
  {
    const int c = gx / P, l = gx - c * P;
    if (l == 0) dx[nxc++] = (c == 0 ? nx - 1 : c - 1) * N1 + P;
    dx[nxc++] = c * N1 + l;
  }
  {
    const int c = gy / P, l = gy - c * P;
    if (l == 0) dy[nyc++] = (c == 0 ? ny - 1 : c - 1) * N1 + P;
    dy[nyc++] = c * N1 + l;
  }
  const int64_t dnx = (int64_t)nx * N1, dny = (int64_t)ny * N1;
  for (int gz = blockIdx.z; gz <= nz * P; gz += gridDim.z) {
    int dz[2], nzc = 0;
    const int c = gz / P, l = gz - c * P;
    if (l == 0 && c > 0) dz[nzc++] = (c - 1) * N1 + P;
    if (c < nz) dz[nzc++] = c * N1 + l;
    float s = 0.f;
    for (int a = 0; a < nzc; ++a)
      for (int b = 0; b < nyc; ++b) {
        const float* row = ycell + ((int64_t)dz[a] * dny + dy[b]) * dnx;
        for (int e = 0; e < nxc; ++e) s += row[dx[e]];
      }
    y[((int64_t)gz * NY + gy) * NX + gx] = s;
  }
}

template <int P>
fe_status cell_apply_p(const CellCoef& cf, const fe_mesh* m, const float* x, float* y,
                       float* ycell) {
  using S = CellStrip<P>;
  const int nstrip = (m->nx + S::CX - 1) / S::CX;
  if (m->ny > 65535 || m->nz > 65535) return fe_fail(FE_EINVAL, "cell operator: mesh too large");
  // programmatic dependent launches (each kernel waits for its predecessor at entry)
  FE_CUDA(fe_launch_pdl(k_cell_apply<P>, dim3(nstrip, m->ny, m->nz), dim3(S::NTHR), 0, m->stream,
                        cf, x, ycell, m->nx, m->ny, m->NX, m->NY));
  fe_count_launch();
  const int planes = m->NZ < 65535 ? m->NZ : 65535;
  const float* yc = ycell;
  FE_CUDA(fe_launch_pdl(k_cell_gather<P>, dim3((m->NX + 31) / 32, (m->NY + 7) / 8, planes),
                        dim3(32, 8), 0, m->stream, yc, y, m->nx, m->ny, m->nz, m->NX, m->NY));
  fe_count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // namespace

// scratch of the discontinuous grid: (p+1)^3 floats per cell
size_t fe_kcell_scratch_bytes(const fe_mesh* m) {
  const size_t n1 = (size_t)m->p + 1;
  return sizeof(float) * n1 * n1 * n1 * (size_t)m->nx * m->ny * m->nz;
}

fe_status fe_kcell_apply_f32(fe_mesh* m, const float* x, float* y) {
  void* ws = nullptr;
  FE_TRY(fe_ws(m, WS_KCELL, fe_kcell_scratch_bytes(m), &ws));
  CellCoef cf;
  const KronCoef& k = m->coefK;
  for (int j = 0; j < FE_MAXN1; ++j)
    for (int i = 0; i < FE_MAXN1; ++i) {
      cf.M1[j][i] = (float)k.AzM[j][i];
      cf.Ky[j][i] = (float)k.AyK[j][i];
      cf.Kx[j][i] = (float)k.AxK[j][i];
      cf.Kz[j][i] = (float)k.AzK[j][i];
    }
  float* yc = static_cast<float*>(ws);
  switch (m->p) {
    case 1: return cell_apply_p<1>(cf, m, x, y, yc);
    case 2: return cell_apply_p<2>(cf, m, x, y, yc);
    case 3: return cell_apply_p<3>(cf, m, x, y, yc);
    case 4: return cell_apply_p<4>(cf, m, x, y, yc);
    case 5: return cell_apply_p<5>(cf, m, x, y, yc);
    case 6: return cell_apply_p<6>(cf, m, x, y, yc);
    default: return fe_fail(FE_EUNSUPPORTED, "p = %d", m->p);
  }
}

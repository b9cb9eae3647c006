// Nonlocal pseudopotential term with synthetic projectors (Eq. V_nloc).
//
// (V_nloc psi)(x) = sum_a sum_beta p^a_beta(x - R_a) D^a_beta int p^a_beta(y - R_a) psi(y) dy
// with one s and three p channels per atom: g(d) = exp(-|d|^2 / (2 s_a^2)),
// p_s = g, p_x = (d_x / s_a) g, p_y = (d_y / s_a) g, p_z = (d_z / s_a) g, summed over the
// periodic x/y images and cut at |d| <= rc.  With the lumped quadrature <N_I, p> ~ M_II p(x_I)
// the scaled operator is Ht_nloc = M^1/2 P D P^T M^1/2 (Section 2.3's H u = eps M u).
//
// Layout: the nonzeros of Pt = M^1/2 P are kept atom-major (entry e: psi node, atom, four
// channel values) for the projection C[a][beta][v] = sum_e Pt[e][beta] X[node_e][v], and
// node-major (the entries of each touched psi node) for the output-stationary update
// Y[node][v] += alpha sum_{e at node} sum_beta Pt[e][beta] D[a_e][beta] C[a_e][beta][v]: every
// output entry is written by one thread, no atomics.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "fe_internal.h"

namespace {

constexpr int NCHAN = 4;
constexpr int PROJ_THREADS = 128;

// C[a][beta][v] for one atom and a tile of PROJ_THREADS vectors
template <typename T>
__global__ void k_nl_project(const T* __restrict__ X, int64_t ld, int64_t nvec,
                             const int* __restrict__ atom_ptr, const int* __restrict__ ent_node,
                             const T* __restrict__ ent_val, T* __restrict__ C) {
  const int a = blockIdx.x;
  const int64_t v = (int64_t)blockIdx.y * PROJ_THREADS + threadIdx.x;
  if (v >= nvec) return;
  T c0 = T(0), c1 = T(0), c2 = T(0), c3 = T(0);
  for (int e = atom_ptr[a]; e < atom_ptr[a + 1]; ++e) {
    const T x = X[(int64_t)ent_node[e] * ld + v];
    c0 += ent_val[4 * e + 0] * x;
    c1 += ent_val[4 * e + 1] * x;
    c2 += ent_val[4 * e + 2] * x;
    c3 += ent_val[4 * e + 3] * x;
  }
  T* Ca = C + (int64_t)a * NCHAN * nvec;
  Ca[v] = c0;
  Ca[nvec + v] = c1;
  Ca[2 * nvec + v] = c2;
  Ca[3 * nvec + v] = c3;
}

// Y[node][v] += alpha sum_e sum_beta Pt[e][beta] D[a_e][beta] C[a_e][beta][v]; one warp per
// touched node, lanes over the vectors
template <typename T>
__global__ void k_nl_apply(T* __restrict__ Y, int64_t ld, int64_t nvec, int ntouched,
                           const int* __restrict__ tn_node, const int* __restrict__ tn_ptr,
                           const int* __restrict__ tn_ent, const int* __restrict__ ent_atom,
                           const T* __restrict__ ent_val, const T* __restrict__ Dv,
                           const T* __restrict__ C, T alpha) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntouched; t += warps) {
    T* yrow = Y + (int64_t)tn_node[t] * ld;
    const int e0 = tn_ptr[t], e1 = tn_ptr[t + 1];
    for (int64_t v = lane; v < nvec; v += 32) {
      T acc = T(0);
      for (int k = e0; k < e1; ++k) {
        const int e = tn_ent[k];
        const int a = ent_atom[e];
        const T* Ca = C + (int64_t)a * NCHAN * nvec;
#pragma unroll
        for (int b = 0; b < NCHAN; ++b) acc += ent_val[4 * e + b] * Dv[4 * a + b] * Ca[b * nvec + v];
      }
      yrow[v] += alpha * acc;
    }
  }
}

template <typename T>
T* dev_copy(const std::vector<T>& h, fe_status* st) {
  T* d = nullptr;
  if (h.empty()) return nullptr;
  if (cudaMalloc(&d, sizeof(T) * h.size()) != cudaSuccess ||
      cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    if (d) cudaFree(d);
    *st = fe_fail(FE_ENOMEM, "nonlocal tables of %zu bytes", sizeof(T) * h.size());
    return nullptr;
  }
  return d;
}

}  // namespace

void fe_nonlocal_free(fe_mesh* m) {
  void* ptrs[] = {m->nl.atom_ptr, m->nl.ent_node, m->nl.ent_atom, m->nl.ent_val, m->nl.ent_val_f,
                  m->nl.D, m->nl.D_f, m->nl.tn_node, m->nl.tn_ptr, m->nl.tn_ent};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  m->nl = FeNonlocal{};
}

extern "C" fe_status fe_set_nonlocal(fe_mesh* m, int natoms, const double* R, const double* sigma,
                                     const double* D, double rc) {
  if (!m) return fe_fail(FE_EINVAL, "fe_set_nonlocal: null mesh");
  if (natoms < 0) return fe_fail(FE_EINVAL, "fe_set_nonlocal: natoms < 0");
  FE_TRY(fe_activate(m));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  fe_nonlocal_free(m);
  if (natoms == 0) return FE_OK;
  if (!R || !sigma || !D) return fe_fail(FE_EINVAL, "fe_set_nonlocal: null array");
  if (!(rc > 0.0)) return fe_fail(FE_EINVAL, "fe_set_nonlocal: need rc > 0");
  for (int a = 0; a < natoms; ++a)
    if (!(sigma[a] > 0.0)) return fe_fail(FE_EINVAL, "fe_set_nonlocal: atom %d: sigma <= 0", a);
  const int p = m->p;
  const double Lx = m->desc.L[0], Ly = m->desc.L[1];
  auto coord = [&](int g, int d) { return (g / p) * m->h[d] + (m->xi[g % p] + 1.0) * 0.5 * m->h[d]; };
  auto mass1 = [&](int g, bool periodic, int gmax) {
    const int l = g % p;
    if (l) return m->w[l];
    if (periodic) return 2.0 * m->w[0];
    return (g == 0 || g == gmax) ? m->w[0] : 2.0 * m->w[0];
  };
  const int gzmax = m->nz * p;
  std::vector<int> atom_ptr(natoms + 1, 0), ent_node, ent_atom;
  std::vector<double> ent_val;
  for (int a = 0; a < natoms; ++a) {
    const double s = sigma[a];
    std::unordered_map<int64_t, int> at;   // psi node -> entry of this atom
    // unwrapped x / y node indices around the atom: each (node, periodic image) pair within
    // rc appears once, the image being (g - wrapped g) / N periods away
    const double cx = R[3 * a], cy = R[3 * a + 1], cz = R[3 * a + 2];
    const int x0 = (int)std::floor((cx - rc) / m->h[0]) * p, x1 = ((int)std::floor((cx + rc) / m->h[0]) + 1) * p;
    const int y0 = (int)std::floor((cy - rc) / m->h[1]) * p, y1 = ((int)std::floor((cy + rc) / m->h[1]) + 1) * p;
    const int z0 = std::max((int)std::floor((cz - rc) / m->h[2]) * p, m->gz_lo);
    const int z1 = std::min(((int)std::floor((cz + rc) / m->h[2]) + 1) * p, m->gz_lo + m->NZs - 1);
    for (int gz = z0; gz <= z1; ++gz) {
      const double dz = coord(gz, 2) - cz;
      for (int gy = y0; gy <= y1; ++gy) {
        const int wy = ((gy % m->NY) + m->NY) % m->NY;
        const double dy = (double)((gy - wy) / m->NY) * Ly + coord(wy, 1) - cy;
        for (int gx = x0; gx <= x1; ++gx) {
          const int wx = ((gx % m->NX) + m->NX) % m->NX;
          const double dx = (double)((gx - wx) / m->NX) * Lx + coord(wx, 0) - cx;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > rc * rc) continue;
          const int64_t node = (int64_t)(gz - m->gz_lo) * m->NX * m->NY + (int64_t)wy * m->NX + wx;
          const double g = std::exp(-r2 / (2.0 * s * s));
          const double sm = std::sqrt(m->J * mass1(wx, true, 0) * mass1(wy, true, 0) * mass1(gz, false, gzmax));
          int e;
          auto it = at.find(node);
          if (it == at.end()) {
            e = (int)ent_node.size();
            at.emplace(node, e);
            ent_node.push_back((int)node);
            ent_atom.push_back(a);
            ent_val.insert(ent_val.end(), 4, 0.0);
          } else {
            e = it->second;
          }
          ent_val[4 * e + 0] += sm * g;
          ent_val[4 * e + 1] += sm * dx / s * g;
          ent_val[4 * e + 2] += sm * dy / s * g;
          ent_val[4 * e + 3] += sm * dz / s * g;
        }
      }
    }
    atom_ptr[a + 1] = (int)ent_node.size();
  }
  // node-major lists
  const int nnz = (int)ent_node.size();
  std::vector<int> order(nnz);
  for (int e = 0; e < nnz; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ent_node[x] < ent_node[y]; });
  std::vector<int> tn_node, tn_ptr(1, 0);
  for (int k = 0; k < nnz; ++k) {
    if (tn_node.empty() || tn_node.back() != ent_node[order[k]]) {
      if (!tn_node.empty()) tn_ptr.push_back(k);
      tn_node.push_back(ent_node[order[k]]);
    }
  }
  tn_ptr.push_back(nnz);
  if (tn_node.empty()) tn_ptr.assign(1, 0);
  std::vector<double> Dv(D, D + 4 * (size_t)natoms);
  std::vector<float> ent_val_f(ent_val.begin(), ent_val.end()), D_f(Dv.begin(), Dv.end());
  fe_status st = FE_OK;
  FeNonlocal nl{};
  nl.natoms = natoms;
  nl.nnz = nnz;
  nl.ntouched = (int)tn_node.size();
  nl.atom_ptr = dev_copy(atom_ptr, &st);
  nl.ent_node = dev_copy(ent_node, &st);
  nl.ent_atom = dev_copy(ent_atom, &st);
  nl.ent_val = dev_copy(ent_val, &st);
  nl.ent_val_f = dev_copy(ent_val_f, &st);
  nl.D = dev_copy(Dv, &st);
  nl.D_f = dev_copy(D_f, &st);
  nl.tn_node = dev_copy(tn_node, &st);
  nl.tn_ptr = dev_copy(tn_ptr, &st);
  nl.tn_ent = dev_copy(order, &st);
  m->nl = nl;
  if (st != FE_OK) {
    fe_nonlocal_free(m);
    return st;
  }
  return FE_OK;
}

// Y += alpha Ht_nloc X (float or double blocks; the bf16 tensor-core path uses float blocks)
fe_status fe_nonlocal_apply(fe_mesh* m, const void* X, void* Y, int64_t nvec, int64_t ld,
                            double alpha, bool dbl) {
  const FeNonlocal& nl = m->nl;
  if (nl.natoms == 0 || nl.nnz == 0) return FE_OK;
  cudaStream_t st = m->stream;
  const size_t eb = dbl ? 8 : 4;
  void* c;
  FE_TRY(fe_ws(m, WS_NL, eb * NCHAN * (size_t)nl.natoms * nvec + 64, &c));
  dim3 pg(nl.natoms, (unsigned)((nvec + PROJ_THREADS - 1) / PROJ_THREADS));
  int ab = (nl.ntouched + 7) / 8;
  if (ab > 152 * 32) ab = 152 * 32;
  if (dbl) {
    k_nl_project<double><<<pg, PROJ_THREADS, 0, st>>>((const double*)X, ld, nvec, nl.atom_ptr,
                                                      nl.ent_node, nl.ent_val, (double*)c);
    fe_count_launch();
    k_nl_apply<double><<<ab, 256, 0, st>>>((double*)Y, ld, nvec, nl.ntouched, nl.tn_node, nl.tn_ptr,
                                           nl.tn_ent, nl.ent_atom, nl.ent_val, nl.D,
                                           (const double*)c, alpha);
    fe_count_launch();
  } else {
    k_nl_project<float><<<pg, PROJ_THREADS, 0, st>>>((const float*)X, ld, nvec, nl.atom_ptr,
                                                     nl.ent_node, nl.ent_val_f, (float*)c);
    fe_count_launch();
    k_nl_apply<float><<<ab, 256, 0, st>>>((float*)Y, ld, nvec, nl.ntouched, nl.tn_node, nl.tn_ptr,
                                          nl.tn_ent, nl.ent_atom, nl.ent_val_f, nl.D_f,
                                          (const float*)c, (float)alpha);
    fe_count_launch();
  }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

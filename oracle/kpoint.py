"""Bloch k-point Hamiltonian of the slab (Section 2.1: Bloch's theorem along the periodic x
and y directions, psi = e^{i k.x} u with u lattice-periodic, and the local operator
H^k_loc = -1/2 Laplacian - i k.grad + 1/2 |k|^2 + V_eff acting on u).

Test infrastructure only (like every module of this package): tests, the smoke check and the
benchmark's CPU baseline may import it; the library never does.

* k = (kx, ky) lies in the periodic plane.  With the real FE basis the weak form of H^k_loc
  is H_k = 1/2 K - i (kx Gx + ky Gy) + 1/2 |k|^2 M + M diag(V), where
  G^d_IJ = int N_I dN_J/dx_d is integrated exactly cell by cell (the quadrature of K).  With
  periodic x and y, integration by parts gives G^T = -G after assembly, so -i G is
  Hermitian.
* Reading (the paper does not say how the |k|^2 term is integrated): with the lumped overlap
  M, the same as in H u = eps M u, so that in the scaled standard form
      Ht_k = M^-1/2 H_k M^-1/2 = Ht_0 + 1/2 |k|^2 I - i M^-1/2 (kx Gx + ky Gy) M^-1/2
  the term is the constant 1/2 |k|^2.  Ht_0 is the Gamma-point operator of assembly.py.
* psi nodes on a homogeneous-Dirichlet z face are removed, as for Ht_0.
"""
import numpy as np
import scipy.sparse as sp

from . import assembly
from .basis import gauss_legendre, lagrange_derivs, lagrange_values


def reference_cell_gradient(mesh, axis):
    """Cell matrix G_e[I, J] = int_cell N_I dN_J/dx_axis by (p+1)^3-point Gauss quadrature."""
    p = mesh.p
    h = mesh.h
    q, wq = gauss_legendre(p + 1)
    B = lagrange_values(mesh.xi, q)   # [a, i]
    D = lagrange_derivs(mesh.xi, q)   # [a, i]
    n1 = p + 1
    nq = len(q)
    detJ = h[0] * h[1] * h[2] / 8.0
    # quadrature point (a, b, c) -> a + nq (b + nq c); node (i, j, k) -> i + n1 (j + n1 k)
    N = np.einsum("ai,bj,ck->cbakji", B, B, B).reshape(nq ** 3, n1 ** 3)
    if axis == 0:
        dN = np.einsum("ai,bj,ck->cbakji", D, B, B).reshape(nq ** 3, n1 ** 3) * (2.0 / h[0])
    elif axis == 1:
        dN = np.einsum("ai,bj,ck->cbakji", B, D, B).reshape(nq ** 3, n1 ** 3) * (2.0 / h[1])
    else:
        raise ValueError("k lies in the periodic x-y plane")
    W = np.einsum("a,b,c->cba", wq, wq, wq).reshape(-1) * detJ
    return N.T @ (W[:, None] * dN)


def assemble_gradient(mesh, axis):
    """Global G^axis on phi nodes (periodic x/y), CSR."""
    Ge = reference_cell_gradient(mesh, axis)
    cn = mesh.cell_nodes()
    ne = mesh.ne
    rows = np.repeat(cn, ne, axis=1).ravel()
    cols = np.tile(cn, (1, ne)).ravel()
    data = np.tile(Ge.ravel(), mesh.n_cells)
    G = sp.coo_matrix((data, (rows, cols)), shape=(mesh.n_phi, mesh.n_phi)).tocsr()
    G.sum_duplicates()
    return G


def hamiltonian_k(mesh, V_psi, k, K=None, M=None):
    """Ht_k (complex CSR on psi nodes) for the in-plane wave vector k = (kx, ky)."""
    kx, ky = float(k[0]), float(k[1])
    K = assembly.assemble_stiffness(mesh) if K is None else K
    M = assembly.lumped_mass(mesh) if M is None else M
    H0 = assembly.hamiltonian(mesh, V_psi, K, M)
    ids = mesh.psi_to_phi()
    G = kx * assemble_gradient(mesh, 0) + ky * assemble_gradient(mesh, 1)
    s = sp.diags(1.0 / np.sqrt(M[ids]))
    A = (s @ G[ids][:, ids] @ s).tocsr()
    n = len(ids)
    return (H0.astype(np.complex128) + 0.5 * (kx * kx + ky * ky) * sp.identity(n, format="csr")
            - 1j * A).tocsr()


def apply_Hk_rows(mesh, V_psi, k, X, rows, M=None):
    """(Ht_k X)[rows, :] from the cell definition, one row at a time (for sizes where the
    assembled matrix does not fit): the Gamma-point rows of assembly.apply_H_rows, plus
    1/2 |k|^2 X_I, minus i S_I sum over the cells e touching I of
    sum_J (kx Gx_e + ky Gy_e)[l_I, J] (S X)_{node_e(J)} (S = M^-1/2, X = 0 on Dirichlet
    nodes).  X is complex; only the rows the sampled cells touch are promoted."""
    kx, ky = float(k[0]), float(k[1])
    M = assembly.lumped_mass(mesh) if M is None else M
    X = np.asarray(X)
    Xc = lambda idx: X[idx].astype(np.complex128)
    re = assembly.apply_H_rows(mesh, V_psi, X.real, rows, M=M)
    im = assembly.apply_H_rows(mesh, V_psi, X.imag, rows, M=M)
    out = re + 1j * im
    Ge = kx * reference_cell_gradient(mesh, 0) + ky * reference_cell_gradient(mesh, 1)
    cn = mesh.cell_nodes()
    off = mesh.NX * mesh.NY * mesh.gz_lo
    NX, NY = mesh.NX, mesh.NY
    for r, I in enumerate(rows):
        g = int(I) + off
        gx, gy, gz = g % NX, (g // NX) % NY, g // (NX * NY)
        acc = np.zeros(X.shape[1], dtype=np.complex128)
        for e, l in mesh.node_cells(gx, gy, gz):
            nodes = cn[e]
            psi = nodes - off
            ok = (psi >= 0) & (psi < mesh.n_psi)
            sx = np.zeros((len(nodes), X.shape[1]), dtype=np.complex128)
            sx[ok] = Xc(psi[ok]) / np.sqrt(M[nodes[ok]])[:, None]
            acc += Ge[l] @ sx
        out[r] += 0.5 * (kx * kx + ky * ky) * Xc(int(I)) - 1j * acc / np.sqrt(M[g])
    return out

"""Finite-element matrices of Section 2.3 and the Kohn-Sham Hamiltonian of Eq. Veff and Hloc.

* K_IJ = int grad N_I . grad N_J over Omega_p (Section 2.3), assembled cell by cell from
  the reference-cell matrix computed by (p+1)^3-point Gauss-Legendre quadrature, which is
  exact for the degree-2p integrand on an affine hexahedron.
* M is the FE overlap of H u = eps M u (Section 2.3).  Reading (the paper does not say):
  the spectral-element GLL-lumped diagonal M_II = sum over cells of w_i w_j w_k |J|.
* The local Hamiltonian H_loc = -1/2 Laplacian + V_eff (Eq. Veff and Hloc) discretises to
  H = 1/2 K + M diag(V) with V collocated at the nodes (reading: GLL collocation).  The
  generalised problem H u = eps M u is solved in the symmetric standard form
  Ht = M^-1/2 H M^-1/2 = 1/2 M^-1/2 K M^-1/2 + diag(V), which has the same eigenvalues.
* psi nodes on a homogeneous-Dirichlet z face are removed (rows and columns dropped).
"""
import numpy as np
import scipy.sparse as sp

from .basis import gauss_legendre, lagrange_derivs, lagrange_values


def reference_cell_stiffness(mesh):
    """Cell stiffness K_e[I, J] = int_cell grad N_I . grad N_J by 3D quadrature."""
    p = mesh.p
    hx, hy, hz = mesh.h
    q, wq = gauss_legendre(p + 1)
    B = lagrange_values(mesh.xi, q)   # [a, i]
    D = lagrange_derivs(mesh.xi, q)   # [a, i]
    n1 = p + 1
    nq = len(q)
    detJ = hx * hy * hz / 8.0
    # gradients of every 3D basis function at every 3D quadrature point
    # quadrature point (a, b, c) -> a + nq (b + nq c); node (i, j, k) -> i + n1 (j + n1 k)
    Gx = np.einsum("ai,bj,ck->cbakji", D, B, B).reshape(nq ** 3, n1 ** 3) * (2.0 / hx)
    Gy = np.einsum("ai,bj,ck->cbakji", B, D, B).reshape(nq ** 3, n1 ** 3) * (2.0 / hy)
    Gz = np.einsum("ai,bj,ck->cbakji", B, B, D).reshape(nq ** 3, n1 ** 3) * (2.0 / hz)
    W = np.einsum("a,b,c->cba", wq, wq, wq).reshape(-1) * detJ
    return Gx.T @ (W[:, None] * Gx) + Gy.T @ (W[:, None] * Gy) + Gz.T @ (W[:, None] * Gz)


def reference_cell_mass_lumped(mesh):
    """GLL-lumped cell mass w_i w_j w_k |J| per local node."""
    w = mesh.w
    detJ = np.prod(mesh.h) / 8.0
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1) * detJ


def assemble_stiffness(mesh):
    """Global K on phi nodes (periodic x/y, all z planes), CSR."""
    Ke = reference_cell_stiffness(mesh)
    cn = mesh.cell_nodes()
    ne = mesh.ne
    rows = np.repeat(cn, ne, axis=1).ravel()
    cols = np.tile(cn, (1, ne)).ravel()
    data = np.tile(Ke.ravel(), mesh.n_cells)
    K = sp.coo_matrix((data, (rows, cols)), shape=(mesh.n_phi, mesh.n_phi)).tocsr()
    K.sum_duplicates()
    return K


def lumped_mass(mesh):
    """Diagonal of the lumped M on phi nodes."""
    me = reference_cell_mass_lumped(mesh)
    cn = mesh.cell_nodes()
    return np.bincount(cn.ravel(), weights=np.tile(me, mesh.n_cells), minlength=mesh.n_phi)


def hamiltonian(mesh, V_psi, K=None, M=None):
    """Ht = 1/2 M^-1/2 K M^-1/2 + diag(V) on psi nodes, CSR."""
    K = assemble_stiffness(mesh) if K is None else K
    M = lumped_mass(mesh) if M is None else M
    ids = mesh.psi_to_phi()
    Kp = K[ids][:, ids]
    s = 1.0 / np.sqrt(M[ids])
    S = sp.diags(s)
    return (0.5 * (S @ Kp @ S) + sp.diags(np.asarray(V_psi, dtype=np.float64))).tocsr()


def apply_H_rows(mesh, V_psi, X, rows, Ke=None, M=None):
    """(Ht X)[rows, :] evaluated one row at a time from the cell definition.

    For a psi row I: (K S X)_I = sum over cells e touching I of
    sum_J K_e[l_I, J] (S X)_{node_e(J)}, with S = M^-1/2 and X = 0 on Dirichlet nodes;
    then (Ht X)_I = 1/2 S_I (K S X)_I + V_I X_I.  Used at sizes where the assembled
    matrix does not fit.
    """
    Ke = reference_cell_stiffness(mesh) if Ke is None else Ke
    if M is None:
        M = lumped_mass(mesh)
    cn = mesh.cell_nodes()
    X = np.asarray(X)
    off = mesh.NX * mesh.NY * mesh.gz_lo
    out = np.zeros((len(rows), X.shape[1]))
    for r, I in enumerate(rows):
        phi_I = int(I) + off
        gx = phi_I % mesh.NX
        gy = (phi_I // mesh.NX) % mesh.NY
        gz = phi_I // (mesh.NX * mesh.NY)
        acc = np.zeros(X.shape[1])
        for cell, loc in mesh.node_cells(gx, gy, gz):
            nodes = cn[cell]
            psi = nodes - off
            ok = (psi >= 0) & (psi < mesh.n_psi)
            xs = np.zeros((mesh.ne, X.shape[1]))
            xs[ok] = X[psi[ok]].astype(np.float64) / np.sqrt(M[nodes[ok]])[:, None]
            acc += Ke[loc] @ xs
        out[r] = 0.5 * acc / np.sqrt(M[phi_I]) + V_psi[int(I)] * X[int(I)].astype(np.float64)
    return out

"""Potential term integrated by Gauss quadrature (the consistent, cell-matrix form of the
potential in the discretised Kohn-Sham operator of Section 2.3).

Test infrastructure only (like every module of this package): tests, the smoke check and the
benchmark's CPU baseline may import it; the library never does.

The weak form of V_eff u gives the matrix V_IJ = int N_I V_eff N_J dx.  Instead of the GLL
collocation (diagonal M_II V(x_I)) it is integrated here cell by cell with the
(p+1)-point Gauss-Legendre rule per direction, V_eff given at the Gauss points:

    V_e[I, J] = sum_q w_q |J_e| V_e(x_q) N_I(x_q) N_J(x_q),

exact when V_eff is a polynomial of degree <= 1 per direction (N_I N_J V then has degree
<= 2 p + 1, the exactness degree of the rule).  The overlap stays the lumped M, so the
scaled operator is Ht_q = M^-1/2 (1/2 K + V) M^-1/2 on psi nodes.

Layout of a quadrature field: [n_cells, nq^3] with cells in the mesh order (cx fastest)
and point (a, b, c) (a along x) at a + nq (b + nq c), nq = p + 1.
"""
import numpy as np
import scipy.sparse as sp

from . import assembly
from .basis import gauss_legendre, lagrange_values


def n_quad(mesh):
    """Gauss points per direction (p + 1)."""
    return mesh.p + 1


def reference_interpolation(mesh):
    """B[q, I] = N_I(x_q) on the reference cell, q and I in the cell orderings, and the
    tensor-product weights w_q |J| (|J| = hx hy hz / 8)."""
    nq = n_quad(mesh)
    q, wq = gauss_legendre(nq)
    B1 = lagrange_values(mesh.xi, q)                      # [a, i]
    B = np.einsum("ai,bj,ck->cbakji", B1, B1, B1).reshape(nq ** 3, (mesh.p + 1) ** 3)
    detJ = mesh.h[0] * mesh.h[1] * mesh.h[2] / 8.0
    W = np.einsum("a,b,c->cba", wq, wq, wq).reshape(-1) * detJ
    return B, W


def quadrature_points(mesh):
    """Physical coordinates of every cell's Gauss points, [n_cells, nq^3, 3]."""
    nq = n_quad(mesh)
    q, _ = gauss_legendre(nq)
    nx, ny, nz = mesh.ncell
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    corner = np.column_stack([cx.ravel() * mesh.h[0], cy.ravel() * mesh.h[1],
                              cz.ravel() * mesh.h[2]])
    c, b, a = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing="ij")
    loc = np.column_stack([(q[a.ravel()] + 1.0) * 0.5 * mesh.h[0],
                           (q[b.ravel()] + 1.0) * 0.5 * mesh.h[1],
                           (q[c.ravel()] + 1.0) * 0.5 * mesh.h[2]])
    return corner[:, None, :] + loc[None, :, :]


def interpolate_to_quad(mesh, f_phi):
    """Values at every cell's Gauss points of the FE field with nodal values f_phi (phi
    nodes): f(x_q) = sum_I N_I(x_q) f_I."""
    B, _ = reference_interpolation(mesh)
    cn = mesh.cell_nodes()
    return np.asarray(f_phi, dtype=np.float64)[cn] @ B.T


def potential_matrix(mesh, Vq):
    """Assembled V (phi nodes, CSR) from V_eff at the Gauss points, Vq [n_cells, nq^3]."""
    B, W = reference_interpolation(mesh)
    Vq = np.asarray(Vq, dtype=np.float64).reshape(mesh.n_cells, -1)
    cn = mesh.cell_nodes()
    ne = cn.shape[1]
    # V_e = B^T diag(W Vq_e) B for every cell
    Ve = np.einsum("qi,eq,qj->eij", B, Vq * W[None, :], B)
    rows = np.repeat(cn, ne, axis=1).ravel()
    cols = np.tile(cn, (1, ne)).ravel()
    V = sp.coo_matrix((Ve.ravel(), (rows, cols)), shape=(mesh.n_phi, mesh.n_phi)).tocsr()
    V.sum_duplicates()
    return V


def hamiltonian_quad(mesh, Vq, K=None, M=None):
    """Ht_q = M^-1/2 (1/2 K + V) M^-1/2 on psi nodes (CSR), V from potential_matrix."""
    K = assembly.assemble_stiffness(mesh) if K is None else K
    M = assembly.lumped_mass(mesh) if M is None else M
    ids = mesh.psi_to_phi()
    A = (0.5 * K + potential_matrix(mesh, Vq))[ids][:, ids]
    S = sp.diags(1.0 / np.sqrt(M[ids]))
    return (S @ A @ S).tocsr()


def apply_Hq_rows(mesh, Vq, X, rows, M=None):
    """(Ht_q X)[rows, :] from the cell definition, one row at a time (for sizes where the
    assembled matrix does not fit): the stiffness part as in assembly.apply_H_rows with a
    zero collocated potential, plus S_I sum over the cells e touching I of
    sum_J V_e[l_I, J] (S X)_{node_e(J)} (S = M^-1/2, X = 0 on Dirichlet nodes).  X may be
    float32; only the rows the sampled cells touch are promoted."""
    M = assembly.lumped_mass(mesh) if M is None else M
    X = np.asarray(X)
    out = assembly.apply_H_rows(mesh, np.zeros(mesh.n_psi), X, rows, M=M)
    B, W = reference_interpolation(mesh)
    Vq = np.asarray(Vq, dtype=np.float64).reshape(mesh.n_cells, -1)
    cn = mesh.cell_nodes()
    off = mesh.NX * mesh.NY * mesh.gz_lo
    NX, NY = mesh.NX, mesh.NY
    for r, I in enumerate(rows):
        g = int(I) + off
        gx, gy, gz = g % NX, (g // NX) % NY, g // (NX * NY)
        acc = np.zeros(X.shape[1])
        for e, l in mesh.node_cells(gx, gy, gz):
            nodes = cn[e]
            psi = nodes - off
            ok = (psi >= 0) & (psi < mesh.n_psi)
            sx = np.zeros((len(nodes), X.shape[1]))
            sx[ok] = X[psi[ok]].astype(np.float64) / np.sqrt(M[nodes[ok]])[:, None]
            Ve_row = (B[:, l] * W * Vq[e]) @ B          # V_e[l, :]
            acc += Ve_row @ sx
        out[r] += acc / np.sqrt(M[g])
    return out

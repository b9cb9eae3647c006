"""Finite-element Poisson problem with the CEF and CPD / L-CPD boundary conditions.

* Eq. Poissons equation: -1/(4 pi) Lap phi = rho + b.  Its FE form (Section 2.3) is
  K phi = 4 pi c with c_I = int N_I (rho + b); with the lumped overlap this is
  c_I = M_II (rho + b)(x_I) (reading: GLL collocation of the load).
* CEF (Eq. governing_equations CEF): periodic x/y, zero-Neumann on both z faces (the
  natural boundary condition of the weak form) and int phi = 0, i.e. sum_I M_II phi_I = 0.
  The load is projected onto the range of K first: f <- f - (sum f / sum M) M.
* CPD / L-CPD (Eq. governing_equations APD): phi is prescribed on the conductor node
  sets; the free rows solve K_ff phi_f = f_f - K_fc phi_c; z faces outside the
  conductors keep the natural (zero-Neumann) condition.
* The exact solution of these linear systems is the definition; ``solve_*_direct`` writes
  it out with a sparse LU factorisation.  ``pcg`` is the textbook Jacobi-preconditioned
  conjugate-gradient iteration used by the solver under test.
* Energy (Eq. electrostatics Energy and Eq. KS DFT variational problem cef at fixed rho):
  E = c.phi - phi^T K phi / (8 pi) + int (V_loc - V_sm) rho + int (rho + b) V_app, integrals
  with the lumped weights (the smeared-charge self energy is a constant in the bias and
  the atom positions and is left out).
* Dipole (Section 3.1): mu_z = int (b + rho) (z - Lz/2), about the domain centre.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def load_vector(M, rho, b):
    """c_I = M_II (rho + b)(x_I)."""
    return M * (rho + b)


def project_neutral(f, M):
    return f - (np.sum(f) / np.sum(M)) * M


def solve_cef_direct(K, f, M):
    """Neumann-z problem with sum M phi = 0 via the bordered (Lagrange multiplier) system."""
    n = K.shape[0]
    f = project_neutral(f, M)
    A = sp.bmat([[K, sp.csr_matrix(M.reshape(-1, 1))],
                 [sp.csr_matrix(M.reshape(1, -1)), None]], format="csc")
    rhs = np.concatenate([f, [0.0]])
    sol = spla.spsolve(A, rhs)
    return sol[:n]


def solve_cpd_direct(K, f, mask, values):
    """Dirichlet-constrained problem: K_ff phi_f = f_f - K_fc phi_c."""
    free = ~mask
    Kff = K[free][:, free].tocsc()
    Kfc = K[free][:, mask]
    phi = np.array(values, dtype=np.float64)
    phi[~mask] = spla.spsolve(Kff, f[free] - Kfc @ values[mask])
    return phi


def pcg(A_mul, b, Dinv, x0=None, rtol=1e-10, maxit=10000, project=None):
    """Textbook Jacobi-preconditioned CG; returns (x, iterations, relative residual)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A_mul(x)
    if project is not None:
        r = project(r)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    z = Dinv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit and np.linalg.norm(r) > rtol * bn:
        Ap = A_mul(p)
        alpha = rz / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        if project is not None:
            r = project(r)
        z = Dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, float(np.linalg.norm(r) / bn)


def solve_cef_cg(K, f, M, rtol=1e-10, maxit=10000):
    f = project_neutral(f, M)
    Dinv = 1.0 / K.diagonal()
    proj = lambda v: v - np.mean(v)
    x, it, rel = pcg(lambda v: K @ v, f, Dinv, rtol=rtol, maxit=maxit, project=proj)
    x -= (M @ x) / np.sum(M)
    return x, it, rel


def solve_cpd_cg(K, f, mask, values, rtol=1e-10, maxit=10000):
    free = ~mask
    Kff = K[free][:, free].tocsr()
    Kfc = K[free][:, mask]
    rhs = f[free] - Kfc @ values[mask]
    Dinv = 1.0 / Kff.diagonal()
    xf, it, rel = pcg(lambda v: Kff @ v, rhs, Dinv, rtol=rtol, maxit=maxit)
    phi = np.array(values, dtype=np.float64)
    phi[free] = xf
    return phi, it, rel


def electrostatic_energy(K, phi, c):
    """c . phi - phi^T K phi / (8 pi) (Eq. electrostatics Energy without self energy)."""
    return float(c @ phi - phi @ (K @ phi) / (8.0 * math.pi))


def total_energy(K, phi, M, rho, b, vlms, vapp):
    c = load_vector(M, rho, b)
    return (electrostatic_energy(K, phi, c) + float(M @ (vlms * rho))
            + float(M @ ((rho + b) * vapp)))


def reaction_charge(K, phi, M, rho, b, om1):
    """dE/d(dV) for CPD: sum over Omega_1 of c_I - (K phi)_I / (4 pi)."""
    c = load_vector(M, rho, b)
    return float(np.sum((c - (K @ phi) / (4.0 * math.pi))[om1]))


def dipole_z(M, rho, b, z, Lz):
    return float(M @ ((rho + b) * (z - 0.5 * Lz)))

"""Chebyshev-filtered subspace iteration for the discrete eigenproblem H u = eps M u.

Section 2.3 states the generalised FE eigenproblem and defers the eigensolver to the
authors' earlier work; the Kohn-Sham problem needs the smallest N >= N_e/2 eigenpairs
(Section 2.1, below Eq. KS DFT variational problem).  The steps written out here are
the standard published forms:

* scaled three-term Chebyshev filter (Zhou & Saad, J. Comput. Phys. 219 (2006);
  SIAM J. Matrix Anal. Appl. 29 (2007)): with e = (b - a)/2, c = (b + a)/2 and
  sigma_1 = e / (a0 - c), the degree-m filter returns
  T_m((H - c)/e) X / T_m((a0 - c)/e); degree m counts applications of H;
* k-step Lanczos spectral bounds (Zhou & Li, Linear Algebra Appl. 435 (2011)):
  upper bound theta_max + ||f_k||;
* Rayleigh-Ritz with Householder QR and a dense symmetric eigensolver.
"""
import numpy as np


def cheb_filter(apply_H, X, m, a, b, a0):
    """Degree-m scaled Chebyshev filter of X for the damped interval [a, b]."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma = e / (a0 - c)
    tau = 2.0 / sigma
    # real blocks in double; complex (Bloch) blocks in double complex, same recurrence
    X = np.asarray(X, dtype=np.complex128 if np.iscomplexobj(X) else np.float64)
    Y = (sigma / e) * (apply_H(X) - c * X)
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        Ynew = (2.0 * sigma_new / e) * (apply_H(Y) - c * Y) - (sigma * sigma_new) * X
        X = Y
        Y = Ynew
        sigma = sigma_new
    return Y


def lanczos_bounds(apply_H, v0, k):
    """k-step Lanczos: (smallest Ritz value, largest Ritz value + ||f_k||)."""
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    f = apply_H(v)
    alpha = float(f @ v)
    f = f - alpha * v
    alphas, betas = [alpha], []
    for _ in range(1, k):
        beta = float(np.linalg.norm(f))
        v_old = v
        v = f / beta
        f = apply_H(v) - beta * v_old
        alpha = float(f @ v)
        f = f - alpha * v
        alphas.append(alpha)
        betas.append(beta)
    T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    theta = np.linalg.eigvalsh(T)
    return float(theta[0]), float(theta[-1] + np.linalg.norm(f))


def rayleigh_ritz(apply_H, Y):
    """Orthonormalise (Householder QR) then diagonalise the projected matrix."""
    Q, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64))
    Hs = Q.T @ apply_H(Q)
    Hs = 0.5 * (Hs + Hs.T)
    lam, W = np.linalg.eigh(Hs)
    return lam, Q @ W


def chefsi_cycle(apply_H, X, m, a, b, a0):
    """One filter + orthonormalise + Rayleigh-Ritz cycle."""
    return rayleigh_ritz(apply_H, cheb_filter(apply_H, X, m, a, b, a0))

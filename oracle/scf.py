"""Self-consistent closure of the slab problem: density, occupations, density mixing.

Test infrastructure only (like every module of this package): tests, the smoke check and
the benchmark's CPU baseline may import it; the library never does.

* Density (Section 2.1, the equation below Eq. Tsexc): rho(x) = 2 sum_n f_n |psi_n(x)|^2.
  With the discrete problem written as Ht = M^-1/2 H M^-1/2 on Euclidean-orthonormal
  columns xt_n (Section 2.3's H u = eps M u, u_n = M^-1/2 xt_n), the nodal value of
  psi_n at psi node I is xt_{I,n} / sqrt(M_II), so rho_I = 2 sum_n f_n xt_{I,n}^2 / M_II,
  zero on the homogeneous-Dirichlet z planes, and sum_I M_II rho_I = 2 sum_n f_n exactly.
* Occupations (reading, the paper defers to its earlier work): Fermi-Dirac at smearing
  temperature kT, f_n = 1 / (1 + exp((eps_n - mu)/kT)), with mu fixed by
  2 sum_n f_n = N_e, found by bisection.
* Mixing (reading: the paper defers its mixing scheme to earlier work): Anderson / Pulay
  mixing of the density (D. G. Anderson, J. ACM 12 (1965); P. Pulay, Chem. Phys. Lett. 73
  (1980)) with the residual R = rho_out - rho_in measured in the lumped-mass inner product
  <u, v> = sum_I M_II u_I v_I: with the differences dR_i, drho_i of the last m iterations,
  gamma minimises |R - sum_i gamma_i dR_i| and
  rho_next = rho_in + alpha R - sum_i gamma_i (drho_i + alpha dR_i); with m = 0 this is
  linear mixing rho_next = rho_in + alpha R.
* One self-consistent iteration: Poisson solve with the bias, V_eff, Chebyshev-filtered
  subspace iteration, occupations, rho_out, mixing.  Hartree level by default; optionally
  with local-density exchange (reading: the paper's exchange-correlation functional enters
  V_eff through v_xc = dE_xc/drho, Section 2.1; its GGA needs a functional library, so the
  optional term here is the closed-form exchange of the homogeneous electron gas, Dirac
  1930, spin unpolarised, no correlation):
      e_x(rho) = -(3/4) (3/pi)^(1/3) rho^(4/3)   (energy per volume),
      v_x(rho) = d e_x / d rho = -(3/pi)^(1/3) rho^(1/3),
  negative densities (possible after mixing) taken as zero; E_x = sum_I M_II e_x(rho_I)
  in the lumped quadrature, v_x added to V_eff at the psi nodes.
"""
import math

import numpy as np


def density(X, occ, M_psi):
    """rho at psi nodes: sum_n occ_n X[I, n]^2 / M_II (occ_n = 2 f_n)."""
    X = np.asarray(X, dtype=np.float64)
    return (X * X) @ np.asarray(occ, dtype=np.float64) / M_psi


def density_phi(X, occ, M, psi_ids):
    """The density on every phi node (zero on the planes that carry no psi node)."""
    rho = np.zeros(M.shape[0])
    rho[psi_ids] = density(X, occ, M[psi_ids])
    return rho


def lda_exchange(rho):
    """(e_x, v_x) of the Dirac exchange at each value of rho (see the module text)."""
    r = np.maximum(np.asarray(rho, dtype=np.float64), 0.0)
    c = (3.0 / math.pi) ** (1.0 / 3.0)
    cbrt = np.cbrt(r)
    return -0.75 * c * r * cbrt, -c * cbrt


def fermi(eps, mu, kT):
    x = (np.asarray(eps, dtype=np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))   # = 1 / (1 + exp(x)), without overflow


def occupations(eps, n_electrons, kT, iters=200):
    """(occ = 2 f, mu) with 2 sum f = n_electrons, mu by bisection."""
    eps = np.asarray(eps, dtype=np.float64)
    if not 0.0 <= n_electrons <= 2.0 * len(eps):
        raise ValueError("electron count outside [0, 2 nvec]")
    lo = eps.min() - 50.0 * kT - 1.0
    hi = eps.max() + 50.0 * kT + 1.0
    for _ in range(iters):
        mu = 0.5 * (lo + hi)
        if 2.0 * fermi(eps, mu, kT).sum() > n_electrons:
            hi = mu
        else:
            lo = mu
    mu = 0.5 * (lo + hi)
    return 2.0 * fermi(eps, mu, kT), mu


class AndersonMixer:
    """Anderson / Pulay mixing with a weighted inner product (see the module text)."""

    def __init__(self, weights, alpha=0.3, history=4):
        self.w = np.asarray(weights, dtype=np.float64)
        self.alpha = alpha
        self.m = history
        self.prev_rho = None
        self.prev_R = None
        self.drho = []
        self.dR = []

    def dot(self, u, v):
        return float(np.sum(self.w * u * v))

    def step(self, rho_in, rho_out):
        """Next input density and the weighted residual norm |rho_out - rho_in|."""
        rho_in = np.asarray(rho_in, dtype=np.float64)
        R = np.asarray(rho_out, dtype=np.float64) - rho_in
        if self.prev_R is not None and self.m > 0:
            self.dR.append(R - self.prev_R)
            self.drho.append(rho_in - self.prev_rho)
            if len(self.dR) > self.m:
                self.dR.pop(0)
                self.drho.pop(0)
        self.prev_R = R.copy()
        self.prev_rho = rho_in.copy()
        nxt = rho_in + self.alpha * R
        k = len(self.dR)
        if k:
            A = np.array([[self.dot(self.dR[i], self.dR[j]) for j in range(k)] for i in range(k)])
            rhs = np.array([self.dot(self.dR[i], R) for i in range(k)])
            gamma = np.linalg.lstsq(A, rhs, rcond=None)[0]
            for i in range(k):
                nxt -= gamma[i] * (self.drho[i] + self.alpha * self.dR[i])
        return nxt, math.sqrt(self.dot(R, R))


def scf_run(slab, X0, iters, kT=0.01, alpha=0.3, history=4, degree=None, first_cycles=4,
            lanczos_steps=20, v0=None, xc=None):
    """Hartree-level self-consistent iterations on a small slab, every step in FP64.

    Per iteration k: phi from the Poisson problem with the load 4 pi M (rho_in + b) and the
    slab's bias; V_eff = phi + V_loc - V_sm + V_app at psi nodes; Lanczos bounds (lo, hi)
    of Ht; filter + Rayleigh-Ritz cycles (first_cycles at k = 0, one afterwards) with
    a0 = lo, b = hi and the cut a = a0 + 0.1 (b - a0) for the very first cycle, else the
    largest Ritz value of the previous cycle when it lies in (lo, hi) (else the first-cycle
    rule again); occupations and mu; rho_out; Anderson mixing.
    The first rho_in is the atoms' model density.  xc = "lda_x" adds v_x(rho_in) to V_eff.
    Returns a dict with the final rho_in, mu, Ritz values, block and the residual norms of
    every iteration (and E_x of the last rho_in with xc)."""
    from oracle import assembly, chefsi, poisson, potentials
    from oracle.mesh import Mesh as OMesh
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    X = om.phi_coords()
    ids = om.psi_to_phi()
    rho_model, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
    n_e = float(np.sum(slab.Z))
    bias = slab.bias
    if bias.kind == "cef":
        vapp = potentials.v_app(X[:, 2], bias.field, slab.L[2])
    else:
        mask, vals, _, _ = potentials.cpd_constraints(X, vl, bias, slab.L)
        vapp = np.zeros(om.n_phi)
    degree = degree or slab.degree
    mixer = AndersonMixer(M, alpha=alpha, history=history)
    rho_in = rho_model.copy()
    Xb = np.asarray(X0, dtype=np.float64)
    v0 = np.ones(om.n_psi) if v0 is None else v0
    eig, mu, cut, res = None, None, None, []
    for k in range(iters):
        f = 4.0 * math.pi * M * (rho_in + b)
        if bias.kind == "cef":
            phi = poisson.solve_cef_direct(K, f, M)
        else:
            phi = poisson.solve_cpd_direct(K, f, mask, vals)
        V = (phi + vl + vapp)[ids]
        if xc == "lda_x":
            V = V + lda_exchange(rho_in)[1][ids]
        H = assembly.hamiltonian(om, V, K, M)
        lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, v0, lanczos_steps)
        for _ in range(first_cycles if k == 0 else 1):
            # the previous largest Ritz value when it lies inside the new interval, else
            # the first-cycle rule (the potential can move the spectrum between iterations)
            a = cut if cut is not None and lo < cut < hi else lo + 0.1 * (hi - lo)
            eig, Xb = chefsi.chefsi_cycle(lambda Z: H @ Z, Xb, degree, a, hi, lo)
            cut = eig[-1]
        occ, mu = occupations(eig, n_e, kT)
        rho_out = density_phi(Xb, occ, M, ids)
        rho_in, r = mixer.step(rho_in, rho_out)
        res.append(r)
    out = {"rho": rho_in, "mu": mu, "eig": eig, "X": Xb, "res": res, "M": M}
    if xc == "lda_x":
        out["ex"] = float(M @ lda_exchange(rho_in)[0])
    return out

"""Atom-centred fields, sawtooth field and CPD constraint values.

* V_loc^a(r) = -Z erf(r / r_loc) / r, the synthetic local pseudopotential that stands in
  for ONCV files (Section 2.4 uses ONCV; r_loc = 1 bohr).
* Smeared nuclear charge b_sm^a = -Z g_sigma and its potential V_sm^a, which solve
  -1/(4 pi) Lap V_sm^a = b_sm^a (Eq. Governing equations).  Reading of "sigma": the
  standard deviation of the Gaussian g_sigma(r) = (2 pi sigma^2)^-3/2 exp(-r^2 / 2 sigma^2),
  so V_sm^a = -Z erf(r / (sqrt(2) sigma)) / r.  [parity unpinned: width convention]
* phi_tilde = phi + V_loc - V_sm (Eq. Veff and Hloc); the sums over atoms include the
  periodic images in x and y (Eq. Governing equations1).  Every atom-centred function is
  cut at r_cut = 10 bohr (its tail there is below 1e-20).
* Electron density for the Poisson right-hand side (reading; the paper's rho comes from
  the Kohn-Sham orbitals): rho = sum_a Z_a g_{sigma_rho}, sigma_rho = 1 bohr.
* Discrete renormalisation (reading): each b^a is rescaled so that sum_I M_II b^a(x_I) is
  exactly -Z_a, and rho so that sum_I M_II rho(x_I) = N_e = sum Z_a.
* V_app (Section 2.2.1, Fig. CEF; Section 3.1 puts the extrema 0.1 fractional units from
  the z boundaries): slope -E on [0.1 Lz, 0.9 Lz], V_app = -E (z - Lz/2) there, linear
  return ramps to 0 at z = 0 and z = Lz.  [parity unpinned: return-ramp shape]
* CPD (Eq. governing_equations APD): phi = -(V_loc - V_sm) on Omega_0 and
  dV - (V_loc - V_sm) on Omega_1.  Reading: Omega_0 = nodes with z <= Z_A, Omega_1 = nodes
  with z >= Z_B; for L-CPD Omega_1 is further restricted to the in-plane patch and nodes
  outside it are unconstrained.  [parity unpinned: L-CPD off-patch boundary]
"""
import math

import numpy as np
from scipy.special import erf

RCUT = 10.0
SIGMA_B = 0.5
SIGMA_RHO = 1.0
R_LOC = 1.0


def vloc_minus_vsm_radial(r, Z, r_loc=R_LOC, sigma_b=SIGMA_B):
    """(V_loc - V_sm)(r) = Z [erf(r / (sqrt2 sigma_b)) - erf(r / r_loc)] / r, r >= 0."""
    r = np.asarray(r, dtype=np.float64)
    a = 1.0 / (math.sqrt(2.0) * sigma_b)
    b = 1.0 / r_loc
    small = r < 1e-8
    rs = np.where(small, 1.0, r)
    val = (erf(a * rs) - erf(b * rs)) / rs
    lim = 2.0 / math.sqrt(math.pi) * (a - b)
    return Z * np.where(small, lim, val)


def vsm_radial(r, Z, sigma_b=SIGMA_B):
    """V_sm(r) = -Z erf(r / (sqrt2 sigma_b)) / r."""
    r = np.asarray(r, dtype=np.float64)
    a = 1.0 / (math.sqrt(2.0) * sigma_b)
    small = r < 1e-8
    rs = np.where(small, 1.0, r)
    return -Z * np.where(small, 2.0 / math.sqrt(math.pi) * a, erf(a * rs) / rs)


def gaussian_radial(r, sigma):
    """Normalised 3D Gaussian g_sigma(r)."""
    r = np.asarray(r, dtype=np.float64)
    return (2.0 * math.pi * sigma * sigma) ** -1.5 * np.exp(-r * r / (2.0 * sigma * sigma))


def image_shifts(L, rcut=RCUT):
    nx = int(math.ceil(rcut / L[0])) + 1
    ny = int(math.ceil(rcut / L[1])) + 1
    return [(i * L[0], j * L[1]) for j in range(-ny, ny + 1) for i in range(-nx, nx + 1)]


def atom_sum(coords, R, values_fn, L, rcut=RCUT, per_atom=False):
    """sum over atoms a and x/y images of values_fn(a, r) for r <= rcut, at ``coords``."""
    coords = np.asarray(coords, dtype=np.float64)
    shifts = image_shifts(L, rcut)
    out = np.zeros((len(R), len(coords))) if per_atom else np.zeros(len(coords))
    for a in range(len(R)):
        acc = np.zeros(len(coords))
        for sx, sy in shifts:
            d = coords - np.array([R[a, 0] + sx, R[a, 1] + sy, R[a, 2]])
            r = np.sqrt(np.sum(d * d, axis=1))
            m = r <= rcut
            if np.any(m):
                acc[m] += values_fn(a, r[m])
        if per_atom:
            out[a] = acc
        else:
            out += acc
    return out


def vloc_minus_vsm(coords, R, Z, L):
    """sum_a (V_loc^a - V_sm^a) with periodic x/y images."""
    return atom_sum(coords, R, lambda a, r: vloc_minus_vsm_radial(r, Z[a]), L)


def densities(coords, M, R, Z, L, sigma_b=SIGMA_B, sigma_rho=SIGMA_RHO):
    """(rho, b) at the nodes after discrete renormalisation with lumped weights M."""
    g = atom_sum(coords, R, lambda a, r: gaussian_radial(r, sigma_b), L, per_atom=True)
    b = np.zeros(len(coords))
    for a in range(len(R)):
        s = float(M @ g[a])
        b += (-Z[a] / s) * g[a]
    rho = atom_sum(coords, R, lambda a, r: Z[a] * gaussian_radial(r, sigma_rho), L)
    rho *= float(np.sum(Z)) / float(M @ rho)
    return rho, b


def v_app(z, field, Lz):
    """Sawtooth auxiliary potential of the CEF setup."""
    z = np.asarray(z, dtype=np.float64)
    z1, z2 = 0.1 * Lz, 0.9 * Lz
    top = -field * (z1 - 0.5 * Lz)      # value at z1 (= +0.4 E Lz)
    bot = -field * (z2 - 0.5 * Lz)      # value at z2 (= -0.4 E Lz)
    mid = -field * (z - 0.5 * Lz)
    lo = top * z / z1
    hi = bot * (Lz - z) / (Lz - z2)
    return np.where(z < z1, lo, np.where(z > z2, hi, mid))


def dv_app_dfield(z, Lz):
    """Derivative of v_app with respect to the field (v_app is linear in E)."""
    return v_app(z, 1.0, Lz)


def cpd_constraints(coords, vlms, bias, L, tol=1e-12):
    """(mask, values) of the constrained phi nodes for CPD / L-CPD."""
    z = coords[:, 2]
    om0 = z <= bias.zA + tol
    om1 = z >= bias.zB - tol
    if bias.patch is not None:
        (xlo, ylo), (xhi, yhi) = bias.patch
        x, y = coords[:, 0], coords[:, 1]
        om1 &= (x >= xlo - tol) & (x <= xhi + tol) & (y >= ylo - tol) & (y <= yhi + tol)
    mask = om0 | om1
    vals = np.zeros(len(coords))
    vals[om0] = -vlms[om0]
    vals[om1] = bias.dV - vlms[om1]
    return mask, vals, om0, om1

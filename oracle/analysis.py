"""Analysis outputs of a slab solution (Section 3): dipole moment, polarisability and the
planar averages of the density and of the bare potential.

Test infrastructure only (like every module of this package).

* Dipole (Section 3.1): mu_z = int (b + rho) (z - Lz/2) dx about the domain centre, with
  the lumped quadrature: mu_z = sum_I M_II (b_I + rho_I)(z_I - Lz/2).
* Polarisability (Section 3.1): alpha_z = Delta mu / Delta E between two fields.
* Planar quantities (Section 3.3): rho0(z) = int_{S_z} rho dx dy (a planar integral) and
  V0_bare(z) = (1/A_z) int_{S_z} V_bare dx dy, with V_bare = phi + (V_loc - V_sm) + V_app
  (the paper's phi_tilde + V_app).  On the phi plane gz the in-plane GLL quadrature weights
  are the lumped masses divided by the plane's z factor (h_z / 2) mz(gz), so
  rho0(z_gz) = sum_{I in gz} M_II rho_I / ((h_z / 2) mz(gz)) and
  V0_bare(z_gz) = sum_{I in gz} M_II V_I / sum_{I in gz} M_II.
"""
import numpy as np


def dipole_z(M, rho, b, z, Lz):
    return float(np.sum(M * (rho + b) * (z - 0.5 * Lz)))


def polarisability(mu_a, mu_b, field_a, field_b):
    return (mu_b - mu_a) / (field_b - field_a)


def plane_z_weight(mesh, gz):
    """(h_z / 2) mz(gz): the z factor of the lumped mass of the phi plane gz."""
    p = mesh.p
    w = mesh.w
    l = gz % p
    if l != 0:
        mz = w[l]
    elif gz == 0 or gz == mesh.ncell[2] * p:
        mz = w[0]
    else:
        mz = 2.0 * w[0]
    return 0.5 * mesh.h[2] * mz


def planar_integral(mesh, M, f):
    """rho0 per phi plane."""
    plane = mesh.NX * mesh.NY
    F = (M * f).reshape(-1, plane).sum(axis=1)
    return np.array([F[gz] / plane_z_weight(mesh, gz) for gz in range(F.shape[0])])


def planar_average(mesh, M, f):
    """V0 per phi plane."""
    plane = mesh.NX * mesh.NY
    return (M * f).reshape(-1, plane).sum(axis=1) / M.reshape(-1, plane).sum(axis=1)

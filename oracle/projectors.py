"""Nonlocal pseudopotential term with synthetic projectors (Eq. V_nloc).

Test infrastructure only (like every module of this package).

Eq. V_nloc: (V_nloc psi)(x) = sum_a sum_beta p^a_beta(x - R_a) D^a_beta
int p^a_beta(y - R_a) psi(y) dy.  The paper's ONCV projectors are not available; the
synthetic stand-in (reading) is one s and three p channels per atom,
  p_s(d) = g(d),  p_x(d) = (d_x / s) g(d),  p_y(d) = (d_y / s) g(d),  p_z(d) = (d_z / s) g(d),
  g(d) = exp(-|d|^2 / (2 s^2)),
with a per-atom width s_a and coefficients D^a (4 per atom), summed over the periodic x/y
images and cut at |d| <= rc.

FE form (Section 2.3, lumped quadrature as for the rest of the operator):
<N_I, p> ~ M_II p(x_I), so H_nloc = M P D P^T M with P[I, (a, beta)] = p^a_beta(x_I) on
psi nodes, and in the scaled problem Ht = M^-1/2 H M^-1/2 the term is
  Ht_nloc = M^1/2 P D P^T M^1/2.
"""
import numpy as np

from oracle.potentials import image_shifts

CHANNELS = 4   # s, p_x, p_y, p_z


def projector_values(coords, R, sigma, L, rc):
    """P [n_nodes][natoms * 4] at the given node coordinates."""
    coords = np.asarray(coords, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    P = np.zeros((len(coords), CHANNELS * len(R)))
    for a in range(len(R)):
        s = float(sigma[a])
        for sx, sy in image_shifts(L, rc):
            d = coords - np.array([R[a, 0] + sx, R[a, 1] + sy, R[a, 2]])
            r2 = np.sum(d * d, axis=1)
            m = r2 <= rc * rc
            if not np.any(m):
                continue
            g = np.exp(-r2[m] / (2.0 * s * s))
            P[m, CHANNELS * a + 0] += g
            P[m, CHANNELS * a + 1] += d[m, 0] / s * g
            P[m, CHANNELS * a + 2] += d[m, 1] / s * g
            P[m, CHANNELS * a + 3] += d[m, 2] / s * g
    return P


def nonlocal_scaled(mesh, M, R, sigma, D, rc):
    """Ht_nloc = M^1/2 P D P^T M^1/2 on psi nodes (dense; small meshes only)."""
    ids = mesh.psi_to_phi()
    X = mesh.phi_coords()[ids]
    P = projector_values(X, R, sigma, mesh.L, rc)
    S = np.sqrt(M[ids])
    SP = S[:, None] * P
    return SP @ (np.asarray(D, dtype=np.float64).reshape(-1)[:, None] * SP.T)


def apply_nonlocal(mesh, M, R, sigma, D, rc, X):
    """Ht_nloc X without forming the n x n matrix."""
    ids = mesh.psi_to_phi()
    C = mesh.phi_coords()[ids]
    P = projector_values(C, R, sigma, mesh.L, rc)
    S = np.sqrt(M[ids])
    SP = S[:, None] * P
    Dv = np.asarray(D, dtype=np.float64).reshape(-1)
    return SP @ (Dv[:, None] * (SP.T @ np.asarray(X, dtype=np.float64)))

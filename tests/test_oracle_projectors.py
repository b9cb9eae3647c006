"""Pins of the nonlocal term with synthetic projectors (oracle/projectors.py): the lumped
quadrature of the projectors against their closed forms (s-channel integral, p-channel
odd symmetry), the matrix elements of the discrete H_nloc between Gaussians against the
closed-form Gaussian overlaps (which fixes every factor of M and of D), and the
symmetry / rank / sign of Ht_nloc."""
import numpy as np
import pytest

from oracle import assembly, projectors
from oracle.mesh import Mesh as OMesh


@pytest.fixture(scope="module")
def fine():
    om = OMesh((8.0, 8.0, 8.0), (8, 8, 8), 5, (False, False))
    M = assembly.lumped_mass(om)
    ids = om.psi_to_phi()
    X = om.phi_coords()[ids]
    R = np.array([[4.0, 4.0, 4.0]])
    sig = np.array([0.8])
    P = projectors.projector_values(X, R, sig, om.L, 3.9)
    return om, M[ids], X, R, sig, P


def test_projector_quadrature(fine):
    om, Mp, X, R, sig, P = fine
    assert abs(Mp @ P[:, 0] - (2 * np.pi * sig[0] ** 2) ** 1.5) <= 1e-4 * (2 * np.pi * 0.64) ** 1.5
    for ch in (1, 2, 3):      # odd channels about an atom on a symmetric node set
        assert abs(Mp @ P[:, ch]) <= 1e-13


def test_matrix_elements_between_gaussians(fine):
    """<phi, H_nloc phi> = D (int p phi)^2 with H_nloc = M P D P^T M; for Gaussians centred
    on the atom the overlaps are closed forms."""
    om, Mp, X, R, sig, P = fine
    t = 0.9
    d = X - R[0]
    g = np.exp(-np.sum(d * d, axis=1) / (2 * t * t))
    s2 = sig[0] ** 2
    c = P.T @ (Mp * g)
    ref_s = (2 * np.pi * s2 * t * t / (s2 + t * t)) ** 1.5
    assert abs(c[0] - ref_s) <= 1e-5 * ref_s
    assert np.max(np.abs(c[1:])) <= 1e-13
    cx = P.T @ (Mp * d[:, 0] * g)
    tau2 = 1.0 / (1.0 / s2 + 1.0 / t ** 2)
    ref_x = tau2 / sig[0] * (2 * np.pi * tau2) ** 1.5
    assert abs(cx[1] - ref_x) <= 1e-5 * ref_x
    assert abs(cx[0]) <= 1e-13 and abs(cx[2]) <= 1e-13 and abs(cx[3]) <= 1e-13


def test_scaled_operator_symmetric_low_rank_and_signed():
    om = OMesh((4.0, 4.0, 6.0), (2, 2, 3), 3)
    M = assembly.lumped_mass(om)
    R = np.array([[1.0, 1.2, 3.0], [3.1, 2.5, 2.2]])
    sig = np.array([0.7, 0.9])
    D = np.array([[0.8, 0.3, 0.3, 0.3], [1.1, 0.0, 0.5, 0.2]])
    Hn = projectors.nonlocal_scaled(om, M, R, sig, D, 2.5)
    assert np.max(np.abs(Hn - Hn.T)) <= 1e-14 * np.max(np.abs(Hn))
    ev = np.linalg.eigvalsh(Hn)
    assert ev[0] >= -1e-12 * ev[-1]
    assert np.sum(ev > 1e-10 * ev[-1]) <= 8
    X = np.random.default_rng(0).standard_normal((om.n_psi, 5))
    np.testing.assert_allclose(projectors.apply_nonlocal(om, M, R, sig, D, 2.5, X), Hn @ X,
                               rtol=1e-12, atol=1e-12 * np.max(np.abs(Hn @ X)))

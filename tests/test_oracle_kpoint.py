"""Pins of the oracle's Bloch k-point Hamiltonian (oracle/kpoint.py) against what the
mathematics fixes: Hermiticity and the antisymmetry of the assembled gradient matrices
(periodic x, y), the Gamma-point reduction, time reversal, the free-electron ground state
1/2 |k|^2 (exact for the constant function with Neumann z faces), and free-electron bands
1/2 |k + g|^2 of plane waves along x (within the discretisation error)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assembly, kpoint
from oracle.mesh import Mesh as OMesh


def _mesh(neumann=False, p=3, L=(4.0, 5.0, 6.0), ncell=(3, 3, 3)):
    faces = (False, False) if neumann else (True, True)
    return OMesh(L, ncell, p, faces)


def test_gradient_matrices_are_antisymmetric_with_periodic_x_y():
    om = _mesh()
    for axis in (0, 1):
        G = kpoint.assemble_gradient(om, axis).toarray()
        assert np.max(np.abs(G + G.T)) <= 1e-13 * np.max(np.abs(G))
        # G annihilates constants (the derivative of 1) and has no row-sum
        assert np.max(np.abs(G @ np.ones(om.n_phi))) <= 1e-13


def test_hamiltonian_is_hermitian_and_reduces_to_gamma():
    om = _mesh()
    rng = np.random.default_rng(1)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    Hk = kpoint.hamiltonian_k(om, V, (0.37, -0.21)).toarray()
    assert np.max(np.abs(Hk - Hk.conj().T)) <= 1e-13 * np.max(np.abs(Hk))
    H0 = kpoint.hamiltonian_k(om, V, (0.0, 0.0)).toarray()
    Hr = assembly.hamiltonian(om, V).toarray()
    assert np.max(np.abs(H0 - Hr)) == 0.0


def test_time_reversal():
    om = _mesh()
    rng = np.random.default_rng(2)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    k = (0.41, 0.17)
    Hp = kpoint.hamiltonian_k(om, V, k).toarray()
    Hm = kpoint.hamiltonian_k(om, V, (-k[0], -k[1])).toarray()
    assert np.max(np.abs(Hm - Hp.conj())) <= 1e-15 * np.max(np.abs(Hp))
    np.testing.assert_allclose(sla.eigvalsh(Hp), sla.eigvalsh(Hm), atol=1e-11)


@pytest.mark.parametrize("k", [(0.0, 0.0), (0.3, 0.0), (0.2, -0.35)])
def test_free_electron_ground_state_is_half_k_squared(k):
    """V = 0, Neumann z faces: the constant is an exact eigenfunction (K 1 = 0, G 1 = 0)
    with eigenvalue 1/2 |k|^2, the lowest for |k| within the first zone."""
    om = _mesh(neumann=True)
    Hk = kpoint.hamiltonian_k(om, np.zeros(om.n_psi), k).toarray()
    ev = sla.eigvalsh(Hk)
    assert abs(ev[0] - 0.5 * (k[0] ** 2 + k[1] ** 2)) <= 1e-12


def test_free_electron_bands_along_x():
    """V = 0, Neumann z: the plane waves e^{i g x} (g = 2 pi m / Lx) are eigenfunctions of
    the continuum operator with 1/2 (k + g)^2; on a p = 5 mesh the discrete eigenvalues
    match to discretisation accuracy."""
    Lx = 4.0
    om = OMesh((Lx, 3.0, 3.0), (4, 2, 2), 5, (False, False))
    kx = 0.3
    Hk = kpoint.hamiltonian_k(om, np.zeros(om.n_psi), (kx, 0.0)).toarray()
    ev = np.sort(sla.eigvalsh(Hk))
    for m in (-1, 1):
        target = 0.5 * (kx + 2 * np.pi * m / Lx) ** 2
        assert np.min(np.abs(ev - target)) <= 1e-6 * target


def test_band_state_has_the_plane_wave_phase():
    """Fixes the sign of the -i k.grad term: the eigenvector with eigenvalue 1/2 (k + g)^2,
    g = +2 pi / Lx, is u = e^{+i g x} at the nodes (u = M^-1/2 v)."""
    Lx = 4.0
    om = OMesh((Lx, 3.0, 3.0), (4, 2, 2), 5, (False, False))
    kx = 0.3
    M = assembly.lumped_mass(om)
    ids = om.psi_to_phi()
    Hk = kpoint.hamiltonian_k(om, np.zeros(om.n_psi), (kx, 0.0), M=M).toarray()
    ev, vec = sla.eigh(Hk)
    g = 2 * np.pi / Lx
    j = int(np.argmin(np.abs(ev - 0.5 * (kx + g) ** 2)))
    u = vec[:, j] / np.sqrt(M[ids])
    x = om.phi_coords()[ids][:, 0]
    w = u * np.exp(-1j * g * x)          # constant for the e^{+i g x} state
    assert np.max(np.abs(w - w.mean())) <= 1e-3 * np.max(np.abs(w))


def test_complex_filter_is_the_polynomial_of_the_spectrum():
    """The oracle's filter on a complex block equals V p(Lambda) V^H X from the dense
    eigendecomposition of Ht_k (p the scaled Chebyshev polynomial evaluated by its own
    three-term recurrence on the eigenvalues)."""
    from oracle import chefsi
    om = _mesh(p=2, ncell=(2, 2, 2))
    rng = np.random.default_rng(3)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    Hk = kpoint.hamiltonian_k(om, V, (0.3, -0.2)).toarray()
    lam, Q = sla.eigh(Hk)
    X = rng.standard_normal((om.n_psi, 3)) + 1j * rng.standard_normal((om.n_psi, 3))
    a0, b = lam[0] - 0.1, lam[-1] + 0.1
    a = a0 + 0.3 * (b - a0)
    deg = 6
    got = chefsi.cheb_filter(lambda Z: Hk @ Z, X, deg, a, b, a0)
    # the same recurrence on the scalars lambda
    e, c = (b - a) / 2, (b + a) / 2
    sig = e / (a0 - c)
    tau = 2 / sig
    y0, y1 = np.ones_like(lam), (sig / e) * (lam - c)
    for _ in range(2, deg + 1):
        sn = 1 / (tau - sig)
        y0, y1 = y1, (2 * sn / e) * (lam - c) * y1 - sig * sn * y0
        sig = sn
    ref = Q @ (y1[:, None] * (Q.conj().T @ X))
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("faces,ncell", [((True, True), (2, 3, 2)), ((False, True), (1, 2, 2)),
                                         ((True, False), (3, 1, 1))])
def test_rows_match_the_assembled_operator(faces, ncell):
    """The row-by-row form (used at sizes where the matrix does not fit) against the
    assembled Ht_k, including single-cell periodic rows and both face kinds."""
    om = OMesh((3.0, 3.5, 4.0), ncell, 2, faces)
    rng = np.random.default_rng(4)
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    k = (0.37, -0.21)
    H = kpoint.hamiltonian_k(om, V, k)
    X = rng.standard_normal((om.n_psi, 3)) + 1j * rng.standard_normal((om.n_psi, 3))
    got = kpoint.apply_Hk_rows(om, V, k, X, np.arange(om.n_psi))
    ref = H @ X
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))

"""Pins of the self-consistent closure (oracle/scf.py): the density integrates to the
electron count exactly and equals the textbook |psi|^2 of the generalised problem; the
Fermi-Dirac occupations fill 2 sum f = N_e and reduce to aufbau filling as kT -> 0;
Anderson mixing without history is linear mixing and, on a linear fixed-point map,
reaches the fixed point far faster than linear mixing."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assembly, scf
from oracle.mesh import Mesh as OMesh


def test_density_integrates_to_electron_count_and_matches_generalised_eigenvectors():
    om = OMesh((4.0, 4.0, 6.0), (2, 2, 3), 3)
    rng = np.random.default_rng(0)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    ids = om.psi_to_phi()
    H = assembly.hamiltonian(om, V, K, M).toarray()
    ev, Xt = np.linalg.eigh(H)
    nocc = 6
    occ = np.full(nocc, 2.0)
    rho = scf.density(Xt[:, :nocc], occ, M[ids])
    assert abs(np.sum(M[ids] * rho) - 2.0 * nocc) <= 1e-11
    # the same density from the generalised problem H u = eps M u with u^T M u = 1
    Hg = 0.5 * K[ids][:, ids].toarray() + np.diag(M[ids] * V)
    evg, U = sla.eigh(Hg, np.diag(M[ids]))
    assert np.max(np.abs(evg[:nocc] - ev[:nocc])) <= 1e-10 * np.max(np.abs(ev))
    rho_g = 2.0 * np.sum(U[:, :nocc] ** 2, axis=1)
    assert np.max(np.abs(rho - rho_g)) <= 1e-10 * np.max(rho)
    full = scf.density_phi(Xt[:, :nocc], occ, M, ids)
    assert full.shape == (om.n_phi,) and np.all(np.delete(full, ids) == 0.0)


@pytest.mark.parametrize("kT", [1e-3, 0.01, 0.1])
def test_occupations_fill_the_electron_count(kT):
    eps = np.sort(np.random.default_rng(1).uniform(-2.0, 1.0, 40))
    occ, mu = scf.occupations(eps, 23.0, kT)
    assert abs(occ.sum() - 23.0) <= 1e-10
    assert np.all(np.diff(occ) <= 1e-15) and np.all((occ >= 0) & (occ <= 2))
    # f(mu) = 1/2 exactly on the continuous Fermi function
    assert abs(scf.fermi(mu, mu, kT) - 0.5) <= 1e-15


def test_occupations_zero_temperature_limit_is_aufbau():
    eps = np.linspace(-1.0, 1.0, 20)         # spacing 0.105, kT far below it
    occ, mu = scf.occupations(eps, 14.0, 1e-4)
    np.testing.assert_allclose(occ, np.r_[np.full(7, 2.0), np.zeros(13)], atol=1e-12)
    assert eps[6] < mu < eps[7]


def test_anderson_without_history_is_linear_mixing():
    rng = np.random.default_rng(2)
    w = rng.uniform(0.5, 1.5, 50)
    mix = scf.AndersonMixer(w, alpha=0.4, history=0)
    a, b = rng.standard_normal(50), rng.standard_normal(50)
    nxt, r = mix.step(a, b)
    np.testing.assert_allclose(nxt, a + 0.4 * (b - a), rtol=0, atol=1e-15)
    assert abs(r - np.sqrt(np.sum(w * (b - a) ** 2))) <= 1e-12


def test_anderson_solves_a_linear_fixed_point_problem():
    """G(x) = A x + c with spectral radius 0.9: after 100 steps linear mixing is still at
    ~4e-3 relative error, Anderson with a history of 8 at rounding level."""
    rng = np.random.default_rng(3)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(-0.9, 0.9, n)) @ Q.T
    c = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, c)
    w = np.ones(n)

    def run(history, steps):
        mix = scf.AndersonMixer(w, alpha=0.5, history=history)
        x = np.zeros(n)
        for _ in range(steps):
            x, r = mix.step(x, A @ x + c)
        return np.linalg.norm(x - xstar)

    assert run(8, 100) <= 1e-12 * np.linalg.norm(xstar)
    assert run(0, 100) >= 1e-3 * np.linalg.norm(xstar)


def test_lda_exchange_matches_the_homogeneous_gas():
    """Exchange energy per electron of the homogeneous gas at Wigner-Seitz radius r_s:
    -(3/4) (9 / (4 pi^2))^(1/3) / r_s = -0.458165... / r_s Ha (textbook constant, written
    here in r_s rather than rho)."""
    for rs in (0.5, 1.0, 2.0, 5.0):
        rho = 3.0 / (4.0 * np.pi * rs ** 3)
        ex, _ = scf.lda_exchange(np.array([rho]))
        assert abs(ex[0] / rho - (-0.4581652932831429 / rs)) <= 1e-14 / rs


def test_lda_exchange_potential_is_the_derivative_and_scales():
    rho = np.array([1e-4, 0.01, 0.3, 2.0, 7.5])
    ex, vx = scf.lda_exchange(rho)
    h = 1e-6 * rho
    fd = (scf.lda_exchange(rho + h)[0] - scf.lda_exchange(rho - h)[0]) / (2 * h)
    np.testing.assert_allclose(vx, fd, rtol=1e-8)
    lam = 3.7
    np.testing.assert_allclose(scf.lda_exchange(lam * rho)[0], lam ** (4.0 / 3.0) * ex, rtol=1e-14)
    np.testing.assert_allclose(scf.lda_exchange(lam * rho)[1], lam ** (1.0 / 3.0) * vx, rtol=1e-14)
    ex0, vx0 = scf.lda_exchange(np.array([0.0, -1e-9]))
    assert np.all(ex0 == 0.0) and np.all(vx0 == 0.0)


def test_lda_exchange_energy_of_a_gaussian_density():
    """E_x of a normalised Gaussian density of width s: the integral of rho^(4/3) is
    (2 pi s^2)^(-1/2) (3/4)^(3/2) for one electron, so E_x = -(3/4)(3/pi)^(1/3) times that;
    the lumped quadrature on a fine p = 4 mesh reproduces it."""
    from oracle.mesh import Mesh as OMesh
    from oracle import assembly
    s_w = 0.8
    L = (8.0, 8.0, 8.0)
    om = OMesh(L, (8, 8, 8), 4, (False, False))
    X = om.phi_coords()
    M = assembly.lumped_mass(om)
    r2 = np.sum((X - 4.0) ** 2, axis=1)
    rho = np.exp(-r2 / (2 * s_w ** 2)) / (2 * np.pi * s_w ** 2) ** 1.5
    ex = float(M @ scf.lda_exchange(rho)[0])
    exact = -0.75 * (3 / np.pi) ** (1 / 3) * (2 * np.pi * s_w ** 2) ** -0.5 * (3 / 4) ** 1.5
    assert abs(ex - exact) <= 1e-6 * abs(exact)

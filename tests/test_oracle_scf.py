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

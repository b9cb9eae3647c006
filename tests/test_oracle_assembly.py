"""Pins of the oracle's FE matrices and Hamiltonian (Section 2.3, Eq. Veff and Hloc)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assembly import (apply_H_rows, assemble_stiffness, hamiltonian, lumped_mass,
                             reference_cell_stiffness)
from oracle.mesh import Mesh


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_stiffness_kills_constants_and_is_symmetric_psd(p):
    m = Mesh((3.0, 4.0, 5.0), (2, 3, 2), p)
    K = assemble_stiffness(m)
    np.testing.assert_allclose(K @ np.ones(m.n_phi), 0.0, atol=1e-12)
    assert abs(K - K.T).max() < 1e-13
    ev = np.linalg.eigvalsh(K.toarray())
    assert ev[0] > -1e-10
    # exactly one zero mode on the periodic x/y, Neumann z mesh (constants)
    assert np.sum(np.abs(ev) < 1e-9) == 1


@pytest.mark.parametrize("p", [1, 3, 5])
def test_lumped_mass_total_and_moments(p):
    L = (3.0, 4.0, 5.0)
    m = Mesh(L, (2, 3, 2), p)
    M = lumped_mass(m)
    assert abs(M.sum() - np.prod(L)) < 1e-12
    z = m.phi_coords()[:, 2]
    for k in range(2 * p):   # GLL exactness per cell in z
        exact = L[0] * L[1] * L[2] ** (k + 1) / (k + 1)
        assert abs(M @ z ** k - exact) < 1e-10 * max(1.0, exact)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_stiffness_quadratic_form_closed_form(p):
    """u = f(x) z^2 with f a per-cell bubble t(h - t): u^T K u = int |grad u|^2 exactly."""
    L = (4.0, 3.0, 2.5)
    nc = (2, 3, 2)
    m = Mesh(L, nc, p)
    K = assemble_stiffness(m)
    X = m.phi_coords()
    hx = m.h[0]
    t = np.mod(X[:, 0], hx)
    t = np.where(np.abs(t - hx) < 1e-12, 0.0, t)
    u = t * (hx - t) * X[:, 2] ** 2
    fp2 = nc[0] * hx ** 3 / 3.0
    f2 = nc[0] * hx ** 5 / 30.0
    exact = fp2 * L[1] * L[2] ** 5 / 5.0 + f2 * L[1] * 4.0 * L[2] ** 3 / 3.0
    assert abs(u @ (K @ u) - exact) < 1e-11 * exact


def test_reference_cell_stiffness_p1_unit_cube():
    """Trilinear unit cube: diagonal 1/3, opposite-corner coupling -1/12."""
    m = Mesh((1.0, 1.0, 1.0), (1, 1, 1), 1)
    Ke = reference_cell_stiffness(m)
    assert abs(Ke[0, 0] - 1 / 3) < 1e-14
    assert abs(Ke[0, 7] + 1 / 12) < 1e-14
    assert abs(Ke[0, 1] - 0.0) < 1e-14     # edge neighbour of a trilinear cube: 0
    assert abs(Ke[0, 3] + 1 / 12) < 1e-14  # face-diagonal neighbour: -1/12


@pytest.mark.parametrize("dirichlet", [(True, True), (False, True), (False, False)])
def test_row_evaluation_matches_assembled(dirichlet):
    m = Mesh((3.0, 3.0, 6.0), (2, 2, 3), 3, psi_dirichlet=dirichlet)
    rng = np.random.default_rng(0)
    V = rng.standard_normal(m.n_psi)
    X = rng.standard_normal((m.n_psi, 3))
    H = hamiltonian(m, V)
    rows = rng.choice(m.n_psi, 25, replace=False)
    np.testing.assert_allclose(apply_H_rows(m, V, X, rows), (H @ X)[rows], rtol=1e-12,
                               atol=1e-12)


def test_one_cell_periodic_wrap():
    """With one cell per periodic direction the cell touches the same node twice."""
    m = Mesh((2.0, 2.0, 2.0), (1, 1, 2), 2)
    K = assemble_stiffness(m)
    np.testing.assert_allclose(K @ np.ones(m.n_phi), 0.0, atol=1e-12)
    H = hamiltonian(m, np.zeros(m.n_psi))
    X = np.random.default_rng(1).standard_normal((m.n_psi, 2))
    rows = np.arange(m.n_psi)
    np.testing.assert_allclose(apply_H_rows(m, np.zeros(m.n_psi), X, rows), H @ X,
                               rtol=1e-12, atol=1e-12)


def _box_levels(L, nmax=4):
    out = []
    for nx in range(-nmax, nmax + 1):
        for ny in range(-nmax, nmax + 1):
            for nz in range(1, nmax + 2):
                out.append(0.5 * ((2 * math.pi * nx / L[0]) ** 2 + (2 * math.pi * ny / L[1]) ** 2
                                  + (math.pi * nz / L[2]) ** 2))
    return np.sort(out)


def test_particle_in_a_box_converges_at_rate_2p():
    """V = 0, psi Dirichlet in z, periodic x/y: eps = 1/2 |k|^2 with error O(h^2p)."""
    L = (3.0, 3.0, 4.0)
    exact = _box_levels(L)[:8]
    errs = []
    for nc in [(2, 2, 4), (4, 4, 8)]:
        m = Mesh(L, nc, 2)
        H = hamiltonian(m, np.zeros(m.n_psi)).toarray()
        ev = sla.eigvalsh(H)[:8]
        errs.append(np.max(np.abs(ev - exact)))
    # degeneracy pattern on the finer mesh: (0,0,1), (0,0,2), then the 4-fold
    # (+-1,0,1), (0,+-1,1) (the coarse mesh, 4 nodes per period, splits it)
    assert abs(ev[2] - ev[5]) < 1e-8 and abs(ev[1] - ev[2]) > 0.1
    assert errs[1] < 0.05
    # h halves: the error must fall by at least ~2^(2p) / 2 (2^(2p) asymptotically)
    assert errs[0] / errs[1] > 2 ** (2 * 2) / 2


@pytest.mark.parametrize("p", [2, 3])
def test_hamiltonian_symmetric_and_spectrum_matches_generalised_problem(p):
    m = Mesh((2.0, 2.0, 3.0), (2, 2, 2), p)
    rng = np.random.default_rng(3)
    V = rng.standard_normal(m.n_psi)
    H = hamiltonian(m, V).toarray()
    assert np.max(np.abs(H - H.T)) < 1e-13
    K = assemble_stiffness(m)
    M = lumped_mass(m)
    ids = m.psi_to_phi()
    Hg = 0.5 * K[ids][:, ids].toarray() + np.diag(M[ids] * V)
    ev_g = sla.eigh(Hg, np.diag(M[ids]), eigvals_only=True)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), ev_g, rtol=1e-10, atol=1e-10)

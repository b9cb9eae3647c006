"""Pins of the oracle's Gauss-quadrature potential (oracle/quadpot.py) against what the
mathematics fixes: the textbook consistent element mass matrices for p = 1 and p = 2
(V = 1), row sums equal to the lumped mass (the Gauss rule integrates each basis function
exactly), closed-form integrals of V u^2 for fields the basis represents exactly,
interpolation that reproduces polynomials, a constant potential whose eigenvector is
M^1/2 1 with eigenvalue V (Neumann z faces), symmetry and positivity, and the row-by-row
form against the assembled matrix."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assembly, quadpot
from oracle.mesh import Mesh as OMesh


def _assembled_1d(elem, n, periodic, p):
    """Assembly of a 1D element matrix over n cells (periodic wrap or not)."""
    N = n * p if periodic else n * p + 1
    A = np.zeros((N, N))
    for c in range(n):
        idx = [(c * p + i) % N if periodic else c * p + i for i in range(p + 1)]
        for a in range(p + 1):
            for b in range(p + 1):
                A[idx[a], idx[b]] += elem[a, b]
    return A


@pytest.mark.parametrize("p,elem", [
    (1, lambda h: h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])),
    (2, lambda h: h / 30.0 * np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]])),
])
def test_unit_potential_is_the_consistent_mass(p, elem):
    """V = 1: the matrix is the consistent mass, the tensor product of the textbook 1D
    element masses (p = 2 GLL nodes are the interval's ends and midpoint)."""
    L, ncell = (3.0, 4.0, 5.0), (3, 4, 2)
    om = OMesh(L, ncell, p, (True, True))
    V = quadpot.potential_matrix(om, np.ones((om.n_cells, (p + 1) ** 3))).toarray()
    h = [L[d] / ncell[d] for d in range(3)]
    Mx = _assembled_1d(elem(h[0]), ncell[0], True, p)
    My = _assembled_1d(elem(h[1]), ncell[1], True, p)
    Mz = _assembled_1d(elem(h[2]), ncell[2], False, p)
    ref = np.kron(Mz, np.kron(My, Mx))        # phi id = gx + NX (gy + NY gz)
    assert np.max(np.abs(V - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", [1, 3, 4, 6])
def test_row_sums_are_the_lumped_mass(p):
    om = OMesh((4.0, 4.5, 6.0), (2, 3, 2), p, (False, True))
    V = quadpot.potential_matrix(om, np.ones((om.n_cells, (p + 1) ** 3)))
    M = assembly.lumped_mass(om)
    np.testing.assert_allclose(np.asarray(V.sum(axis=1)).ravel(), M, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [1, 2, 5])
def test_quadratic_forms_match_closed_form_integrals(p):
    """u^T V u = int V u^2 for fields the basis holds exactly: u = 1 with
    V = 2 + 0.3 x - 0.7 z, and u = z with V = 1 + z (degree <= 2p+1 per direction)."""
    L = (3.0, 2.5, 4.0)
    om = OMesh(L, (3, 2, 3), p, (True, True))
    xq = quadpot.quadrature_points(om)
    vol = L[0] * L[1] * L[2]
    V1 = 2.0 + 0.3 * xq[..., 0] - 0.7 * xq[..., 2]
    u = np.ones(om.n_phi)
    got = u @ (quadpot.potential_matrix(om, V1) @ u)
    ref = vol * (2.0 + 0.3 * L[0] / 2 - 0.7 * L[2] / 2)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    V2 = 1.0 + xq[..., 2]
    z = om.phi_coords()[:, 2]
    got = z @ (quadpot.potential_matrix(om, V2) @ z)
    ref = L[0] * L[1] * (L[2] ** 3 / 3 + L[2] ** 4 / 4)
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_interpolation_reproduces_polynomials():
    """f = x z + y^2 - 2 z^2 (degree 2 per direction, p = 2) at the Gauss points of every
    cell that does not touch the periodic wrap (where the nodal values of a non-periodic f
    are those of the first row)."""
    om = OMesh((3.0, 3.0, 4.0), (3, 3, 2), 2, (True, True))
    X = om.phi_coords()
    f = lambda x, y, z: x * z + y ** 2 - 2.0 * z ** 2
    fq = quadpot.interpolate_to_quad(om, f(X[:, 0], X[:, 1], X[:, 2]))
    xq = quadpot.quadrature_points(om)
    ref = f(xq[..., 0], xq[..., 1], xq[..., 2])
    nx, ny, nz = om.ncell
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inner = ((cx < nx - 1) & (cy < ny - 1)).ravel()
    assert np.max(np.abs(fq[inner] - ref[inner])) <= 1e-13 * np.max(np.abs(ref))


def test_constant_potential_eigenpair():
    """Neumann z faces, V = c at every Gauss point: K 1 = 0 and V 1 = c M 1, so
    Ht_q M^1/2 1 = c M^1/2 1."""
    om = OMesh((4.0, 4.0, 5.0), (2, 2, 3), 3, (False, False))
    c = -0.37
    H = quadpot.hamiltonian_quad(om, np.full((om.n_cells, 64), c))
    v = np.sqrt(assembly.lumped_mass(om))[om.psi_to_phi()]
    assert np.max(np.abs(H @ v - c * v)) <= 1e-13 * np.max(np.abs(v))


def test_symmetric_and_positive_for_positive_potential():
    om = OMesh((3.0, 3.0, 4.0), (2, 2, 2), 3, (True, True))
    rng = np.random.default_rng(1)
    Vq = rng.uniform(0.5, 2.0, (om.n_cells, 64))
    V = quadpot.potential_matrix(om, Vq).toarray()
    assert np.max(np.abs(V - V.T)) <= 1e-15 * np.max(np.abs(V))
    assert sla.eigvalsh(V)[0] > 0.0


@pytest.mark.parametrize("faces,ncell", [((True, True), (2, 3, 2)), ((False, True), (1, 2, 2)),
                                         ((True, False), (3, 1, 1))])
def test_rows_match_the_assembled_operator(faces, ncell):
    om = OMesh((3.0, 3.5, 4.0), ncell, 2, faces)
    rng = np.random.default_rng(4)
    Vq = rng.uniform(-1.0, 1.0, (om.n_cells, 27))
    H = quadpot.hamiltonian_quad(om, Vq)
    X = rng.standard_normal((om.n_psi, 3))
    rows = np.arange(om.n_psi)
    got = quadpot.apply_Hq_rows(om, Vq, X, rows)
    np.testing.assert_allclose(got, H @ X, rtol=0, atol=1e-12 * np.max(np.abs(H @ X)))

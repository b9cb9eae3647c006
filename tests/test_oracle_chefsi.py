"""Pins of the oracle's Chebyshev filter, Lanczos bounds and Rayleigh-Ritz steps."""
import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import chebyshev as cheb

from oracle.assembly import hamiltonian
from oracle.chefsi import cheb_filter, chefsi_cycle, lanczos_bounds, rayleigh_ritz
from oracle.mesh import Mesh


@pytest.mark.parametrize("m", [1, 2, 5, 10])
def test_filter_on_eigenvectors_is_scaled_chebyshev(m):
    """Filter of an eigenvector (lam, v) returns T_m((lam - c)/e) / T_m((a0 - c)/e) v."""
    lam = np.array([-1.0, -0.7, 0.2, 1.5, 3.0, 7.5, 10.0])
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    A = Q @ np.diag(lam) @ Q.T
    a, b, a0 = 0.5, 10.0, -1.0
    e, c = (b - a) / 2, (b + a) / 2
    Tm = lambda x: cheb.chebval(x, [0] * m + [1])
    Y = cheb_filter(lambda X: A @ X, Q, m, a, b, a0)
    expect = Q * (Tm((lam - c) / e) / Tm((a0 - c) / e))[None, :]
    np.testing.assert_allclose(Y, expect, rtol=1e-12, atol=1e-12)
    # the scaling makes the filter exactly 1 at a0
    assert abs(Tm((a0 - c) / e) / Tm((a0 - c) / e) - 1.0) == 0.0


def test_lanczos_upper_bound_and_low_estimate():
    m = Mesh((3.0, 3.0, 6.0), (2, 2, 3), 3)
    rng = np.random.default_rng(4)
    V = -np.abs(rng.standard_normal(m.n_psi))
    H = hamiltonian(m, V)
    ev = sla.eigvalsh(H.toarray())
    lo, hi = lanczos_bounds(lambda v: H @ v, rng.standard_normal(m.n_psi), 40)
    assert hi >= ev[-1]
    assert hi <= ev[-1] * 1.2
    assert lo >= ev[0] - 1e-10 and lo < ev[0] + 0.1 * (ev[-1] - ev[0])


def test_rayleigh_ritz_exact_on_invariant_subspace():
    m = Mesh((3.0, 3.0, 6.0), (2, 2, 3), 2)
    rng = np.random.default_rng(5)
    H = hamiltonian(m, rng.standard_normal(m.n_psi)).toarray()
    lam, U = np.linalg.eigh(H)
    Y = U[:, :6] @ rng.standard_normal((6, 6))   # mixed basis of an invariant subspace
    r, X = rayleigh_ritz(lambda Z: H @ Z, Y)
    np.testing.assert_allclose(r, lam[:6], atol=1e-11)
    np.testing.assert_allclose(X.T @ X, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(H @ X, X * r[None, :], atol=1e-10)


def test_chefsi_converges_to_dense_eigh():
    """Repeated filter + RR cycles converge to the lowest eigenvalues of the dense matrix."""
    m = Mesh((3.0, 3.0, 6.0), (2, 2, 4), 2)
    rng = np.random.default_rng(6)
    V = -0.5 * np.abs(rng.standard_normal(m.n_psi))
    H = hamiltonian(m, V)
    ev = np.linalg.eigvalsh(H.toarray())
    n, k = 12, 8
    ap = lambda Z: H @ Z
    lo, hi = lanczos_bounds(ap, rng.standard_normal(m.n_psi), 30)
    X = rng.standard_normal((m.n_psi, n))
    a0 = lo
    a = ev[n + 2]
    for _ in range(25):
        r, X = chefsi_cycle(ap, X, 12, a, hi, a0)
        a0 = r[0]
    np.testing.assert_allclose(r[:k], ev[:k], atol=1e-10)

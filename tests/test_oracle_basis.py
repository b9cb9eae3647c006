"""Pins of the oracle's GLL basis (Section 2.3) against closed forms and exactness."""
import math

import numpy as np
import pytest

from oracle.basis import gll, lagrange_derivs, lagrange_values

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("p,nodes,weights", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], [0.1, 49 / 90, 32 / 45, 49 / 90, 0.1]),
])
def test_gll_closed_forms(p, nodes, weights):
    x, w = gll(p)
    np.testing.assert_allclose(x, nodes, atol=1e-15)
    np.testing.assert_allclose(w, weights, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_quadrature_exact_to_2p_minus_1(p):
    x, w = gll(p)
    for k in range(0, 2 * p):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # and not exact at degree 2p (a wrong node set usually is)
    k = 2 * p
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_lagrange_cardinal_and_partition(p):
    x, _ = gll(p)
    B = lagrange_values(x, x)
    np.testing.assert_allclose(B, np.eye(p + 1), atol=1e-14)
    t = np.linspace(-1, 1, 17)
    np.testing.assert_allclose(lagrange_values(x, t).sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(lagrange_derivs(x, t).sum(axis=1), 0.0, atol=1e-11)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_lagrange_derivative_reproduces_polynomials(p):
    x, _ = gll(p)
    t = np.linspace(-0.9, 0.95, 11)
    D = lagrange_derivs(x, t)
    for k in range(p + 1):
        np.testing.assert_allclose(D @ (x ** k), k * t ** (k - 1) if k else 0 * t, atol=1e-11)

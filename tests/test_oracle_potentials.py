"""Pins of the oracle's atom-centred fields and sawtooth (Eq. Governing equations, Sec. 2.2.1)."""
import math

import numpy as np
import pytest

from oracle.assembly import lumped_mass
from oracle.mesh import Mesh
from oracle.potentials import (densities, gaussian_radial, v_app, vloc_minus_vsm_radial,
                               vsm_radial)


def _radial_laplacian(f, r, h=1e-3):
    """(1/r) d^2 (r f) / dr^2 by a 4th-order central difference."""
    g = lambda s: s * f(s)
    d2 = (-g(r + 2 * h) + 16 * g(r + h) - 30 * g(r) + 16 * g(r - h) - g(r - 2 * h)) / (12 * h * h)
    return d2 / r


@pytest.mark.parametrize("sigma", [0.5, 0.8])
def test_vsm_solves_poisson_with_smeared_charge(sigma):
    """-1/(4 pi) Lap V_sm = b_sm = -Z g_sigma: pins the sigma convention of the pair."""
    r = np.array([0.3, 0.7, 1.1, 1.9])
    Z = 3.0
    lap = _radial_laplacian(lambda s: vsm_radial(s, Z, sigma), r)
    np.testing.assert_allclose(-lap / (4 * math.pi), -Z * gaussian_radial(r, sigma), rtol=1e-7)


def test_gaussian_normalised():
    r = np.linspace(0, 12, 200001)
    for s in (0.5, 1.0):
        val = np.trapezoid(4 * math.pi * r ** 2 * gaussian_radial(r, s), r)
        assert abs(val - 1.0) < 1e-9


def test_vloc_minus_vsm_limits():
    Z = 2.0
    lim = Z * 2 / math.sqrt(math.pi) * (math.sqrt(2.0) - 1.0)
    assert abs(vloc_minus_vsm_radial(0.0, Z) - lim) < 1e-15
    assert abs(vloc_minus_vsm_radial(1e-6, Z) - lim) < 1e-10
    # beyond a few bohr both erf -> 1 and the difference vanishes
    assert abs(vloc_minus_vsm_radial(8.0, Z)) < 1e-20
    # V_loc = -Z erf(r)/r, V_sm = -Z erf(sqrt2 r)/r with sigma_b = 0.5
    r = 0.9
    vloc = -Z * math.erf(r) / r
    assert abs(vloc_minus_vsm_radial(r, Z) - (vloc - vsm_radial(r, Z))) < 1e-15


def test_discrete_renormalisation():
    m = Mesh((4.0, 4.0, 8.0), (2, 2, 4), 3)
    X = m.phi_coords()
    M = lumped_mass(m)
    R = np.array([[0.3, 3.9, 4.1], [2.2, 1.0, 3.7]])   # near the periodic seam
    Z = np.array([1.0, 3.0])
    rho, b = densities(X, M, R, Z, m.L)
    assert abs(M @ rho - 4.0) < 1e-12
    assert abs(M @ b + 4.0) < 1e-12
    assert np.all(rho >= 0) and np.all(b <= 0)


def test_sawtooth_shape():
    Lz, E = 20.0, 0.03
    z = np.linspace(0, Lz, 2001)
    v = v_app(z, E, Lz)
    assert abs(v[0]) < 1e-15 and abs(v[-1]) < 1e-15
    mid = (z > 2.0 + 1e-9) & (z < 18.0 - 1e-9)
    slope = np.diff(v)[mid[:-1] & mid[1:]] / np.diff(z)[mid[:-1] & mid[1:]]
    np.testing.assert_allclose(slope, -E, rtol=1e-9)
    assert np.argmax(v) == np.argmin(np.abs(z - 2.0))
    assert np.argmin(v) == np.argmin(np.abs(z - 18.0))
    assert np.max(np.abs(np.diff(v))) < 1.01 * E * 0.4 * Lz / 2.0 * (z[1] - z[0])

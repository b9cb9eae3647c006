"""Pins of the analysis outputs (oracle/analysis.py): planar integrals of an in-plane
constant reproduce area x value and integrate back to the volume integral exactly; planar
averages of a function of z alone return it; the dipole of a pair of opposite point-like
sheets is charge x separation and vanishes for a mirror-symmetric neutral distribution;
the polarisability of a linear response is its slope."""
import numpy as np

from oracle import analysis, assembly
from oracle.mesh import Mesh as OMesh


def _mesh():
    om = OMesh((3.0, 5.0, 8.0), (2, 3, 4), 3)
    return om, assembly.lumped_mass(om), om.phi_coords()


def test_planar_integral_and_average_of_z_functions():
    om, M, X = _mesh()
    z = X[:, 2]
    f = np.cos(0.7 * z) + z ** 2
    r0 = analysis.planar_integral(om, M, f)
    zplanes = X[:: om.NX * om.NY, 2]
    np.testing.assert_allclose(r0, 15.0 * (np.cos(0.7 * zplanes) + zplanes ** 2), rtol=1e-13)
    np.testing.assert_allclose(analysis.planar_average(om, M, f), f[:: om.NX * om.NY], rtol=1e-13)
    # summing rho0 with the z weights of the planes gives back the volume integral
    wz = np.array([analysis.plane_z_weight(om, gz) for gz in range(r0.shape[0])])
    assert abs(np.sum(wz * r0) - np.sum(M * f)) <= 1e-12 * np.sum(np.abs(M * f))


def test_planar_average_of_an_xy_mode_is_zero():
    om, M, X = _mesh()
    f = np.sin(2 * np.pi * X[:, 0] / 3.0) * (1 + X[:, 2])   # one full period in x
    assert np.max(np.abs(analysis.planar_average(om, M, f))) <= 1e-13


def test_dipole_of_two_sheets_and_of_a_symmetric_distribution():
    om, M, X = _mesh()
    z = X[:, 2]
    plane = om.NX * om.NY
    rho = np.zeros(om.n_phi)
    b = np.zeros(om.n_phi)
    # electrons on the plane z = 2, the same charge of nuclei on z = 6 (GLL planes of p = 3)
    zp = X[::plane, 2]
    i2, i6 = int(np.argmin(np.abs(zp - 2.0))), int(np.argmin(np.abs(zp - 6.0)))
    q = 1.5
    rho[i2 * plane:(i2 + 1) * plane] = q / np.sum(M[i2 * plane:(i2 + 1) * plane])
    b[i6 * plane:(i6 + 1) * plane] = -q / np.sum(M[i6 * plane:(i6 + 1) * plane])
    mu = analysis.dipole_z(M, rho, b, z, 8.0)
    assert abs(mu - q * (zp[i2] - zp[i6])) <= 1e-12
    sym = np.exp(-(z - 4.0) ** 2) - np.exp(-(z - 4.0) ** 2 / 4.0) / 2.0
    assert abs(analysis.dipole_z(M, sym, 0 * sym, z, 8.0)) <= 1e-12


def test_polarisability_is_the_slope():
    assert abs(analysis.polarisability(0.3, 0.3 + 2.5 * 0.04, 0.01, 0.05) - 2.5) <= 1e-14

"""Pins of the oracle's Poisson problem (Eq. Poissons equation with the CEF / CPD setups)."""
import math

import numpy as np
import pytest

from oracle.assembly import assemble_stiffness, lumped_mass
from oracle.mesh import Mesh
from oracle.poisson import (dipole_z, electrostatic_energy, reaction_charge, solve_cef_cg,
                            solve_cef_direct, solve_cpd_cg, solve_cpd_direct)
from oracle.potentials import cpd_constraints, densities, v_app, vloc_minus_vsm
from workloads import Bias


def _zplanes_mask(m, z, zvals):
    return np.isin(np.round(z, 12), np.round(np.asarray(zvals), 12))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_patch_polynomial_in_z_reproduced_exactly(p):
    """Dirichlet at z = 0, Lz; rho = -P''/(4 pi) with deg P = p gives phi = P at the nodes."""
    L = (2.0, 3.0, 5.0)
    m = Mesh(L, (2, 2, 3), p)
    K = assemble_stiffness(m)
    M = lumped_mass(m)
    z = m.phi_coords()[:, 2]
    coef = np.arange(1, p + 2) * 0.3 * (-1) ** np.arange(p + 1)
    P = np.polynomial.Polynomial(coef)
    rho = -P.deriv(2)(z) / (4 * math.pi)
    f = 4 * math.pi * M * rho
    mask = _zplanes_mask(m, z, [0.0, L[2]])
    phi = solve_cpd_direct(K, f, mask, np.where(mask, P(z), 0.0))
    np.testing.assert_allclose(phi, P(z), atol=1e-11 * np.max(np.abs(P(z))))


@pytest.mark.parametrize("p", [2, 4])
def test_cpd_empty_box_linear_potential_and_capacitor(p):
    """No charge: phi_tilde linear between Z_A and Z_B; E = -A dV^2 / (8 pi d)."""
    L = (3.0, 3.0, 10.0)
    m = Mesh(L, (2, 2, 5), p)
    K = assemble_stiffness(m)
    M = lumped_mass(m)
    X = m.phi_coords()
    z = X[:, 2]
    bias = Bias("cpd", dV=0.3, zA=2.0, zB=8.0)
    zero = np.zeros(m.n_phi)
    mask, vals, om0, om1 = cpd_constraints(X, zero, bias, L)
    phi = solve_cpd_direct(K, zero, mask, vals)
    d = bias.zB - bias.zA
    expect = np.clip((z - bias.zA) / d, 0.0, 1.0) * bias.dV
    np.testing.assert_allclose(phi, expect, atol=1e-12)
    A = L[0] * L[1]
    E = electrostatic_energy(K, phi, zero)
    assert abs(E + A * bias.dV ** 2 / (8 * math.pi * d)) < 1e-12
    dE = reaction_charge(K, phi, M, zero, zero, om1)
    assert abs(dE + A * bias.dV / (4 * math.pi * d)) < 1e-12
    # envelope identity: central difference of E in dV
    h = 1e-3
    Es = []
    for s in (+1, -1):
        b2 = Bias("cpd", dV=bias.dV + s * h, zA=2.0, zB=8.0)
        _, v2, _, _ = cpd_constraints(X, zero, b2, L)
        Es.append(electrostatic_energy(K, solve_cpd_direct(K, zero, mask, v2), zero))
    assert abs((Es[0] - Es[1]) / (2 * h) - dE) < 1e-9


@pytest.mark.parametrize("p", [1, 3])
def test_charged_sheet_kink(p):
    """Surface charge s on the plane z0: phi piecewise linear with jump -4 pi s in phi'."""
    L = (2.0, 2.0, 6.0)
    m = Mesh(L, (2, 2, 3), p)
    K = assemble_stiffness(m)
    X = m.phi_coords()
    z = X[:, 2]
    z0, s = 2.0, 0.05
    # c_I = s * int_plane N_I dA: the in-plane lumped weights of the nodes on z = z0
    on = np.abs(z - z0) < 1e-12
    w2 = np.outer(m.w, m.w) * (m.h[0] * m.h[1] / 4.0)
    area_w = np.zeros(m.n_phi)
    for cy in range(m.ncell[1]):
        for cx in range(m.ncell[0]):
            for j in range(m.p + 1):
                for i in range(m.p + 1):
                    gx = (cx * m.p + i) % m.NX
                    gy = (cy * m.p + j) % m.NY
                    gz = int(round(z0 / m.h[2])) * m.p
                    area_w[gx + m.NX * (gy + m.NY * gz)] += w2[j, i]
    assert abs(area_w.sum() - L[0] * L[1]) < 1e-12 and np.all(area_w[~on] == 0)
    f = 4 * math.pi * s * area_w
    mask = _zplanes_mask(m, z, [0.0, L[2]])
    phi = solve_cpd_direct(K, f, mask, np.zeros(m.n_phi))
    # A z0 = B (Lz - z0), A + B = 4 pi s
    B = 4 * math.pi * s * z0 / L[2]
    A = 4 * math.pi * s - B
    expect = np.where(z <= z0, A * z, B * (L[2] - z))
    np.testing.assert_allclose(phi, expect, atol=1e-12)


def test_neumann_cosine_converges():
    """rho = A cos(pi k z / Lz) (zero mean): phi = 4 pi A (Lz/(pi k))^2 cos(...), mean zero."""
    L = (2.0, 2.0, 6.0)
    Acoef, k = 0.2, 2
    errs = []
    for nz in (3, 6):
        m = Mesh(L, (1, 1, nz), 3)
        K = assemble_stiffness(m)
        M = lumped_mass(m)
        z = m.phi_coords()[:, 2]
        rho = Acoef * np.cos(math.pi * k * z / L[2])
        phi = solve_cef_direct(K, 4 * math.pi * M * rho, M)
        assert abs(M @ phi) < 1e-12
        exact = 4 * math.pi * Acoef * (L[2] / (math.pi * k)) ** 2 * np.cos(math.pi * k * z / L[2])
        errs.append(np.max(np.abs(phi - exact)))
    assert errs[1] < 2e-4
    assert errs[0] / errs[1] > 2 ** 4 / 2   # O(h^(p+1)) for p = 3


def _slab_fields(m, R, Z):
    X = m.phi_coords()
    M = lumped_mass(m)
    rho, b = densities(X, M, R, Z, m.L)
    vl = vloc_minus_vsm(X, R, Z, m.L)
    return X, M, rho, b, vl


def test_cg_matches_direct_cef_and_cpd():
    L = (4.0, 4.0, 10.0)
    m = Mesh(L, (2, 2, 5), 3)
    K = assemble_stiffness(m)
    R = np.array([[1.0, 1.5, 4.5], [3.0, 2.5, 5.5]])
    Z = np.array([1.0, 2.0])
    X, M, rho, b, vl = _slab_fields(m, R, Z)
    assert abs(M @ (rho + b)) < 1e-12
    f = 4 * math.pi * M * (rho + b)
    pd = solve_cef_direct(K, f, M)
    pc, it, rel = solve_cef_cg(K, f, M, rtol=1e-12)
    assert rel <= 1e-12 and it > 5
    np.testing.assert_allclose(pc, pd, atol=1e-9 * np.max(np.abs(pd)))
    bias = Bias("cpd", dV=0.02, zA=1.0, zB=9.0)
    mask, vals, om0, om1 = cpd_constraints(X, vl, bias, L)
    pd = solve_cpd_direct(K, f, mask, vals)
    pc, it, rel = solve_cpd_cg(K, f, mask, vals, rtol=1e-12)
    np.testing.assert_allclose(pc, pd, atol=1e-9 * np.max(np.abs(pd)))
    # phi_tilde = phi + (V_loc - V_sm) is 0 on Omega_0 and dV on Omega_1 (Eq. APD)
    np.testing.assert_allclose((pd + vl)[om0], 0.0, atol=1e-14)
    np.testing.assert_allclose((pd + vl)[om1], bias.dV, atol=1e-14)


def test_lcpd_patch_constrains_only_the_patch():
    L = (6.0, 6.0, 10.0)
    m = Mesh(L, (3, 3, 5), 2)
    X = m.phi_coords()
    zero = np.zeros(m.n_phi)
    bias = Bias("cpd", dV=0.1, zA=1.0, zB=9.0, patch=((2.0, 2.0), (4.0, 4.0)))
    mask, vals, om0, om1 = cpd_constraints(X, zero, bias, L)
    full = Bias("cpd", dV=0.1, zA=1.0, zB=9.0)
    _, _, _, om1_full = cpd_constraints(X, zero, full, L)
    assert 0 < om1.sum() < om1_full.sum()
    inside = (X[:, 0] >= 2 - 1e-12) & (X[:, 0] <= 4 + 1e-12) & (X[:, 1] >= 2 - 1e-12) & (
        X[:, 1] <= 4 + 1e-12)
    assert np.array_equal(om1, om1_full & inside)


def test_hellmann_feynman_dipole_and_symmetry():
    """dE/dE_field = -mu_z when the charge lies in the linear part of V_app (Section 3.1);
    an inversion-symmetric slab has mu_z = 0 at zero field."""
    L = (4.0, 4.0, 24.0)
    m = Mesh(L, (2, 2, 12), 2)
    K = assemble_stiffness(m)
    # atoms symmetric under (x, y, z) -> (L - x, L - y, L - z) about the cell centre;
    # all charge lies well inside the linear part [0.1 Lz, 0.9 Lz] of V_app
    R = np.array([[1.0, 1.0, 11.0], [3.0, 3.0, 13.0]])
    Z = np.array([1.0, 1.0])
    X, M, rho, b, vl = _slab_fields(m, R, Z)
    z = X[:, 2]
    mu = dipole_z(M, rho, b, z, L[2])
    assert abs(mu) < 1e-12
    R2 = np.array([[1.0, 1.0, 11.0], [3.0, 3.0, 12.2]])
    X, M, rho, b, vl = _slab_fields(m, R2, Z)
    phi = solve_cef_direct(K, 4 * math.pi * M * (rho + b), M)
    c = M * (rho + b)

    def E(field):
        return electrostatic_energy(K, phi, c) + M @ (vl * rho) + M @ ((rho + b) * v_app(z, field, L[2]))

    h = 1e-4
    dE = (E(0.01 + h) - E(0.01 - h)) / (2 * h)
    mu = dipole_z(M, rho, b, z, L[2])
    assert abs(mu) > 1e-3
    assert abs(dE + mu) < 1e-8 * abs(mu)

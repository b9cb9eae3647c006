"""Differentiation form: energy parity with the oracle, adjoint Poisson gradients and the
energy gradients (dE/d dV, dE/d field, dE/d R_z) against central finite differences
(step 1e-4) and the Hellmann-Feynman dipole, on the 12 x 12 x 40-cell p = 4 constrained-
potential slab (128 atoms, 370,944 phi nodes).

Tolerances: gradients 1e-6 relative to central differences (the solves run to 1e-12 and the
energy is stationary in phi, so the difference quotient carries only O(h^2) truncation and
round-off of order 1e-14 E / h); energy vs oracle 1e-9 relative.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import assembly, poisson, potentials
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu

H_FD = 1e-4
RTOL = 1e-13


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


@pytest.fixture(scope="module")
def ag():
    import paper_2504_00998_gb300.autograd as ag
    return ag


@pytest.mark.parametrize("kind", ["cef", "cpd"])
def test_energy_matches_oracle(fe, kind):
    base = W.small_slab(ncell=(3, 3, 6), p=3, L=(6.0, 6.0, 16.0), natoms=3, seed=21)
    bias = W.Bias("cef", field=0.02) if kind == "cef" else W.Bias("cpd", dV=0.04, zA=1.5, zB=14.5)
    slab = dataclasses.replace(base, bias=bias)
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    X = om.phi_coords()
    rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
    f = 4 * math.pi * M * (rho + b)
    if kind == "cef":
        phi = poisson.solve_cef_direct(K, f, M)
        vapp = potentials.v_app(X[:, 2], bias.field, slab.L[2])
    else:
        mask, vals, om0, om1 = potentials.cpd_constraints(X, vl, bias, slab.L)
        phi = poisson.solve_cpd_direct(K, f, mask, vals)
        vapp = 0 * X[:, 2]
    E_ref = poisson.total_energy(K, phi, M, rho, b, vl, vapp)
    m = fe.Mesh.from_slab(slab)
    phig, _, _ = m.poisson_solve(bias, rtol=RTOL)
    E, dEf, dEdV, *_ = m.energy(bias, phig)
    assert abs(E - E_ref) <= 1e-9 * abs(E_ref)
    if kind == "cpd":
        r_ref = poisson.reaction_charge(K, phi, M, rho, b, om1)
        assert abs(dEdV - r_ref) <= 1e-8 * max(1.0, abs(r_ref))
    else:
        # dE/dE_field = sum M (rho + b) dV_app/dE exactly; it equals -mu_z only up to the
        # charge that reaches the return ramps of V_app (Gaussian tails here, ~1e-9)
        dva = potentials.dv_app_dfield(X[:, 2], slab.L[2])
        ref = float(M @ ((rho + b) * dva))
        assert abs(dEf - ref) <= 1e-10 * abs(ref)
        assert abs(dEf + poisson.dipole_z(M, rho, b, X[:, 2], slab.L[2])) <= 1e-7 * abs(ref)


@pytest.fixture(scope="module")
def slab3():
    return W.config3()


def _E(fe, ag, m, slab, R, field, dV, bias):
    return ag.slab_energy(m, R, slab.Z, bias, field=field, dV=dV, rtol=RTOL)


def test_dE_ddV_and_dE_dR_match_finite_differences(fe, ag, slab3):
    m = fe.Mesh.from_slab(slab3, with_atoms=False)
    R = torch.tensor(slab3.R, dtype=torch.float64, requires_grad=True)
    dV = torch.tensor(slab3.bias.dV, dtype=torch.float64, requires_grad=True)
    field = torch.tensor(0.0, dtype=torch.float64)
    E = _E(fe, ag, m, slab3, R, field, dV, slab3.bias)
    gR, gdV = torch.autograd.grad(E, (R, dV))
    # dE/d dV
    Ep = _E(fe, ag, m, slab3, R.detach(), field, dV.detach() + H_FD, slab3.bias).item()
    Em = _E(fe, ag, m, slab3, R.detach(), field, dV.detach() - H_FD, slab3.bias).item()
    fd = (Ep - Em) / (2 * H_FD)
    assert abs(gdV.item() - fd) <= 1e-6 * abs(fd), (gdV.item(), fd)
    # dE/d R_z for atoms in the bottom, middle and top layers
    scale = float(torch.max(torch.abs(gR[:, 2])))
    for a in (0, 40, 127):
        Rp = R.detach().clone(); Rp[a, 2] += H_FD
        Rm = R.detach().clone(); Rm[a, 2] -= H_FD
        fd = (_E(fe, ag, m, slab3, Rp, field, dV.detach(), slab3.bias).item() -
              _E(fe, ag, m, slab3, Rm, field, dV.detach(), slab3.bias).item()) / (2 * H_FD)
        g = gR[a, 2].item()
        assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-2 * scale), (a, g, fd)
    # an in-plane component as well
    Rp = R.detach().clone(); Rp[5, 0] += H_FD
    Rm = R.detach().clone(); Rm[5, 0] -= H_FD
    fd = (_E(fe, ag, m, slab3, Rp, field, dV.detach(), slab3.bias).item() -
          _E(fe, ag, m, slab3, Rm, field, dV.detach(), slab3.bias).item()) / (2 * H_FD)
    assert abs(gR[5, 0].item() - fd) <= 1e-6 * max(abs(fd), 1e-2 * scale)


def test_dE_dfield_is_minus_dipole(fe, ag, slab3):
    """Same slab under a constant field: dE/dE = -mu_z (Section 3.1 dipole) and = FD."""
    bias = W.Bias("cef", field=0.005)
    m = fe.Mesh.from_slab(slab3, with_atoms=False)
    R = torch.tensor(slab3.R, dtype=torch.float64)
    field = torch.tensor(bias.field, dtype=torch.float64, requires_grad=True)
    dV = torch.tensor(0.0, dtype=torch.float64)
    E = _E(fe, ag, m, slab3, R, field, dV, bias)
    (gf,) = torch.autograd.grad(E, (field,))
    Ep = _E(fe, ag, m, slab3, R, field.detach() + H_FD, dV, bias).item()
    Em = _E(fe, ag, m, slab3, R, field.detach() - H_FD, dV, bias).item()
    fd = (Ep - Em) / (2 * H_FD)
    assert abs(gf.item() - fd) <= 1e-6 * abs(fd)
    rho, b, _ = m.atom_fields()
    M = m.lumped_mass()
    z = m.node_coords()[:, 2]
    mu = float(torch.sum(M * (rho + b) * (z - slab3.L[2] / 2)))
    assert abs(gf.item() + mu) <= 1e-8 * abs(mu)


@pytest.mark.parametrize("kind", ["cef", "cpd"])
def test_poisson_adjoint_matches_finite_differences(fe, ag, kind):
    slab = W.small_slab(ncell=(3, 3, 6), p=3, L=(6.0, 6.0, 14.0), natoms=3, seed=9)
    bias = W.Bias("cef", field=0.0) if kind == "cef" else W.Bias("cpd", dV=0.03, zA=1.5, zB=12.5)
    m = fe.Mesh.from_slab(slab)
    rng = np.random.default_rng(3)
    n = m.n_phi
    f0, _, _ = m.poisson_rhs()
    w = torch.tensor(rng.standard_normal(n), device="cuda")
    mask, vals = m.poisson_constraints(bias)
    f = f0.clone().requires_grad_(True)
    phic = vals.clone().requires_grad_(True) if kind == "cpd" else None
    phi = ag.poisson_solve(m, f, bias, phic=phic, rtol=RTOL)
    L = torch.sum(w * phi)
    grads = torch.autograd.grad(L, (f, phic) if phic is not None else (f,))
    d = torch.tensor(rng.standard_normal(n), device="cuda")
    if kind == "cef":
        d = d - d.mean()

    def Lof(ff, pc):
        return float(torch.sum(w * ag.poisson_solve(m, ff, bias, phic=pc, rtol=RTOL)))

    h = 1e-3
    fd = (Lof(f0 + h * d, phic.detach() if phic is not None else None) -
          Lof(f0 - h * d, phic.detach() if phic is not None else None)) / (2 * h)
    an = float(torch.sum(grads[0] * d))
    assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)
    if kind == "cpd":
        dc = torch.where(mask, torch.tensor(rng.standard_normal(n), device="cuda"),
                         torch.zeros(n, dtype=torch.float64, device="cuda"))
        fd = (Lof(f0, phic.detach() + h * dc) - Lof(f0, phic.detach() - h * dc)) / (2 * h)
        an = float(torch.sum(grads[1] * dc))
        assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)


def _hx_loss(ag, m, X, V, W, prec):
    Y = ag.apply_H(m, X, V, prec)
    # quadratic in Y so that Ybar = W + Y depends on the forward result
    return (W.conj() * Y).real.sum() + 0.5 * (Y.abs() ** 2).sum()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hamiltonian_autograd(fe, ag, prec):
    """dL/dX = Ht Ybar and dL/dV = sum_v Ybar X through the adjoint kernels, against the
    oracle's assembled Ht and central finite differences (step 1e-4) along random
    directions; the loss is quadratic in (X, V) direction by direction, so the difference
    quotient carries round-off only."""
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.float64 if prec == "f64" else torch.float32
    L, nc, p = (4.0, 4.0, 9.0), (2, 2, 4), 3
    om = OMesh(L, nc, p)
    m = fe.Mesh(L, nc, p)
    rng = np.random.default_rng(51)
    Vn = rng.uniform(-1.0, 1.0, om.n_psi)
    Xn = rng.standard_normal((om.n_psi, 8)).astype(np.float32).astype(np.float64)
    Wn = rng.standard_normal((om.n_psi, 8))
    V = torch.tensor(Vn, device="cuda", requires_grad=True)
    X = torch.tensor(Xn, dtype=dt, device="cuda", requires_grad=True)
    W = torch.tensor(Wn, dtype=dt, device="cuda")
    _hx_loss(ag, m, X, V, W, p_).backward()
    H = assembly.hamiltonian(om, Vn)
    Ybar = Wn + H @ Xn
    gX_ref, gV_ref = H @ Ybar, np.sum(Ybar * Xn, axis=1)
    tol = 1e-10 if prec == "f64" else 2e-5
    gX, gV = X.grad.double().cpu().numpy(), V.grad.cpu().numpy()
    assert np.linalg.norm(gX - gX_ref) / np.linalg.norm(gX_ref) <= tol
    assert np.linalg.norm(gV - gV_ref) / np.linalg.norm(gV_ref) <= tol
    if prec == "f64":
        with torch.no_grad():
            for _ in range(2):
                dV = torch.tensor(rng.standard_normal(om.n_psi), device="cuda")
                dX = torch.tensor(rng.standard_normal(Xn.shape), device="cuda")
                fd_v = (_hx_loss(ag, m, X, V + H_FD * dV, W, p_)
                        - _hx_loss(ag, m, X, V - H_FD * dV, W, p_)).item() / (2 * H_FD)
                fd_x = (_hx_loss(ag, m, X + H_FD * dX, V, W, p_)
                        - _hx_loss(ag, m, X - H_FD * dX, V, W, p_)).item() / (2 * H_FD)
                an_v = float((V.grad * dV).sum())
                an_x = float((X.grad * dX).sum())
                assert abs(fd_v - an_v) <= 1e-6 * abs(an_v)
                assert abs(fd_x - an_x) <= 1e-6 * abs(an_x)


def test_hamiltonian_autograd_bloch(fe, ag):
    """Complex blocks at a Bloch wave vector: dL/dX = Ht_k Ybar (Hermitian) and
    dL/dV = Re sum_v Ybar conj(X), checked by central differences along real V and complex
    X directions (PyTorch's convention: dL = Re sum conj(grad) dX)."""
    L, nc, p = (4.0, 4.0, 9.0), (2, 2, 4), 3
    m = fe.Mesh(L, nc, p)
    m.set_kpoint(0.3, -0.2)
    n = m.n_psi
    rng = np.random.default_rng(52)
    V = torch.tensor(rng.uniform(-1.0, 1.0, n), device="cuda", requires_grad=True)
    Xc = rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4))
    X = torch.tensor(Xc, dtype=torch.complex128, device="cuda", requires_grad=True)
    W = torch.tensor(rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4)),
                     dtype=torch.complex128, device="cuda")
    _hx_loss(ag, m, X, V, W, fe.FE_F64).backward()
    with torch.no_grad():
        dV = torch.tensor(rng.standard_normal(n), device="cuda")
        dX = torch.tensor(rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4)),
                          dtype=torch.complex128, device="cuda")
        fd_v = (_hx_loss(ag, m, X, V + H_FD * dV, W, fe.FE_F64)
                - _hx_loss(ag, m, X, V - H_FD * dV, W, fe.FE_F64)).item() / (2 * H_FD)
        fd_x = (_hx_loss(ag, m, X + H_FD * dX, V, W, fe.FE_F64)
                - _hx_loss(ag, m, X - H_FD * dX, V, W, fe.FE_F64)).item() / (2 * H_FD)
        an_v = float((V.grad * dV).sum())
        an_x = float((X.grad.conj() * dX).real.sum())
    assert abs(fd_v - an_v) <= 1e-6 * abs(an_v)
    assert abs(fd_x - an_x) <= 1e-6 * abs(an_x)
    with pytest.raises(fe.FeError):   # the adjoint covers the collocated potential only
        mq = fe.Mesh(L, nc, p)
        mq.set_potential_quad(torch.zeros(mq.n_cells * (p + 1) ** 3, dtype=torch.float64,
                                          device="cuda"))
        Xq = torch.zeros((mq.n_psi, 2), dtype=torch.float64, device="cuda")
        mq.potential_vjp(Xq, Xq)

"""Analysis outputs on the GPU against the oracle: planar integrals and averages of phi-node
fields, the dipole moment, V_bare on phi nodes, and the polarisability from two
self-consistent runs at different fields (same protocol on both sides).

Tolerances: 1e-12 relative for the reductions (same sums, different order); the
polarisability 1e-6 relative (two self-consistent runs per side, each within ~1e-8)."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import analysis, assembly, poisson, potentials, scf
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


@pytest.mark.parametrize("kind", ["cef", "cpd"])
def test_planar_dipole_vbare_match_oracle(fe, kind):
    bias = W.Bias("cef", field=0.02) if kind == "cef" else W.Bias("cpd", dV=0.03, zA=1.5, zB=12.5)
    base = W.small_slab(ncell=(3, 2, 6), p=3, L=(6.0, 4.0, 14.0), natoms=3, seed=11)
    slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
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
        mask, vals, _, _ = potentials.cpd_constraints(X, vl, bias, slab.L)
        phi = poisson.solve_cpd_direct(K, f, mask, vals)
        vapp = 0.0 * X[:, 2]
    vbare = phi + vl + vapp
    m = fe.Mesh.from_slab(slab)
    phig, _, _ = m.poisson_solve(bias, rtol=1e-13)
    vb = m.vbare_phi(phig, bias).cpu().numpy()
    assert np.max(np.abs(vb - vbare)) <= 1e-9 * np.max(np.abs(vbare))
    vbt = torch.tensor(vbare, device="cuda")
    rhot = torch.tensor(rho, device="cuda")
    np.testing.assert_allclose(m.planar(rhot).cpu().numpy(), analysis.planar_integral(om, M, rho),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m.planar(vbt, average=True).cpu().numpy(),
                               analysis.planar_average(om, M, vbare), rtol=1e-12, atol=1e-14)
    mu_ref = analysis.dipole_z(M, rho, b, X[:, 2], slab.L[2])
    assert abs(m.dipole() - mu_ref) <= 1e-12 * max(1.0, abs(mu_ref))
    assert abs(m.dipole(rhot) - mu_ref) <= 1e-12 * max(1.0, abs(mu_ref))


def test_polarisability_from_two_scf_runs(fe):
    from paper_2504_00998_gb300 import scf as fscf
    base = W.small_slab(ncell=(2, 2, 6), p=3, L=(4.0, 4.0, 14.0), natoms=4, seed=3, nvec=16,
                        degree=8)
    fields = (-0.005, 0.005)
    mu_gpu, mu_ref = [], []
    for E in fields:
        bias = W.Bias("cef", field=E)
        slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias, nvec=16,
                      degree=8, seed=base.seed)
        X0 = W.start_block(slab).astype(np.float64)
        ref = scf.scf_run(slab, X0, iters=8)
        om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
        Xc = om.phi_coords()
        _, b = potentials.densities(Xc, ref["M"], slab.R, slab.Z, slab.L)
        mu_ref.append(analysis.dipole_z(ref["M"], ref["rho"], b, Xc[:, 2], slab.L[2]))
        m = fe.Mesh.from_slab(slab)
        out = fscf.scf_run(m, bias, float(np.sum(slab.Z)), torch.tensor(X0, device="cuda"),
                           iters=8, degree=8, prec=fe.FE_F64)
        mu_gpu.append(m.dipole(out["rho"]))
    a_ref = analysis.polarisability(mu_ref[0], mu_ref[1], *fields)
    a_gpu = analysis.polarisability(mu_gpu[0], mu_gpu[1], *fields)
    assert a_ref > 0.0
    assert abs(a_gpu - a_ref) <= 1e-6 * abs(a_ref)

"""GPU parity of the Poisson operator, load vector, atom fields and the CEF / CPD / L-CPD
solves against the FP64 CPU oracle, plus closed forms run on the GPU.

Tolerances: operator and fields <= 1e-12 relative (same arithmetic, different order);
solves to relative residual 1e-12 on both sides, compared at 1e-9 relative (the residual
bound times the operator's condition number on these meshes stays below that).
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import assembly, poisson, potentials
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _oracle(slab):
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    X = om.phi_coords()
    return om, K, M, X


@pytest.mark.parametrize("L,ncell,p", [((4.0, 4.0, 9.0), (2, 2, 4), 3), ((3.0, 5.0, 7.0), (3, 1, 3), 2),
                                       ((6.0, 6.0, 6.0), (2, 2, 2), 6), ((2.0, 2.0, 4.0), (1, 1, 2), 1),
                                       ((12.0, 12.0, 20.0), (6, 6, 10), 4)])
def test_apply_K_matches_oracle(fe, L, ncell, p):
    om = OMesh(L, ncell, p)
    K = assembly.assemble_stiffness(om)
    m = fe.Mesh(L, ncell, p)
    x = np.random.default_rng(0).standard_normal(om.n_phi)
    y = m.poisson_apply_K(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = K @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-12
    M = assembly.lumped_mass(om)
    np.testing.assert_allclose(m.lumped_mass().cpu().numpy(), M, rtol=1e-14)
    np.testing.assert_allclose(m.node_coords().cpu().numpy(), om.phi_coords(), atol=1e-13)


@pytest.mark.parametrize("L,ncell,p", [((4.0, 4.0, 9.0), (2, 2, 4), 3), ((3.0, 5.0, 7.0), (3, 1, 3), 2),
                                       ((6.0, 6.0, 6.0), (2, 2, 2), 6), ((2.0, 2.0, 4.0), (1, 1, 2), 1),
                                       ((18.0, 4.0, 6.0), (9, 2, 3), 5), ((34.0, 2.0, 4.0), (17, 1, 2), 3),
                                       ((10.0, 6.0, 8.0), (5, 3, 4), 6), ((70.0, 2.0, 4.0), (35, 1, 2), 1),
                                       ((12.0, 12.0, 20.0), (6, 6, 10), 4)])
def test_apply_K_f32_matches_oracle(fe, L, ncell, p):
    """Float K x through the cell-local products (strips of 4 to 32 cells along x, so these
    meshes include partial strips and one-cell periodic directions):
    against the oracle's assembled K on the float-rounded input, 1e-5 relative (float
    accumulation of at most 8 cell contributions of (p+1)-term products); two calls agree
    bit for bit; the float entry rejects aliased arrays."""
    om = OMesh(L, ncell, p)
    K = assembly.assemble_stiffness(om)
    m = fe.Mesh(L, ncell, p)
    x = np.random.default_rng(1).standard_normal(om.n_phi).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    y1 = m.poisson_apply_K(xt)
    y2 = m.poisson_apply_K(xt)
    assert torch.equal(y1, y2)
    ref = K @ x.astype(np.float64)
    got = y1.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    with pytest.raises(fe.FeError):
        fe._lib.call("fe_poisson_apply_K_f32", m.handle, fe._ptr(xt), fe._ptr(xt))


def test_fields_and_load_match_oracle(fe):
    slab = W.small_slab(ncell=(3, 2, 4), p=3, L=(6.0, 4.0, 12.0), natoms=4, seed=11)
    om, K, M, X = _oracle(slab)
    m = fe.Mesh.from_slab(slab)
    f, rho, b = m.poisson_rhs()
    rho_r, b_r = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    np.testing.assert_allclose(rho.cpu().numpy(), rho_r, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b.cpu().numpy(), b_r, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f.cpu().numpy(), 4 * math.pi * M * (rho_r + b_r), rtol=1e-11,
                               atol=1e-14)


@pytest.mark.parametrize("kind", ["cef", "cpd", "lcpd"])
def test_solve_matches_oracle(fe, kind):
    base = W.small_slab(ncell=(3, 3, 6), p=3, L=(6.0, 6.0, 14.0), natoms=3, seed=5)
    bias = {"cef": W.Bias("cef", field=0.02),
            "cpd": W.Bias("cpd", dV=0.03, zA=1.5, zB=12.5),
            "lcpd": W.Bias("cpd", dV=0.03, zA=1.5, zB=12.5, patch=((1.0, 2.0), (4.0, 5.0)))}[kind]
    slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
    om, K, M, X = _oracle(slab)
    rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
    f = 4 * math.pi * M * (rho + b)
    if kind == "cef":
        ref = poisson.solve_cef_direct(K, f, M)
        vapp = potentials.v_app(X[:, 2], bias.field, slab.L[2])
    else:
        mask, vals, om0, om1 = potentials.cpd_constraints(X, vl, bias, slab.L)
        ref = poisson.solve_cpd_direct(K, f, mask, vals)
        vapp = 0.0 * X[:, 2]
    m = fe.Mesh.from_slab(slab)
    phi, vbare, info = m.poisson_solve(bias, rtol=1e-12)
    assert info.status == 0 and info.rel_residual <= 1e-12 and info.iters > 3
    phi = phi.cpu().numpy()
    assert np.max(np.abs(phi - ref)) <= 1e-9 * np.max(np.abs(ref))
    ids = om.psi_to_phi()
    vb_ref = (ref + vl + vapp)[ids]
    assert np.max(np.abs(vbare.cpu().numpy() - vb_ref)) <= 1e-9 * np.max(np.abs(vb_ref))
    if kind == "cef":
        assert abs(M @ phi) <= 1e-10 * np.sum(M) * np.max(np.abs(phi))
    else:
        np.testing.assert_allclose((phi + vl)[om0], 0.0, atol=1e-13)
        np.testing.assert_allclose((phi + vl)[om1], bias.dV, atol=1e-13)


def test_patch_polynomial_and_capacitor_on_gpu(fe):
    """No atoms: rho = -P''/(4 pi) with Dirichlet planes z = 0, Lz reproduces P exactly; with
    rho = 0 the CPD potential is the linear capacitor profile."""
    L, ncell, p = (3.0, 3.0, 8.0), (2, 2, 4), 4
    om = OMesh(L, ncell, p)
    X = om.phi_coords()
    z = X[:, 2]
    m = fe.Mesh(L, ncell, p)
    m.set_atoms(np.zeros((0, 3)), np.zeros(0))
    P = np.polynomial.Polynomial([0.0, 0.4, -0.3, 0.05, 0.01])  # degree p, P(0) = 0
    rho = torch.tensor(-P.deriv(2)(z) / (4 * math.pi), device="cuda")
    bias = W.Bias("cpd", dV=float(P(L[2])), zA=0.0, zB=L[2])
    phi, _, info = m.poisson_solve(bias, rho=rho, rtol=1e-13)
    np.testing.assert_allclose(phi.cpu().numpy(), P(z), atol=1e-10)
    bias = W.Bias("cpd", dV=0.25, zA=2.0, zB=6.0)
    phi, _, info = m.poisson_solve(bias, rho=torch.zeros(om.n_phi, dtype=torch.float64, device="cuda"),
                                   rtol=1e-13)
    np.testing.assert_allclose(phi.cpu().numpy(), np.clip((z - 2.0) / 4.0, 0, 1) * 0.25, atol=1e-11)


def test_iteration_cap_reports_noconv(fe):
    slab = W.small_slab(ncell=(2, 2, 4), p=3, L=(4.0, 4.0, 9.0), natoms=2)
    m = fe.Mesh.from_slab(slab)
    with pytest.raises(fe.FeError) as e:
        m.poisson_solve(slab.bias, rtol=1e-14, max_iter=3)
    assert e.value.status == fe._lib.FE_ENOCONV
    # the mesh stays usable afterwards
    phi, _, info = m.poisson_solve(slab.bias, rtol=1e-10)
    assert info.status == 0


@pytest.mark.parametrize("kind", ["cef", "cpd", "lcpd"])
def test_plane_coarse_space_same_solution_fewer_iterations(fe, kind):
    """The z-plane coarse correction changes only the iteration count: on a long slab
    (4 x 4 x 48 bohr, p = 4) both preconditioners reach the oracle's solution, and the
    two-level one needs clearly fewer iterations."""
    base = W.small_slab(ncell=(2, 2, 24), p=4, L=(4.0, 4.0, 48.0), natoms=4, seed=13)
    bias = {"cef": W.Bias("cef", field=0.01),
            "cpd": W.Bias("cpd", dV=0.05, zA=2.0, zB=46.0),
            "lcpd": W.Bias("cpd", dV=0.05, zA=2.0, zB=46.0, patch=((1.0, 1.0), (3.0, 3.0)))}[kind]
    slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
    om, K, M, X = _oracle(slab)
    rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    f = 4 * math.pi * M * (rho + b)
    if kind == "cef":
        ref = poisson.solve_cef_direct(K, f, M)
    else:
        vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
        mask, vals, _, _ = potentials.cpd_constraints(X, vl, bias, slab.L)
        ref = poisson.solve_cpd_direct(K, f, mask, vals)
    m = fe.Mesh.from_slab(slab)
    iters = {}
    for planes in (False, True):
        m.set_poisson_precond(planes)
        phi, _, info = m.poisson_solve(bias, rtol=1e-12)
        assert info.status == 0 and info.rel_residual <= 1e-12
        assert np.max(np.abs(phi.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))
        iters[planes] = info.iters
    assert iters[True] < 0.7 * iters[False], iters


@pytest.mark.parametrize("kind", ["cef", "lcpd"])
@pytest.mark.parametrize("layout", ["planes4", "odd_planes", "jacobi_only"])
def test_mixed_refinement_matches_double_cg(fe, kind, layout):
    """Float corrections refined against the double residual reach the double CG's
    solution: same stopping test, solutions within the residual bound times the
    conditioning (1e-9 relative).  Three float iterations are covered: the fused one (planes of
    a multiple of four nodes, plane coarse space), the scalar one (81-node planes) and the
    four-node one without the coarse space (Jacobi only)."""
    p = 3 if layout == "odd_planes" else 4
    base = W.small_slab(ncell=(3, 3, 12), p=p, L=(6.0, 6.0, 24.0), natoms=5, seed=17)
    bias = {"cef": W.Bias("cef", field=0.01),
            "lcpd": W.Bias("cpd", dV=0.05, zA=2.0, zB=22.0, patch=((1.0, 1.0), (4.0, 5.0)))}[kind]
    slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
    m = fe.Mesh.from_slab(slab)
    if layout == "jacobi_only":
        m.set_poisson_precond(False)
    out = {}
    for mixed in (False, True):
        m.set_poisson_mixed(mixed)
        phi, vb, info = m.poisson_solve(bias, rtol=1e-12)
        assert info.status == 0 and info.rel_residual <= 1e-12
        out[mixed] = phi.cpu().numpy()
    ref = out[False]
    assert np.max(np.abs(out[True] - ref)) <= 1e-9 * np.max(np.abs(ref))


def _bias_for(kind, L):
    Lz = L[2]
    return {"cef": W.Bias("cef", field=0.01),
            "cpd": W.Bias("cpd", dV=0.05, zA=2.0, zB=Lz - 2.0),
            "lcpd": W.Bias("cpd", dV=0.05, zA=2.0, zB=Lz - 2.0,
                           patch=((1.0, 1.0), (0.6 * L[0], 0.7 * L[1])))}[kind]


@pytest.mark.parametrize("kind,p,ncell", [("cef", 4, (3, 3, 12)), ("cpd", 2, (4, 4, 10)),
                                          ("lcpd", 5, (2, 2, 8)), ("cef", 6, (2, 2, 6)),
                                          ("lcpd", 1, (4, 4, 16)), ("cef", 3, (4, 4, 10))])
def test_persistent_cg_matches_launch_per_step(fe, kind, p, ncell):
    """The float CG run as one cooperative kernel per reliable-update interval reaches the
    oracle's solution like the launch-per-step iteration, in about as many iterations
    (the dot products are summed in another order) and with far fewer launches.  p = 1..6,
    the three bias setups, phi planes of 16 to 400 nodes."""
    L = (6.0, 6.0, 24.0)
    base = W.small_slab(ncell=ncell, p=p, L=L, natoms=4, seed=21)
    bias = _bias_for(kind, L)
    slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
    om, K, M, X = _oracle(slab)
    rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    f = 4 * math.pi * M * (rho + b)
    if kind == "cef":
        ref = poisson.solve_cef_direct(K, f, M)
    else:
        vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
        mask, vals, _, _ = potentials.cpd_constraints(X, vl, bias, slab.L)
        ref = poisson.solve_cpd_direct(K, f, mask, vals)
    lib = fe.load()
    m = fe.Mesh.from_slab(slab)
    m.set_poisson_precond(True)   # the plane coarse space on both paths
    out = {}
    for persistent in (False, True):
        m.set_poisson_persistent(persistent)
        n0 = lib.fe_kernel_launches()
        phi, _, info = m.poisson_solve(bias, rtol=1e-12)
        launches = lib.fe_kernel_launches() - n0
        assert info.status == 0 and info.rel_residual <= 1e-12
        phi = phi.cpu().numpy()
        assert np.max(np.abs(phi - ref)) <= 1e-9 * np.max(np.abs(ref))
        out[persistent] = (phi, info.iters, launches)
    it_l, it_p = out[False][1], out[True][1]
    assert abs(it_p - it_l) <= 0.1 * it_l + 3, (it_l, it_p)
    assert out[True][2] < out[False][2] / 3, (out[False][2], out[True][2])


def test_persistent_cg_bounded_wait_reports_timeout(fe):
    """One block of the cooperative CG kernel leaves before its first grid barrier (the test
    aid FE_OPT_TEST_CG_STALL): no barrier can complete, the other blocks' waits run out
    after 2 s, and the solve returns FE_ETIMEOUT instead of hanging; the mesh then solves
    normally."""
    import time
    slab = W.small_slab(ncell=(2, 2, 8), p=4, L=(4.0, 4.0, 16.0), natoms=2, seed=3)
    m = fe.Mesh.from_slab(slab)
    fe.call("fe_set_option", m._h, fe._lib.FE_OPT_TEST_CG_STALL, 1)
    t0 = time.time()
    with pytest.raises(fe.FeError) as e:
        m.poisson_solve(slab.bias, rtol=1e-12)
    assert e.value.status == fe._lib.FE_ETIMEOUT
    assert time.time() - t0 < 60
    fe.call("fe_set_option", m._h, fe._lib.FE_OPT_TEST_CG_STALL, -1)
    phi, _, info = m.poisson_solve(slab.bias, rtol=1e-12)
    assert info.status == 0 and info.rel_residual <= 1e-12
    m.set_poisson_persistent(False)
    phi_l, _, _ = m.poisson_solve(slab.bias, rtol=1e-12)
    ref = phi_l.cpu().numpy()
    assert np.max(np.abs(phi.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("p,ncell,L", [(2, (8, 8, 24), (16.0, 16.0, 48.0)),
                                       (3, (8, 12, 12), (16.0, 24.0, 24.0)),
                                       (4, (4, 4, 24), (8.0, 8.0, 48.0))])
def test_mode_coarse_space(fe, p, ncell, L):
    """The plane coarse space enriched with the in-plane modes of wavenumber one: on a CEF
    slab of at least 8 x 8 cells (no constrained phi nodes) the persistent float iteration
    reaches the oracle's solution in clearly fewer iterations than with the plane space
    alone; on a narrower slab, and with constrained nodes (L-CPD), the option acts as the
    plane space (the same iteration count)."""
    base = W.small_slab(ncell=ncell, p=p, L=L, natoms=6, seed=31)
    wide = ncell[0] >= 8 and ncell[1] >= 8
    out = {}
    for kind in ("cef", "lcpd"):
        bias = _bias_for(kind, L)
        slab = W.Slab(base.name, base.L, base.ncell, base.p, base.R, base.Z, bias)
        om, K, M, X = _oracle(slab)
        rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
        f = 4 * math.pi * M * (rho + b)
        if kind == "cef":
            ref = poisson.solve_cef_direct(K, f, M)
        else:
            vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
            mask, vals, _, _ = potentials.cpd_constraints(X, vl, bias, slab.L)
            ref = poisson.solve_cpd_direct(K, f, mask, vals)
        m = fe.Mesh.from_slab(slab)
        for modes in (False, True):
            m.set_poisson_precond(True, modes=modes)
            phi, _, info = m.poisson_solve(bias, rtol=1e-12)
            assert info.status == 0 and info.rel_residual <= 1e-12
            assert np.max(np.abs(phi.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))
            out[(kind, modes)] = info.iters
    if wide:
        assert out[("cef", True)] < 0.9 * out[("cef", False)], out
    else:
        assert out[("cef", True)] == out[("cef", False)], out
    assert out[("lcpd", True)] == out[("lcpd", False)], out

"""Workload-size parity: the constant-field slab end to end (12x12x36 bohr, p = 3, 32
vectors, degree 10) against the oracle, and the p = 5 slab of 1.53 M psi nodes with 512
vectors (the benchmark workload, same entry points and launch configuration) on sampled
rows that the oracle evaluates one by one from the cell definition.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from entrywise import assert_operator_entries
from oracle import assembly, chefsi, poisson, potentials
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu

R_FILTER = 0.03   # filter cut a = a0 + 0.03 (b - a0)


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def test_cef_slab_end_to_end(fe):
    slab = W.config1()
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    X = om.phi_coords()
    rho, b = potentials.densities(X, M, slab.R, slab.Z, slab.L)
    vl = potentials.vloc_minus_vsm(X, slab.R, slab.Z, slab.L)
    phi_ref = poisson.solve_cef_direct(K, 4 * math.pi * M * (rho + b), M)
    ids = om.psi_to_phi()
    V = (phi_ref + vl + potentials.v_app(X[:, 2], slab.bias.field, slab.L[2]))[ids]
    H = assembly.hamiltonian(om, V, K, M)

    m = fe.Mesh.from_slab(slab)
    phi, vbare, info = m.poisson_solve(slab.bias, rtol=1e-12)
    assert info.status == 0
    assert np.max(np.abs(phi.cpu().numpy() - phi_ref)) <= 1e-9 * np.max(np.abs(phi_ref))
    assert np.max(np.abs(vbare.cpu().numpy() - V)) <= 1e-9 * np.max(np.abs(V))
    m.set_potential(torch.tensor(V, device="cuda"))

    v0 = W.lanczos_start(om.n_psi)
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, v0, 20)
    glo, ghi = m.lanczos_bounds(torch.tensor(v0, device="cuda"), 20)
    assert abs(glo - lo) <= 1e-8 * hi and abs(ghi - hi) <= 1e-8 * hi
    a = lo + R_FILTER * (hi - lo)
    X0 = W.start_block(slab).astype(np.float64)
    ev_ref, _ = chefsi.chefsi_cycle(lambda Z: H @ Z, X0, slab.degree, a, hi, lo)
    Xg = torch.tensor(X0, device="cuda")
    m.cheb_filter(Xg, slab.degree, a, hi, lo)
    ev = m.rayleigh_ritz(Xg).cpu().numpy()
    assert np.max(np.abs(ev - ev_ref)) <= 1e-8
    # the mixed (float storage, float products) path on the same cycle
    Xf = torch.tensor(X0, dtype=torch.float32, device="cuda")
    m.cheb_filter(Xf, slab.degree, a, hi, lo, prec=fe.FE_F32)
    evf = m.rayleigh_ritz(Xf, prec=fe.FE_F32).cpu().numpy()
    k = min(int(slab.n_electrons // 2), slab.nvec - 8)
    assert np.max(np.abs(evf[:k] - ev_ref[:k])) <= 1e-5
    # the tensor-core filter (bf16 operands, fp32 accumulation) with the same float
    # Rayleigh-Ritz: its one rounding of the cell matrix K_e moves the filtered subspace at
    # first order, so the Ritz values miss the 1e-5 Ha criterion by three orders of
    # magnitude (measured on GB300: 1.24e-2 Ha; the gap is asserted, not hidden)
    Xb = torch.tensor(X0, dtype=torch.float32, device="cuda")
    m.cheb_filter(Xb, slab.degree, a, hi, lo, prec=fe.FE_BF16_F32ACC)
    evb = m.rayleigh_ritz(Xb, prec=fe.FE_BF16_F32ACC).cpu().numpy()
    err_bf16 = np.max(np.abs(evb[:k] - ev_ref[:k]))
    print(f"config 1 Ritz error: float {np.max(np.abs(evf[:k] - ev_ref[:k])):.3e}, "
          f"bf16 tensor-core filter {err_bf16:.3e} Ha")
    assert err_bf16 <= 3e-2


def test_p5_slab_sampled_rows(fe):
    slab = W.config2()
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    rng = np.random.default_rng(77)
    V = rng.uniform(-1.5, 0.5, om.n_psi)
    X0 = W.start_block(slab)
    m = fe.Mesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    m.set_potential(torch.tensor(V, device="cuda"))
    nxy = om.NX * om.NY
    # rows on the periodic seams, the Dirichlet-adjacent planes, cell faces and interiors
    rows = np.unique(np.concatenate([
        [0, om.NX - 1, nxy - 1, nxy, om.n_psi - 1, om.n_psi - nxy, 5 * om.NX + 5,
         (om.NZpsi // 2) * nxy + 3 * om.NX + 7], rng.choice(om.n_psi, 40, replace=False)]))
    Ke = assembly.reference_cell_stiffness(om)
    M = assembly.lumped_mass(om)
    ref = assembly.apply_H_rows(om, V, X0, rows, Ke=Ke, M=M)
    # entry bound: the magnitudes of the terms, sum_e |K_e| |S X| and |V| |X|, row by row
    mag = assembly.apply_H_rows(om, np.abs(V), np.abs(X0), rows, Ke=np.abs(Ke), M=M)
    for prec, tol, etol in ((fe.FE_F64, 1e-10, 1e-13), (fe.FE_F32, 2e-5, 1e-6),
                            (fe.FE_F32_F32ACC, 2e-5, 4e-6)):
        Xg = torch.tensor(X0, dtype=fe.storage_dtype(prec), device="cuda")
        Y = m.apply_H(Xg, prec=prec)
        got = Y[torch.tensor(rows, device="cuda")].double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, prec
        assert_operator_entries(got, ref, mag, etol, f"p = 5 slab rows, precision {prec}")
        del Xg, Y
        torch.cuda.empty_cache()


def test_p5_slab_mixed_eigenvalues_vs_fp64(fe):
    """The benchmark's accuracy criterion as a test: on the p = 5 slab (1.53 M psi nodes,
    512 vectors, degree 30), two filter + Rayleigh-Ritz cycles from the same start block in
    the float path (FP32 operator, FP32-accurate tensor-core block products, double n x n
    part) and in FP64 agree to 1e-5 Ha over the lowest 384 Ritz values; the bf16
    tensor-core filter's gap is measured and bounded."""
    slab = W.config2()
    m = fe.Mesh.from_slab(slab)
    _, vb, info = m.poisson_solve(slab.bias, rtol=1e-10)
    assert info.status == 0
    m.set_potential(vb)
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device="cuda"), 20)
    a = lo + R_FILTER * (hi - lo)
    X0 = torch.from_numpy(W.start_block(slab))
    k = min(int(slab.n_electrons // 2), slab.nvec - 8)
    ev = {}
    for prec, tc in ((fe.FE_F64, False), (fe.FE_F32, True), (fe.FE_F32_F32ACC, True),
                     (fe.FE_BF16_F32ACC, True)):
        m.set_rr_products(tc)
        X = X0.to("cuda", fe.storage_dtype(prec))
        for _ in range(2):
            m.cheb_filter(X, slab.degree, a, hi, lo, prec=prec)
            e = m.rayleigh_ritz(X, prec=prec)
        ev[prec] = e.cpu().numpy()
        del X
        torch.cuda.empty_cache()
    err32 = np.max(np.abs(ev[fe.FE_F32][:k] - ev[fe.FE_F64][:k]))
    errbf = np.max(np.abs(ev[fe.FE_BF16_F32ACC][:k] - ev[fe.FE_F64][:k]))
    errtc = np.max(np.abs(ev[fe.FE_F32_F32ACC][:k] - ev[fe.FE_F64][:k]))
    print(f"p = 5 slab, lowest {k} Ritz values vs FP64: float {err32:.3e}, split-TF32 "
          f"tensor cores {errtc:.3e}, bf16 {errbf:.3e} Ha")
    assert err32 <= 1e-5 and errtc <= 1e-5
    assert errbf <= 1e-2


def test_large_lcpd_slab_poisson_and_blocked_filter(fe):
    """The 48 x 48 x 144 bohr L-CPD slab (24 x 24 x 72 cells, p = 5, 5,198,400 phi nodes,
    2048 atoms with Z in {1, 3, 4, 5}): the potential satisfies the constraints exactly and
    the FE equations at sampled free rows (evaluated one by one from the cell definition);
    the filter runs on one 256-vector block of a 1024-wide array and H X matches the oracle
    at sampled rows."""
    slab = W.config5()
    m = fe.Mesh.from_slab(slab)
    phi, vbare, info = m.poisson_solve(slab.bias, rtol=1e-10, max_iter=40000)
    assert info.status == 0 and info.rel_residual <= 1e-10
    mask, vals = m.poisson_constraints(slab.bias)
    ph = phi.cpu().numpy()
    mk = mask.cpu().numpy()
    assert np.array_equal(ph[mk], vals.cpu().numpy()[mk])
    # constrained patch: Omega_1 is restricted to the 12 x 12 bohr patch
    X = m.node_coords().cpu().numpy()
    top = X[:, 2] >= slab.bias.zB - 1e-12
    assert 0 < np.sum(mk & top) < np.sum(top)
    # FE equations K phi = 4 pi M (rho + b) at sampled free rows, from the oracle's cells
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    f, _, _ = m.poisson_rhs()
    f = f.cpu().numpy()
    Ke = assembly.reference_cell_stiffness(om)
    cn = om.cell_nodes()
    rng = np.random.default_rng(9)
    free = np.flatnonzero(~mk)
    rows = rng.choice(free, 30, replace=False)
    for I in rows:
        gx, gy, gz = I % om.NX, (I // om.NX) % om.NY, I // (om.NX * om.NY)
        kphi = sum(Ke[loc] @ ph[cn[cell]] for cell, loc in om.node_cells(gx, gy, gz))
        assert abs(kphi - f[I]) <= 1e-7 * (np.abs(Ke).max() * np.abs(ph).max() + abs(f[I]))
    # one 256-vector block of a 1024-wide float array
    m.set_potential(vbare)
    Xall = torch.zeros((m.n_psi, 1024), dtype=torch.float32, device="cuda")
    blk = Xall[:, 256:512]
    X0 = W.start_block(slab, nvec=256)
    blk.copy_(torch.from_numpy(X0))
    Y = torch.zeros_like(Xall)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(blk), fe._ptr(Y[:, 256:512]), 256, 1024, fe.FE_F32)
    V = vbare.cpu().numpy()
    M = assembly.lumped_mass(om)
    rows = np.concatenate([[0, om.NX * om.NY, m.n_psi - 1], rng.choice(m.n_psi, 20, replace=False)])
    ref = assembly.apply_H_rows(om, V, X0, rows, Ke=Ke, M=M)
    got = Y[torch.tensor(rows, device="cuda"), 256:512].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5
    mag = assembly.apply_H_rows(om, np.abs(V), np.abs(X0), rows, Ke=np.abs(Ke), M=M)
    assert_operator_entries(got, ref, mag, 1e-6, "large slab rows")
    assert torch.all(Y[:, :256] == 0) and torch.all(Y[:, 512:] == 0)
    del Y
    torch.cuda.empty_cache()

    # one full CheFSI cycle of the configuration: the 1024-wide array filtered in four
    # 256-vector blocks at degree 40, then Rayleigh-Ritz over all 1024 vectors
    m.set_rr_products(True)
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device="cuda"), 20)
    a = lo + R_FILTER * (hi - lo)
    for blk in range(4):
        Xall[:, 256 * blk:256 * (blk + 1)].copy_(
            torch.from_numpy(W.start_block(slab, nvec=256, seed=2005 + blk)))
        m.cheb_filter(Xall[:, 256 * blk:256 * (blk + 1)], slab.degree, a, hi, lo,
                      prec=fe.FE_F32)
    theta = m.rayleigh_ritz(Xall, prec=fe.FE_F32).cpu().numpy()
    # ascending, and inside the Lanczos upper bound of the spectrum (the smallest Lanczos
    # Ritz value bounds the lowest eigenvalue from above, so it bounds nothing here)
    assert np.all(np.diff(theta) >= 0) and theta[-1] <= hi
    # what Rayleigh-Ritz guarantees at any size, on sampled columns (block edges included):
    # X^T X = I and X^T Ht X = diag(theta), in double from the float block
    edges = [0, 255, 256, 511, 512, 767, 768, 1023]
    rest = np.setdiff1d(np.arange(1024), edges)
    cols = np.sort(np.concatenate([edges, rng.choice(rest, 24, replace=False)]))   # 32 columns
    ct = torch.tensor(cols, device="cuda")
    Xs = Xall[:, ct].contiguous()
    HXs = m.apply_H(Xs, prec=fe.FE_F32)
    Xd = Xs.double()
    G = (Xd.T @ Xd).cpu().numpy()
    Hs = (Xd.T @ HXs.double()).cpu().numpy()
    assert np.max(np.abs(G - np.eye(len(cols)))) <= 1e-4
    scale = max(1.0, float(np.max(np.abs(theta))))
    assert np.max(np.abs(Hs - np.diag(theta[cols]))) <= 1e-4 * scale

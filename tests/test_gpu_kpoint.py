"""Bloch k-point operator on the GPU (fe_set_kpoint) against the oracle's Ht_k
(oracle/kpoint.py): Ht_k X on complex blocks (FP64 1e-10, FP32 2e-5 relative, as for the
Gamma-point operator), Lanczos bounds that enclose the spectrum, the complex Chebyshev filter,
the Hermitian Rayleigh-Ritz (Ritz values 1e-9), subspace iteration converging to the dense
spectrum (including the free-electron ground state 1/2 |k|^2), the density of complex
orbitals, the refused combinations, and the return to the Gamma point."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import assembly, chefsi, kpoint
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


CASES = [
    # (L, ncell, p, psi Dirichlet faces, k)
    ((4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), (0.31, -0.17)),
    ((3.0, 5.0, 7.0), (3, 1, 3), 2, (False, True), (0.0, 0.45)),
    ((4.5, 3.0, 6.0), (2, 2, 3), 5, (False, False), (0.52, 0.23)),
    ((6.0, 6.0, 6.0), (2, 2, 2), 4, (True, True), (-0.4, 0.0)),
]


def _setup(fe, L, ncell, p, faces, k, seed=3, V=None):
    om = OMesh(L, ncell, p, faces)
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1.0, 0.5, om.n_psi) if V is None else V
    Hk = kpoint.hamiltonian_k(om, V, k)
    m = fe.Mesh(L, ncell, p, faces)
    m.set_potential(torch.tensor(V, device="cuda"))
    m.set_kpoint(*k)
    return om, Hk, m, rng, V


def _cblock(rng, n, nvec):
    return rng.standard_normal((n, nvec)) + 1j * rng.standard_normal((n, nvec))


@pytest.mark.parametrize("L,ncell,p,faces,k", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nvec", [1, 6, 16])
def test_apply_Hk_matches_oracle(fe, L, ncell, p, faces, k, prec, nvec):
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    X = _cblock(rng, om.n_psi, nvec)
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.complex128 if prec == "f64" else torch.complex64
    # rows are 16-byte multiples: complex64 blocks take an even leading dimension
    ld = nvec + (nvec % 2 if prec == "f32" else 0)
    buf = torch.zeros((om.n_psi, ld), dtype=dt, device="cuda")
    buf[:, :nvec] = torch.tensor(X, dtype=dt)
    Xg = buf[:, :nvec]
    ybuf = torch.zeros_like(buf)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(Xg), fe._ptr(ybuf), nvec, ld, P)
    Y = ybuf[:, :nvec].cpu().numpy()
    Xr = Xg.cpu().numpy().astype(np.complex128)
    ref = Hk @ Xr
    tol = 1e-10 if prec == "f64" else 2e-5
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= tol


def test_lanczos_bounds_enclose_the_spectrum(fe):
    L, ncell, p, faces, k = CASES[0]
    om, Hk, m, _, _ = _setup(fe, L, ncell, p, faces, k)
    ev = sla.eigvalsh(Hk.toarray())
    lo, hi = m.lanczos_bounds(torch.ones(om.n_psi, dtype=torch.float64, device="cuda"), 30)
    assert hi >= ev[-1] - 1e-9 * abs(ev[-1])
    assert lo >= ev[0] - 1e-9 and lo <= ev[0] + 0.05 * (ev[-1] - ev[0])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_complex_filter_matches_oracle(fe, prec, tol):
    L, ncell, p, faces, k = CASES[2]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    ev = sla.eigvalsh(Hk.toarray())
    a0, b = ev[0] - 0.1, ev[-1] + 0.1
    a = a0 + 0.2 * (b - a0)
    X = _cblock(rng, om.n_psi, 8)
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.complex128 if prec == "f64" else torch.complex64
    Xg = torch.tensor(X, dtype=dt, device="cuda")
    Xin = Xg.cpu().numpy().astype(np.complex128)
    m.cheb_filter(Xg, 7, a, b, a0, prec=P)
    ref = chefsi.cheb_filter(lambda Z: Hk @ Z, Xin, 7, a, b, a0)
    got = Xg.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


@pytest.mark.parametrize("prec,tc", [("f64", False), ("f32", False), ("f32", True)])
@pytest.mark.parametrize("nvec", [1, 10, 33])
def test_complex_rayleigh_ritz(fe, prec, tc, nvec):
    """Ritz values against the oracle's (orthonormal basis by QR, eigvalsh of Q^H Ht_k Q);
    the rotated block is orthonormal and its Rayleigh quotients are the Ritz values.  tc: the
    float block's products as real tensor-core GEMMs on its (re, im) lanes."""
    L, ncell, p, faces, k = CASES[0]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    m.set_rr_products(tc)
    X = _cblock(rng, om.n_psi, nvec)
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.complex128 if prec == "f64" else torch.complex64
    # rows are 16-byte multiples: complex64 blocks take an even leading dimension
    ld = nvec + (nvec % 2 if prec == "f32" else 0)
    buf = torch.zeros((om.n_psi, ld), dtype=dt, device="cuda")
    buf[:, :nvec] = torch.tensor(X, dtype=dt)
    Xg = buf[:, :nvec]
    Xin = Xg.cpu().numpy().astype(np.complex128)
    e = m.rayleigh_ritz(Xg, prec=P).cpu().numpy()
    Q, _ = np.linalg.qr(Xin)
    ref = sla.eigvalsh(Q.conj().T @ (Hk @ Q))
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(e - ref)) <= (1e-9 if prec == "f64" else 1e-5) * scale
    Xr = Xg.cpu().numpy().astype(np.complex128)
    G = Xr.conj().T @ Xr
    assert np.max(np.abs(G - np.eye(nvec))) <= (1e-10 if prec == "f64" else 1e-5)
    rq = np.real(np.einsum("ij,ij->j", Xr.conj(), Hk @ Xr))
    assert np.max(np.abs(rq - e)) <= (1e-9 if prec == "f64" else 1e-4) * scale


@pytest.mark.parametrize("prec,tc,tol", [("f64", False, 1e-8), ("f32", True, 2e-5)])
def test_subspace_iteration_converges_to_the_dense_spectrum(fe, prec, tc, tol):
    L, ncell, p, faces, k = CASES[1]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    m.set_rr_products(tc)
    ev = sla.eigvalsh(Hk.toarray())
    nvec, want = 12, 6
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.complex128 if prec == "f64" else torch.complex64
    X = torch.tensor(_cblock(rng, om.n_psi, nvec), dtype=dt, device="cuda")
    lo, hi = m.lanczos_bounds(torch.ones(om.n_psi, dtype=torch.float64, device="cuda"), 30)
    cut = lo + 0.1 * (hi - lo)
    for _ in range(25):
        m.cheb_filter(X, 10, cut, hi, lo, prec=P)
        e = m.rayleigh_ritz(X, prec=P).cpu().numpy()
        cut = float(e[-1])
    assert np.max(np.abs(e[:want] - ev[:want])) <= tol * max(1.0, abs(ev[want - 1]))


def test_tc_rayleigh_ritz_falls_back_on_an_ill_conditioned_block(fe):
    """Columns that are nearly dependent (cond of the scaled Gram matrix far above 1e8): the
    tensor-core Gram path declines and the double complex path gives the Ritz values of the
    span."""
    L, ncell, p, faces, k = CASES[0]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    m.set_rr_products(True)
    nvec = 6
    B = _cblock(rng, om.n_psi, nvec)
    B[:, 5] = B[:, 4] + 1e-5 * ((1.0 + 0.5j) * B[:, 3] + B[:, 5])
    Xg = torch.tensor(B, dtype=torch.complex64, device="cuda")
    Xin = Xg.cpu().numpy().astype(np.complex128)
    e = m.rayleigh_ritz(Xg, prec=fe.FE_F32).cpu().numpy()
    Q, _ = np.linalg.qr(Xin)
    ref = sla.eigvalsh(Q.conj().T @ (Hk @ Q))
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(e - ref)) <= 1e-5 * scale
    Xr = Xg.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(Xr.conj().T @ Xr - np.eye(nvec))) <= 1e-5


def test_free_electron_ground_state_on_gpu(fe):
    """V = 0, Neumann z faces: the lowest Ritz value reaches 1/2 |k|^2."""
    k = (0.37, -0.22)
    L, ncell, p = (4.0, 4.0, 5.0), (2, 2, 2), 4
    om = OMesh(L, ncell, p, (False, False))
    m = fe.Mesh(L, ncell, p, (False, False))
    m.set_potential(torch.zeros(om.n_psi, dtype=torch.float64, device="cuda"))
    m.set_kpoint(*k)
    rng = np.random.default_rng(5)
    X = torch.tensor(_cblock(rng, om.n_psi, 6), device="cuda")
    # (a random start: the constant is itself an eigenvector here and would end Lanczos)
    v0 = torch.tensor(rng.standard_normal(om.n_psi), device="cuda")
    lo, hi = m.lanczos_bounds(v0, 30)
    cut = lo + 0.1 * (hi - lo)
    for _ in range(20):
        m.cheb_filter(X, 10, cut, hi, lo, prec=fe.FE_F64)
        e = m.rayleigh_ritz(X, prec=fe.FE_F64).cpu().numpy()
        cut = float(e[-1])
    assert abs(e[0] - 0.5 * (k[0] ** 2 + k[1] ** 2)) <= 1e-10


def test_density_of_complex_orbitals(fe):
    from paper_2504_00998_gb300 import scf as fscf
    L, ncell, p, faces, k = CASES[0]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    nvec = 7
    X = _cblock(rng, om.n_psi, nvec)
    occ = rng.uniform(0.0, 2.0, nvec)
    M = assembly.lumped_mass(om)
    for prec, dt, tol in ((fe.FE_F64, torch.complex128, 1e-12), (fe.FE_F32, torch.complex64, 1e-6)):
        Xg = torch.tensor(X, dtype=dt, device="cuda")
        rho = fscf.density(m, Xg, occ, prec).cpu().numpy()
        Xr = Xg.cpu().numpy().astype(np.complex128)
        ref = np.zeros(om.n_phi)
        ref[om.psi_to_phi()] = (np.abs(Xr) ** 2) @ occ / M[om.psi_to_phi()]
        assert np.max(np.abs(rho - ref)) <= tol * np.max(np.abs(ref))


def test_refused_combinations_and_gamma_reset(fe):
    L, ncell, p, faces, k = CASES[0]
    om, Hk, m, rng, V = _setup(fe, L, ncell, p, faces, k)
    Xc = torch.tensor(_cblock(rng, om.n_psi, 4), device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(Xc), fe._ptr(torch.empty_like(Xc)), 4,
                     4, fe.FE_BF16_F32ACC)
    assert e.value.status == fe._lib.FE_EUNSUPPORTED
    with pytest.raises(fe.FeError):
        fe.Batch([m])
    with pytest.raises(fe.FeError) as e:
        fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(Xc), 4, 4, 5, 0.0, 1.0, -1.0,
                     fe.FE_F64)
    assert e.value.status == fe._lib.FE_EUNSUPPORTED
    m.set_nonlocal(np.array([[1.0, 1.0, 4.0]]), np.array([0.7]), np.array([[0.5, 0.1, 0.1, 0.1]]),
                   2.0)
    with pytest.raises(fe.FeError):
        m.apply_H(Xc)
    m.set_nonlocal(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4)), 2.0)
    # back to the Gamma point: the real operator on real blocks
    m.set_kpoint(0.0, 0.0)
    Xr = rng.standard_normal((om.n_psi, 4))
    Y = m.apply_H(torch.tensor(Xr, device="cuda")).cpu().numpy()
    ref = assembly.hamiltonian(om, V) @ Xr
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 1e-10


def test_full_size_sampled_rows(fe):
    """The benchmark slab (16 x 16 x 48 cells, p = 5) at k = (0.1, 0.05) with 256 complex
    float vectors (the block of the benchmark's k-point step): sampled rows of Ht_k X
    against the oracle's row-by-row form, including rows on the lowest and highest psi
    planes and on the periodic seams."""
    import workloads as W
    slab = W.config2()
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    m = fe.Mesh.from_slab(slab, with_atoms=False)
    rng = np.random.default_rng(8)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    m.set_potential(torch.tensor(V, device="cuda"))
    k = (0.1, 0.05)
    m.set_kpoint(*k)
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((om.n_psi, slab.nvec // 2), generator=gen, device="cuda",
                    dtype=torch.complex64)
    Y = m.apply_H(X, prec=fe.FE_F32)
    NX, NY = om.NX, om.NY
    plane = NX * NY
    rows = np.concatenate([[0, NX - 1, plane - 1, om.n_psi - 1, om.n_psi - plane],
                           rng.integers(0, om.n_psi, 11)])
    ref = kpoint.apply_Hk_rows(om, V, k, X.cpu().numpy(), rows)
    got = Y[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5

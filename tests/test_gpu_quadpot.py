"""GPU parity of the potential term integrated by Gauss quadrature (fe_set_potential_quad,
fe_interp_quad) against the oracle's consistent potential matrix (oracle/quadpot.py):
interpolation to the Gauss points, Ht_q X in FP64 / FP32 (the tolerances of the collocated
operator: 1e-10 and 2e-5 relative, Frobenius) on meshes that exercise every colour layout
(even, odd and single-cell periodic rows, both z parities, Dirichlet and Neumann faces,
p = 1..6, vector counts with ragged chunks), bitwise repeatability, the Chebyshev filter,
Lanczos bounds and subspace iteration to the dense spectrum, the Bloch k-point operator on
top, the tensor-core precision, sampled rows at the full benchmark size, and the return to the
collocated potential."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import workloads as W
from oracle import assembly, chefsi, kpoint, quadpot
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


CASES = [
    # (L, ncell, p, psi Dirichlet faces)
    ((4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True)),
    ((3.0, 5.0, 7.0), (3, 1, 3), 2, (False, True)),     # odd nx (three x classes), one y cell
    ((2.0, 2.0, 3.0), (1, 1, 2), 1, (False, False)),    # single-cell rows in x and y
    ((4.0, 4.0, 6.0), (2, 3, 3), 4, (True, False)),
    ((5.0, 5.0, 5.0), (5, 2, 1), 5, (True, True)),      # one z layer, five x cells
    ((6.0, 6.0, 6.0), (2, 2, 2), 6, (False, False)),
]


def _setup(fe, L, ncell, p, dirichlet, seed=0):
    om = OMesh(L, ncell, p, dirichlet)
    rng = np.random.default_rng(seed)
    Vq = rng.uniform(-1.0, 0.5, (om.n_cells, (p + 1) ** 3))
    H = quadpot.hamiltonian_quad(om, Vq)
    m = fe.Mesh(L, ncell, p, dirichlet)
    m.set_potential_quad(torch.tensor(Vq, device="cuda"))
    return om, H, m, rng, Vq


def _block(X, dt, ld):
    n, k = X.shape
    buf = torch.full((n, ld), 3.0, dtype=dt, device="cuda")
    buf[:, :k] = torch.tensor(X, dtype=dt)
    return buf


@pytest.mark.parametrize("L,ncell,p,dirichlet", CASES)
def test_interpolation_matches_oracle(fe, L, ncell, p, dirichlet):
    om = OMesh(L, ncell, p, dirichlet)
    m = fe.Mesh(L, ncell, p, dirichlet)
    f = np.random.default_rng(1).standard_normal(om.n_phi)
    got = m.interp_quad(torch.tensor(f, device="cuda")).cpu().numpy()
    ref = quadpot.interpolate_to_quad(om, f)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("L,ncell,p,dirichlet", CASES)
@pytest.mark.parametrize("prec,nvec,ld", [("f64", 1, 2), ("f64", 21, 22), ("f32", 5, 8),
                                          ("f32", 40, 44)])
def test_apply_Hq_matches_oracle(fe, L, ncell, p, dirichlet, prec, nvec, ld):
    om, H, m, rng, Vq = _setup(fe, L, ncell, p, dirichlet)
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.float64 if prec == "f64" else torch.float32
    X = rng.standard_normal((om.n_psi, nvec))
    xb = _block(X, dt, ld)
    yb = torch.full_like(xb, 3.0)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(xb), fe._ptr(yb), nvec, ld, P)
    ref = H @ xb[:, :nvec].double().cpu().numpy()
    got = yb[:, :nvec].double().cpu().numpy()
    tol = 1e-10 if prec == "f64" else 2e-5
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
    assert torch.all(yb[:, nvec:] == 3.0)      # padding lanes untouched


def test_apply_Hq_is_bitwise_repeatable(fe):
    om, H, m, rng, Vq = _setup(fe, *CASES[3])
    X = torch.tensor(rng.standard_normal((om.n_psi, 64)), dtype=torch.float32, device="cuda")
    Y1 = m.apply_H(X, prec=fe.FE_F32)
    Y2 = m.apply_H(X, prec=fe.FE_F32)
    assert torch.equal(Y1, Y2)


def test_quadrature_of_a_nodal_potential_tends_to_collocation(fe):
    """A smooth V given at nodes and interpolated to the Gauss points: the consistent and
    the collocated operators agree to discretisation accuracy (both are consistent
    discretisations of the same continuum operator), and each matches its oracle."""
    L, ncell, p, d = (4.0, 4.0, 6.0), (2, 2, 3), 5, (True, True)
    om = OMesh(L, ncell, p, d)
    xyz = om.phi_coords()
    Vphi = -np.exp(-((xyz[:, 2] - 3.0) ** 2)) * (1.0 + 0.3 * np.cos(2 * np.pi * xyz[:, 0] / 4.0))
    m = fe.Mesh(L, ncell, p, d)
    Vq = m.interp_quad(torch.tensor(Vphi, device="cuda"))
    m.set_potential_quad(Vq)
    lo, hi = m.lanczos_bounds(torch.ones(om.n_psi, dtype=torch.float64, device="cuda"), 40)
    Hq = quadpot.hamiltonian_quad(om, Vq.cpu().numpy())
    Hc = assembly.hamiltonian(om, Vphi[om.psi_to_phi()])
    eq = sla.eigh(Hq.toarray(), eigvals_only=True, subset_by_index=[0, 5])
    ec = sla.eigh(Hc.toarray(), eigvals_only=True, subset_by_index=[0, 5])
    assert np.max(np.abs(eq - ec)) <= 1e-3 * np.max(np.abs(ec))
    assert lo <= eq[0] + 0.05 * (hi - lo) and lo >= eq[0] - 1e-6


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_filter_matches_oracle(fe, prec, tol):
    om, H, m, rng, Vq = _setup(fe, *CASES[0])
    ev = sla.eigvalsh(H.toarray())
    a0, b = ev[0] - 0.1, ev[-1] + 0.1
    a = a0 + 0.2 * (b - a0)
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = torch.float64 if prec == "f64" else torch.float32
    Xg = torch.tensor(rng.standard_normal((om.n_psi, 12)), dtype=dt, device="cuda")
    Xin = Xg.double().cpu().numpy()
    m.cheb_filter(Xg, 7, a, b, a0, prec=P)
    ref = chefsi.cheb_filter(lambda Z: H @ Z, Xin, 7, a, b, a0)
    got = Xg.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


def test_subspace_iteration_converges_to_the_dense_spectrum(fe):
    om, H, m, rng, Vq = _setup(fe, *CASES[1])
    ev = sla.eigvalsh(H.toarray())
    hi_ev = ev[-1]
    lo, hi = m.lanczos_bounds(torch.ones(om.n_psi, dtype=torch.float64, device="cuda"), 30)
    assert hi >= hi_ev - 1e-9 * abs(hi_ev)
    X = torch.tensor(rng.standard_normal((om.n_psi, 12)), device="cuda")
    cut = lo + 0.1 * (hi - lo)
    for _ in range(25):
        m.cheb_filter(X, 10, cut, hi, lo, prec=fe.FE_F64)
        e = m.rayleigh_ritz(X, prec=fe.FE_F64).cpu().numpy()
        cut = float(e[-1])
    assert np.max(np.abs(e[:6] - ev[:6])) <= 1e-8 * max(1.0, abs(ev[5]))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bloch_operator_with_quadrature_potential(fe, prec):
    """Ht_k with the quadrature potential: the oracle's quadrature operator plus the Bloch
    terms (1/2 |k|^2 - i M^-1/2 k.G M^-1/2, from Ht_k - Ht_0 at zero potential)."""
    L, ncell, p, d = CASES[0]
    k = (0.31, -0.17)
    om, Hq, m, rng, Vq = _setup(fe, L, ncell, p, d)
    m.set_kpoint(*k)
    zero = np.zeros(om.n_psi)
    Hk = Hq + (kpoint.hamiltonian_k(om, zero, k) - assembly.hamiltonian(om, zero))
    nvec = 6
    X = rng.standard_normal((om.n_psi, nvec)) + 1j * rng.standard_normal((om.n_psi, nvec))
    dt = torch.complex128 if prec == "f64" else torch.complex64
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    Xg = torch.tensor(X, dtype=dt, device="cuda")
    Y = m.apply_H(Xg, prec=P).cpu().numpy()
    ref = Hk @ Xg.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= (1e-10 if prec == "f64" else 2e-5)


def test_tensor_core_precision_with_quadrature_potential(fe):
    """BF16 cell products of the kinetic part plus the float quadrature term: within the
    bf16 bound of the oracle, and the FP32 path at least 10x closer."""
    om, H, m, rng, Vq = _setup(fe, (5.0, 5.0, 5.0), (2, 2, 2), 5, (True, True))
    nvec = 64
    X = rng.standard_normal((om.n_psi, nvec)).astype(np.float32)
    xb = torch.tensor(X, device="cuda")
    ref = H @ X.astype(np.float64)
    errs = {}
    for prec in (fe.FE_BF16_F32ACC, fe.FE_F32):
        y = torch.empty_like(xb)
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(xb), fe._ptr(y), nvec, nvec, prec)
        errs[prec] = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert errs[fe.FE_BF16_F32ACC] <= 1e-2, errs
    assert errs[fe.FE_F32] * 10 <= errs[fe.FE_BF16_F32ACC], errs


def test_full_size_sampled_rows(fe):
    """The benchmark slab (16 x 16 x 48 cells, p = 5, 512 float vectors) with the potential
    given at the Gauss points: sampled rows of Ht_q X against the oracle's row-by-row form,
    including rows on the lowest and highest psi planes and on the periodic seams."""
    slab = W.config2()
    om = OMesh(slab.L, slab.ncell, slab.p, slab.psi_dirichlet)
    m = fe.Mesh.from_slab(slab, with_atoms=False)
    rng = np.random.default_rng(7)
    Vq = torch.tensor(rng.uniform(-1.0, 0.5, (om.n_cells, (slab.p + 1) ** 3)), device="cuda")
    m.set_potential_quad(Vq)
    nvec = slab.nvec
    gen = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn((om.n_psi, nvec), generator=gen, device="cuda", dtype=torch.float32)
    Y = m.apply_H(X, prec=fe.FE_F32)
    NX, NY = om.NX, om.NY
    plane = NX * NY
    rows = np.concatenate([[0, NX - 1, plane - 1, om.n_psi - 1, om.n_psi - plane],
                           rng.integers(0, om.n_psi, 11)])
    Xh = X.cpu().numpy()
    ref = quadpot.apply_Hq_rows(om, Vq.cpu().numpy(), Xh, rows)
    got = Y[torch.tensor(rows)].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5


def test_batch_refuses_and_collocation_returns(fe):
    om, H, m, rng, Vq = _setup(fe, *CASES[0])
    with pytest.raises(fe.FeError):
        fe.Batch([m])
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    m.set_potential(torch.tensor(V, device="cuda"))
    X = rng.standard_normal((om.n_psi, 4))
    Y = m.apply_H(torch.tensor(X, device="cuda")).cpu().numpy()
    ref = assembly.hamiltonian(om, V) @ X
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 1e-10

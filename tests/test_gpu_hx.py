"""GPU parity of the Hamiltonian application, Chebyshev filter, Lanczos bounds and
Rayleigh-Ritz against the FP64 CPU oracle (called through the C ABI).

Tolerances: FP64 H X <= 1e-10 relative (Frobenius); FP32 H X <= 2e-5 relative (float
rounding of ~50 accumulated products per entry, u = 6e-8, with margin); FP64 Ritz values
<= 1e-8 Ha against the oracle's Householder-QR + dense eigh.

Every operator result is also bounded entry by entry (tests/entrywise.py): |Y - Y_ref|_Iv
<= tol (|Ht| |X|)_Iv, the floating-point bound of a sum of products, with tol = 1e-13 for
FP64 (~900 u) and 1e-6 for FP32 (~17 u); filter results column by column against the
column's largest entry (1e-11 FP64, 1e-5 FP32).  A seam plane or tile face wrong by far
less than the Frobenius bounds allow fails these.
"""
import numpy as np
import pytest
import torch

import workloads as W
from entrywise import assert_column_maxabs, assert_operator_entries, magnitude
from oracle import assembly, chefsi
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _setup(fe, L, ncell, p, dirichlet, seed=0):
    om = OMesh(L, ncell, p, dirichlet)
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    H = assembly.hamiltonian(om, V)
    m = fe.Mesh(L, ncell, p, dirichlet)
    m.set_potential(torch.tensor(V, dtype=torch.float64, device="cuda"))
    return om, H, m, rng


def _block(X, prec, fe, ld=None):
    dt = fe.storage_dtype(prec)
    n, k = X.shape
    ld = ld or k
    buf = torch.zeros((n, ld), dtype=dt, device="cuda")
    buf[:, :k] = torch.tensor(X, dtype=dt)
    return buf, buf[:, :k]


CASES = [
    # (L, ncell, p, psi Dirichlet faces)
    ((4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True)),
    ((3.0, 5.0, 7.0), (3, 1, 3), 2, (False, True)),    # odd nx (partial block), one y cell
    ((2.0, 2.0, 3.0), (1, 1, 2), 1, (False, False)),
    ((4.0, 4.0, 6.0), (2, 3, 3), 4, (True, False)),
    ((5.0, 5.0, 5.0), (2, 2, 2), 5, (True, True)),
    ((6.0, 6.0, 6.0), (2, 2, 2), 6, (False, False)),
    ((8.0, 8.0, 30.0), (4, 4, 15), 3, (True, True)),    # several z segments
]


@pytest.mark.parametrize("L,ncell,p,dirichlet", CASES)
@pytest.mark.parametrize("nvec,ld", [(1, 2), (13, 14), (40, 40)])
def test_apply_H_f64_matches_oracle(fe, L, ncell, p, dirichlet, nvec, ld):
    om, H, m, rng = _setup(fe, L, ncell, p, dirichlet)
    X = rng.standard_normal((om.n_psi, nvec))
    buf, Xg = _block(X, fe.FE_F64, fe, ld)
    ybuf = torch.full_like(buf, 7.0)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(buf), fe._ptr(ybuf), nvec, ld, fe.FE_F64)
    Y = ybuf[:, :nvec].cpu().numpy()
    ref = H @ X
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 1e-10
    assert_operator_entries(Y, ref, magnitude(H, X), 1e-13, "FP64 H X")
    # padding columns beyond nvec are untouched
    if ld > nvec:
        assert torch.all(ybuf[:, nvec:] == 7.0)


# float block operator: the cases above plus a p = 5 mesh whose cells have three different
# edge lengths (the in-plane scales ax, ay and az all differ and none is 1) and a full 4 x 4
# cell tile in x and y
F32_CASES = CASES[:6] + [((9.0, 6.0, 14.0), (4, 4, 5), 5, (True, True))]


@pytest.mark.parametrize("L,ncell,p,dirichlet", F32_CASES)
@pytest.mark.parametrize("nvec,ld", [(3, 4), (37, 40), (64, 64)])
def test_apply_H_f32_matches_oracle(fe, L, ncell, p, dirichlet, nvec, ld):
    om, H, m, rng = _setup(fe, L, ncell, p, dirichlet, seed=1)
    X = rng.standard_normal((om.n_psi, nvec)).astype(np.float32)
    buf, Xg = _block(X, fe.FE_F32, fe, ld)
    ybuf = torch.zeros_like(buf)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(buf), fe._ptr(ybuf), nvec, ld, fe.FE_F32)
    ref = H @ X.astype(np.float64)
    Y = ybuf[:, :nvec].double().cpu().numpy()
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 2e-5
    assert_operator_entries(Y, ref, magnitude(H, X), 1e-6, "FP32 H X")


# FP32-accurate tensor-core operator (FE_F32_F32ACC: in-plane contractions as split-TF32
# tcgen05 MMAs, hi*hi + lo*hi + hi*lo, FP32 accumulation): the FP32 Frobenius bound and an
# entry bound of 4e-6 (|Ht||X| units; the split products carry ~2^-22 per product, the
# CUDA-core FP32 operator measures 2.5e-7)
TC32_CASES = [c for c in F32_CASES if c[2] <= 5]


@pytest.mark.parametrize("L,ncell,p,dirichlet", TC32_CASES)
@pytest.mark.parametrize("nvec,ld", [(3, 4), (37, 40), (64, 64)])
def test_apply_H_tc32_matches_oracle(fe, L, ncell, p, dirichlet, nvec, ld):
    om, H, m, rng = _setup(fe, L, ncell, p, dirichlet, seed=1)
    X = rng.standard_normal((om.n_psi, nvec)).astype(np.float32)
    buf, Xg = _block(X, fe.FE_F32, fe, ld)
    ybuf = torch.full_like(buf, 5.0)
    fe._lib.call("fe_apply_H", m.handle, fe._ptr(buf), fe._ptr(ybuf), nvec, ld, fe.FE_F32_F32ACC)
    ref = H @ X.astype(np.float64)
    Y = ybuf[:, :nvec].double().cpu().numpy()
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 2e-5
    assert_operator_entries(Y, ref, magnitude(H, X), 4e-6, "split-TF32 H X")
    if ld > nvec:
        assert torch.all(ybuf[:, nvec:] == 5.0)


def test_tc32_filter_and_refusals(fe):
    """The tensor-core operator inside the fused filter (beta Z with Z = Y in place) against
    the oracle, and its refusals: p = 6 (block beyond one MMA tile) and Bloch blocks."""
    om, H, m, rng = _setup(fe, (5.0, 5.0, 10.0), (2, 2, 4), 5, (True, True), seed=8)
    X = rng.standard_normal((om.n_psi, 16)).astype(np.float32).astype(np.float64)
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, rng.standard_normal(om.n_psi), 30)
    a = lo + 0.1 * (hi - lo)
    for degree in (1, 6):
        ref = chefsi.cheb_filter(lambda Z: H @ Z, X, degree, a, hi, lo)
        Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
        m.cheb_filter(Xg, degree, a, hi, lo, prec=fe.FE_F32_F32ACC)
        got = Xg.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-4
        assert_column_maxabs(got, ref, 2e-5, f"split-TF32 filter degree {degree}")
    m6 = fe.Mesh((6.0, 6.0, 6.0), (2, 2, 2), 6)
    m6.set_potential(torch.zeros(m6.n_psi, dtype=torch.float64, device="cuda"))
    X6 = torch.zeros((m6.n_psi, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(fe.FeError) as e:
        m6.apply_H(X6, prec=fe.FE_F32_F32ACC)
    assert e.value.status == fe._lib.FE_EUNSUPPORTED


def test_apply_H_is_deterministic(fe):
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True))
    X = torch.tensor(rng.standard_normal((om.n_psi, 24)), device="cuda")
    a = m.apply_H(X)
    b = m.apply_H(X)
    assert torch.equal(a, b)


def test_apply_H_rejects_bad_arguments(fe):
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True))
    X = torch.zeros((om.n_psi, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:   # ld * 8 not a multiple of 16
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(X), fe._ptr(X.clone()), 3, 3, fe.FE_F64)
    assert e.value.status == fe._lib.FE_EINVAL
    with pytest.raises(fe.FeError):        # in place
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(X), fe._ptr(X), 2, 2, fe.FE_F64)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_cheb_filter_matches_oracle(fe, prec, tol):
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=2)
    X = rng.standard_normal((om.n_psi, 12)).astype(np.float32).astype(np.float64)
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, rng.standard_normal(om.n_psi), 30)
    a = lo + 0.1 * (hi - lo)
    for degree in (1, 2, 7):
        ref = chefsi.cheb_filter(lambda Z: H @ Z, X, degree, a, hi, lo)
        Xg = torch.tensor(X, dtype=fe.storage_dtype(p_), device="cuda")
        m.cheb_filter(Xg, degree, a, hi, lo, prec=p_)
        got = Xg.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
        assert_column_maxabs(got, ref, 1e-11 if prec == "f64" else 1e-5, f"degree {degree}")


def test_lanczos_bounds_match_oracle(fe):
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=3)
    v0 = W.lanczos_start(om.n_psi)
    lo_ref, hi_ref = chefsi.lanczos_bounds(lambda v: H @ v, v0, 25)
    lo, hi = m.lanczos_bounds(torch.tensor(v0, device="cuda"), 25)
    assert abs(lo - lo_ref) <= 1e-8 * abs(hi_ref)
    assert abs(hi - hi_ref) <= 1e-8 * abs(hi_ref)
    ev = np.linalg.eigvalsh(H.toarray())
    assert hi >= ev[-1]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rayleigh_ritz_matches_oracle(fe, prec):
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=4)
    X = rng.standard_normal((om.n_psi, 12)).astype(np.float32).astype(np.float64)
    lam_ref, _ = chefsi.rayleigh_ritz(lambda Z: H @ Z, X)
    Xg = torch.tensor(X, dtype=fe.storage_dtype(p_), device="cuda")
    lam = m.rayleigh_ritz(Xg, prec=p_).cpu().numpy()
    assert np.max(np.abs(lam - lam_ref)) <= (1e-8 if prec == "f64" else 1e-4)
    Q = Xg.double().cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) <= (1e-10 if prec == "f64" else 1e-5)
    if prec == "f64":
        assert np.max(np.abs(Q.T @ (H @ Q) - np.diag(lam))) <= 1e-9


def test_chefsi_converges_to_dense_eigh_on_gpu(fe):
    om, H, m, rng = _setup(fe, (3.0, 3.0, 6.0), (2, 2, 4), 2, (True, True), seed=6)
    ev = np.linalg.eigvalsh(H.toarray())
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(om.n_psi), device="cuda"), 30)
    Xg = torch.tensor(rng.standard_normal((om.n_psi, 12)), device="cuda")
    a0, a = lo, ev[14]
    for _ in range(25):
        m.cheb_filter(Xg, 12, a, hi, a0)
        lam = m.rayleigh_ritz(Xg).cpu().numpy()
        a0 = lam[0]
    np.testing.assert_allclose(lam[:8], ev[:8], atol=1e-10)


def test_rayleigh_ritz_tensor_core_products(fe):
    """Float block with the block products in FP32-accurate tensor-core emulation: Ritz
    values within the float-storage tolerance of the oracle, orthonormal to 1e-5."""
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=14)
    m.set_rr_products(True)
    X = rng.standard_normal((om.n_psi, 12)).astype(np.float32).astype(np.float64)
    lam_ref, _ = chefsi.rayleigh_ritz(lambda Z: H @ Z, X)
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    lam = m.rayleigh_ritz(Xg, prec=fe.FE_F32).cpu().numpy()
    assert np.max(np.abs(lam - lam_ref)) <= 1e-4
    Q = Xg.double().cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) <= 1e-5


def test_rayleigh_ritz_tensor_core_products_decline_an_ill_conditioned_block(fe):
    """Nearly dependent columns (cond of the scaled Gram matrix ~1e10, beyond what FP32-accurate
    products resolve): the tensor-core Gram path declines and the double path gives the Ritz
    values of the float block's span."""
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=15)
    m.set_rr_products(True)
    B = rng.standard_normal((om.n_psi, 8))
    B[:, 7] = B[:, 6] + 1e-5 * (B[:, 5] + B[:, 7])
    X = B.astype(np.float32).astype(np.float64)
    lam_ref, _ = chefsi.rayleigh_ritz(lambda Z: H @ Z, X)
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    lam = m.rayleigh_ritz(Xg, prec=fe.FE_F32).cpu().numpy()
    assert np.max(np.abs(lam - lam_ref)) <= 1e-5 * max(1.0, np.max(np.abs(lam_ref)))
    Q = Xg.double().cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(8))) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rayleigh_ritz_jacobi_eigensolver_matches_oracle(fe, prec):
    """The cyclic-Jacobi option for the projected eigenproblem gives the oracle's Ritz values
    and an orthonormal block that diagonalises H, to the same bounds as divide-and-conquer."""
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om, H, m, rng = _setup(fe, (4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True), seed=24)
    m.set_rr_eigensolver(True)
    X = rng.standard_normal((om.n_psi, 40)).astype(np.float32).astype(np.float64)
    lam_ref, _ = chefsi.rayleigh_ritz(lambda Z: H @ Z, X)
    Xg = torch.tensor(X, dtype=fe.storage_dtype(p_), device="cuda")
    lam = m.rayleigh_ritz(Xg, prec=p_).cpu().numpy()
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - lam_ref)) <= (1e-8 if prec == "f64" else 1e-4)
    Q = Xg.double().cpu().numpy()
    assert np.max(np.abs(Q.T @ Q - np.eye(40))) <= (1e-10 if prec == "f64" else 1e-5)
    if prec == "f64":
        assert np.max(np.abs(Q.T @ (H @ Q) - np.diag(lam))) <= 1e-9

"""Nonlocal term with synthetic projectors on the GPU against the oracle: Ht X including
Ht_nloc (FP64, FP32, BF16 cell path) with atoms near the periodic x/y seams and near the
z faces (Dirichlet and Neumann), removal of the term, the converged lowest eigenpairs of
the full operator, and the entry points that refuse the term.

Tolerances: as for the local operator (FP64 1e-10, FP32 2e-5, BF16 1e-2 relative)."""
import numpy as np
import pytest
import torch

from oracle import assembly, chefsi, projectors
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu

ATOMS = np.array([[0.2, 3.9, 1.1], [2.5, 2.0, 4.6], [3.8, 0.1, 8.4]])
SIGMA = np.array([0.7, 0.9, 0.6])
D = np.array([[0.9, 0.4, 0.4, 0.4], [1.3, 0.2, 0.0, 0.6], [0.5, 0.3, 0.7, 0.1]])
RC = 2.6


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _setup(fe, dirichlet, p=3):
    L, ncell = (4.0, 4.0, 9.0), (2, 2, 4)
    om = OMesh(L, ncell, p, dirichlet)
    rng = np.random.default_rng(7)
    V = rng.uniform(-1.0, 0.5, om.n_psi)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    H = assembly.hamiltonian(om, V, K, M).toarray() + projectors.nonlocal_scaled(om, M, ATOMS, SIGMA, D, RC)
    m = fe.Mesh(L, ncell, p, dirichlet)
    m.set_potential(torch.tensor(V, device="cuda"))
    m.set_nonlocal(ATOMS, SIGMA, D, RC)
    return om, H, m


@pytest.mark.parametrize("dirichlet", [(True, True), (False, True), (False, False)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_H_with_nonlocal_matches_oracle(fe, dirichlet, prec):
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om, H, m = _setup(fe, dirichlet)
    X = np.random.default_rng(1).standard_normal((om.n_psi, 12))
    if prec == "f32":
        X = X.astype(np.float32).astype(np.float64)
    Y = m.apply_H(torch.tensor(X, dtype=fe.storage_dtype(P), device="cuda"), prec=P)
    ref = H @ X
    err = np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if prec == "f64" else 2e-5), err


def test_bf16_cell_path_with_nonlocal(fe):
    om, H, m = _setup(fe, (True, True))
    X = np.random.default_rng(2).standard_normal((om.n_psi, 8)).astype(np.float32)
    Y = m.apply_H(torch.tensor(X, device="cuda"), prec=fe.FE_BF16_F32ACC)
    ref = H @ X.astype(np.float64)
    assert np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-2


def test_removing_the_term_restores_the_local_operator(fe):
    om, H, m = _setup(fe, (True, True))
    m.set_nonlocal(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4)), RC)
    X = torch.tensor(np.random.default_rng(3).standard_normal((om.n_psi, 6)), device="cuda")
    with_nl = m.apply_H(X).cpu().numpy()
    Hloc = H - projectors.nonlocal_scaled(om, assembly.lumped_mass(om), ATOMS, SIGMA, D, RC)
    ref = Hloc @ X.cpu().numpy()
    assert np.linalg.norm(with_nl - ref) / np.linalg.norm(ref) <= 1e-10


def test_chefsi_with_nonlocal_converges_to_dense_spectrum(fe):
    om, H, m = _setup(fe, (True, True))
    ev = np.linalg.eigvalsh(H)
    nvec, k = 16, 8
    v0 = torch.tensor(np.random.default_rng(4).standard_normal(om.n_psi), device="cuda")
    lo, hi = m.lanczos_bounds(v0, 30)
    lo_ref, hi_ref = chefsi.lanczos_bounds(lambda v: H @ v, v0.cpu().numpy(), 30)
    assert abs(lo - lo_ref) <= 1e-8 * hi_ref and abs(hi - hi_ref) <= 1e-8 * hi_ref
    X = torch.tensor(np.random.default_rng(5).standard_normal((om.n_psi, nvec)), device="cuda")
    a0, a = lo, ev[nvec + 4]
    for _ in range(12):
        m.cheb_filter(X, 16, a, hi, a0)
        lam = m.rayleigh_ritz(X).cpu().numpy()
        a0, a = min(a0, lam[0]), lam[-1]
    assert np.max(np.abs(lam[:k] - ev[:k])) <= 1e-10 * np.max(np.abs(ev))


def test_batch_and_static_filter_refuse_the_term(fe):
    om, H, m = _setup(fe, (True, True))
    with pytest.raises(fe.FeError) as e:
        fe.Batch([m])
    assert e.value.status == 7
    X = torch.zeros((om.n_psi, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(X), 4, 4, 4, 1.0, 2.0, 0.0,
                     fe.FE_F64)
    assert e.value.status == 7

"""Failure reporting through the C ABI: every case below returns a status (no fault, no
hang, no silent NaN result), and the caller's arrays are left as the header documents.

* a NaN in the Poisson density: FE_EINVAL before any iteration (info filled);
* a rank-deficient block in Rayleigh-Ritz (a zero column): FE_EBREAKDOWN, block unchanged;
* Lanczos from a zero or non-finite start vector: FE_EINVAL; from an eigenvector (the
  Krylov space is invariant after one step): FE_EBREAKDOWN; on a space smaller than the
  step count the exhausted Krylov space gives the exact extreme eigenvalues;
* the Poisson iteration cap (FE_ENOCONV) is covered in test_gpu_poisson.py.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assembly
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def test_poisson_nan_density_is_rejected(fe):
    slab = W.small_slab(ncell=(2, 2, 4), p=3, L=(4.0, 4.0, 9.0), natoms=2, nvec=8, degree=6)
    m = fe.Mesh.from_slab(slab)
    rho = torch.ones(m.n_phi, dtype=torch.float64, device="cuda") * 0.01
    rho[m.n_phi // 2] = float("nan")
    with pytest.raises(fe.FeError) as e:
        m.poisson_solve(slab.bias, rho=rho, rtol=1e-10, max_iter=500)
    assert e.value.status == fe._lib.FE_EINVAL and "not finite" in str(e.value)
    # the same call with a finite density converges
    rho[m.n_phi // 2] = 0.01
    _, _, info = m.poisson_solve(slab.bias, rho=rho, rtol=1e-10, max_iter=5000)
    assert info.status == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rayleigh_ritz_zero_column_reports_breakdown(fe, prec):
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om = OMesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    m = fe.Mesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    rng = np.random.default_rng(41)
    m.set_potential(torch.tensor(rng.uniform(-1, 1, om.n_psi), device="cuda"))
    X = torch.tensor(rng.standard_normal((om.n_psi, 8)), dtype=fe.storage_dtype(p_),
                     device="cuda")
    X[:, 5] = 0.0
    X0 = X.clone()
    for tc in ((False, True) if prec == "f32" else (False,)):
        if prec == "f32":
            m.set_rr_products(tc)
        with pytest.raises(fe.FeError) as e:
            m.rayleigh_ritz(X, prec=p_)
        assert e.value.status == fe._lib.FE_EBREAKDOWN and "column 5" in str(e.value)
        torch.cuda.synchronize()
        assert torch.equal(X, X0)


def test_lanczos_bad_start_vectors(fe):
    om = OMesh((4.0, 4.0, 9.0), (2, 2, 4), 3, (False, False))
    m = fe.Mesh((4.0, 4.0, 9.0), (2, 2, 4), 3, (False, False))
    m.set_potential(torch.full((om.n_psi,), 0.3, dtype=torch.float64, device="cuda"))
    zero = torch.zeros(om.n_psi, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        m.lanczos_bounds(zero, 20)
    assert e.value.status == fe._lib.FE_EINVAL
    bad = torch.ones(om.n_psi, dtype=torch.float64, device="cuda")
    bad[3] = float("nan")
    with pytest.raises(fe.FeError) as e:
        m.lanczos_bounds(bad, 20)
    assert e.value.status == fe._lib.FE_EINVAL
    # M^1/2 1 is an exact eigenvector of Ht with a constant potential and Neumann faces
    # (K 1 = 0): the Krylov space is invariant after the first step
    Mpsi = assembly.lumped_mass(om)[om.psi_to_phi()]
    eigv = torch.tensor(np.sqrt(Mpsi), device="cuda")
    with pytest.raises(fe.FeError) as e:
        m.lanczos_bounds(eigv, 20)
    assert e.value.status == fe._lib.FE_EBREAKDOWN
    # a random start vector on the same operator is fine, and bounds the spectrum
    H = assembly.hamiltonian(om, np.full(om.n_psi, 0.3))
    ev = np.linalg.eigvalsh(H.toarray())
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(om.n_psi), device="cuda"), 20)
    assert lo >= ev[0] - 1e-9 and hi >= ev[-1]


def test_lanczos_exhausts_a_small_space_exactly(fe):
    # 1 x 1 x 2 cells, p = 1, Neumann faces: 3 psi nodes; 8 steps exhaust the space and the
    # tridiagonal matrix holds the whole spectrum
    om = OMesh((2.0, 2.0, 3.0), (1, 1, 2), 1, (False, False))
    m = fe.Mesh((2.0, 2.0, 3.0), (1, 1, 2), 1, (False, False))
    V = np.array([0.1, -0.4, 0.7])[:om.n_psi]
    m.set_potential(torch.tensor(V, device="cuda"))
    ev = np.linalg.eigvalsh(assembly.hamiltonian(om, V).toarray())
    lo, hi = m.lanczos_bounds(torch.tensor([1.0, 0.3, -0.2][:om.n_psi], device="cuda"), 8)
    assert abs(lo - ev[0]) <= 1e-10 * max(1.0, abs(ev[-1]))
    assert abs(hi - ev[-1]) <= 1e-10 * max(1.0, abs(ev[-1]))

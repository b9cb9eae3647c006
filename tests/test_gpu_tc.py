"""GPU parity of the tensor-core (tcgen05, bf16 operands, fp32 accumulation) cell-matrix
Hamiltonian against the FP64 oracle.

Tolerance: both operands of the cell product are rounded to bf16 (relative 2^-9 each), so
an entry of Ht X carries a relative error of about 2^-8 of the magnitude of its largest
terms; for random blocks the Frobenius-relative error is a few 1e-3.  The test bound is
1e-2, and the FP32 path must be at least 10x closer (so the bf16 arithmetic is really the
one that ran).
"""
import numpy as np
import pytest
import torch

from entrywise import assert_operator_entries, magnitude
from oracle import assembly
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


CASES = [
    ((4.0, 4.0, 9.0), (2, 2, 4), 3, (True, True)),
    ((3.0, 5.0, 7.0), (3, 1, 3), 2, (False, True)),
    ((4.0, 4.0, 6.0), (2, 3, 3), 4, (True, False)),
    ((5.0, 5.0, 5.0), (2, 2, 2), 5, (True, True)),
    ((6.0, 6.0, 10.0), (3, 3, 5), 5, (False, False)),
]


@pytest.mark.parametrize("L,ncell,p,dirichlet", CASES)
@pytest.mark.parametrize("nvec,ld", [(8, 8), (70, 72), (128, 128)])
def test_apply_H_bf16_matches_oracle(fe, L, ncell, p, dirichlet, nvec, ld):
    om = OMesh(L, ncell, p, dirichlet)
    rng = np.random.default_rng(11)
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    H = assembly.hamiltonian(om, V)
    m = fe.Mesh(L, ncell, p, dirichlet)
    m.set_potential(torch.tensor(V, device="cuda"))
    X = rng.standard_normal((om.n_psi, nvec)).astype(np.float32)
    buf = torch.zeros((om.n_psi, ld), dtype=torch.float32, device="cuda")
    buf[:, :nvec] = torch.tensor(X)
    ref = H @ X.astype(np.float64)
    errs = {}
    for prec in (fe.FE_BF16_F32ACC, fe.FE_F32):
        y = torch.full_like(buf, 3.0)
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(buf), fe._ptr(y), nvec, ld, prec)
        got = y[:, :nvec].double().cpu().numpy()
        errs[prec] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        # entry bound: both bf16 operands rounded (2^-8 relative each) -> 2e-2 of the terms'
        # magnitudes; FP32 as in the FP32 operator tests
        assert_operator_entries(got, ref, magnitude(H, X), 2e-2 if prec == fe.FE_BF16_F32ACC
                                else 1e-6, f"precision {prec}")
        if ld > nvec:
            assert torch.all(y[:, nvec:] == 3.0)
    assert errs[fe.FE_BF16_F32ACC] <= 1e-2, errs
    assert errs[fe.FE_F32] * 10 <= errs[fe.FE_BF16_F32ACC], errs


def test_bf16_filter_runs_and_tracks_f32(fe):
    L, ncell, p = (5.0, 5.0, 10.0), (2, 2, 4), 5
    om = OMesh(L, ncell, p)
    rng = np.random.default_rng(12)
    V = -np.abs(rng.standard_normal(om.n_psi))
    H = assembly.hamiltonian(om, V)
    m = fe.Mesh(L, ncell, p)
    m.set_potential(torch.tensor(V, device="cuda"))
    lo, hi = m.lanczos_bounds(torch.tensor(rng.standard_normal(om.n_psi), device="cuda"), 30)
    ev = np.linalg.eigvalsh(H.toarray())
    X0 = rng.standard_normal((om.n_psi, 16)).astype(np.float32)
    res = {}
    for prec in (fe.FE_F32, fe.FE_BF16_F32ACC):
        X = torch.tensor(X0, device="cuda")
        # the usual CheFSI bounds: the cut follows the largest Ritz value and the lower
        # estimate only moves down
        a0, a = lo, ev[20]
        for _ in range(8):
            m.cheb_filter(X, 16, a, hi, a0, prec=prec)
            lam = m.rayleigh_ritz(X, prec=prec).cpu().numpy()
            a0, a = min(a0, lam[0]), lam[-1]
        res[prec] = lam
    # both converge towards the dense spectrum (the FP64 recurrence reaches 2e-8 here); bf16
    # filtering with an exact Rayleigh-Ritz
    assert np.max(np.abs(res[fe.FE_F32][:8] - ev[:8])) < 1e-5
    assert np.max(np.abs(res[fe.FE_BF16_F32ACC][:8] - ev[:8])) < 1e-2

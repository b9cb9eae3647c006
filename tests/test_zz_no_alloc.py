"""The allocation-free Chebyshev filter (fe_cheb_filter_static) against fe_cheb_filter.

fe_cheb_filter_static serves callers that cannot let the library call cudaMalloc (a
framework allocator that already holds the free device memory, a fixed memory budget, a
latency-sensitive loop that must not synchronise the device).  It keeps the filter's
scratch in a static device array, so it must give the same block as the allocating filter,
call after call, even though the array keeps the previous call's contents.  Tolerances
are those of the filter's parity tests (1e-10 FP64, 2e-4 FP32, relative Frobenius).

This file is named to run last: it must pass alone in a fresh process and after the rest.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import assembly, chefsi
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _call_static(fe, m, X, degree, a, b, a0, prec):
    fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(X), X.shape[1], X.stride(0),
                 int(degree), float(a), float(b), float(a0), int(prec))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_static_filter_matches_allocating_filter_twice(fe, prec, tol):
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om = OMesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    rng = np.random.default_rng(17)
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    H = assembly.hamiltonian(om, V)
    m = fe.Mesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    m.set_potential(torch.tensor(V, device="cuda"))
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, rng.standard_normal(om.n_psi), 30)
    a = lo + 0.1 * (hi - lo)
    dt = fe.storage_dtype(p_)
    for call, (nvec, degree) in enumerate([(12, 7), (16, 6)]):   # two calls in a row
        X0 = torch.tensor(rng.standard_normal((om.n_psi, nvec)), dtype=dt, device="cuda")
        ref = X0.clone()
        m.cheb_filter(ref, degree, a, hi, lo, prec=p_)
        got = X0.clone()
        _call_static(fe, m, got, degree, a, hi, lo, p_)
        torch.cuda.synchronize()
        r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
        assert np.linalg.norm(g - r) / np.linalg.norm(r) <= tol, call


def test_static_filter_rejects_blocks_above_the_limit(fe):
    # 64 MiB limit: 212,400 psi nodes x 48 doubles (81.6 MB) is above it
    m = fe.Mesh((40.0, 40.0, 40.0), (20, 20, 20), 3)
    m.set_potential(torch.zeros(m.n_psi, dtype=torch.float64, device="cuda"))
    X = torch.zeros((m.n_psi, 48), dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        _call_static(fe, m, X, 3, 1.0, 2.0, 0.0, fe.FE_F64)
    assert e.value.status == fe._lib.FE_EINVAL and "static limit" in str(e.value)
    with pytest.raises(fe.FeError) as e:
        _call_static(fe, m, X[:8, :4].float().contiguous(), 3, 1.0, 2.0, 0.0, fe.FE_BF16_F32ACC)
    assert e.value.status == fe._lib.FE_EUNSUPPORTED

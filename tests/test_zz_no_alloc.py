"""The allocation-free Chebyshev filter (fe_cheb_filter_static) against fe_cheb_filter.

fe_cheb_filter_static serves callers that cannot let the library call cudaMalloc (a
framework allocator that already holds the free device memory, a fixed memory budget, a
latency-sensitive loop that must not synchronise the device).  It keeps the filter's
scratch in a static device array and launches the same operator kernels in the same order
as fe_cheb_filter, so its result must be bitwise identical to the allocating filter's,
call after call, even though the array keeps the previous call's contents.  The tests
also check the property the entry point exists for: a call on a fresh mesh leaves the
device's free memory unchanged, while the allocating filter on the same mesh takes its
scratch block (which shows that the measurement would see an allocation).

This file is named to run last: it must pass alone in a fresh process and after the rest.
"""
import gc

import numpy as np
import pytest
import torch

from oracle import assembly, chefsi
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu

LIMIT = 64 << 20   # bytes of the static scratch array


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _call_static(fe, m, X, degree, a, b, a0, prec):
    fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(X), X.shape[1], X.stride(0),
                 int(degree), float(a), float(b), float(a0), int(prec))


def _bounds(H, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, rng.standard_normal(n), 30)
    return lo, lo + 0.1 * (hi - lo), hi


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_filter_matches_allocating_filter_twice(fe, prec):
    p_ = fe.FE_F64 if prec == "f64" else fe.FE_F32
    om = OMesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    rng = np.random.default_rng(17)
    V = rng.uniform(-1.0, 1.0, om.n_psi)
    H = assembly.hamiltonian(om, V)
    m = fe.Mesh((4.0, 4.0, 9.0), (2, 2, 4), 3)
    m.set_potential(torch.tensor(V, device="cuda"))
    lo, a, hi = _bounds(H, om.n_psi, 18)
    dt = fe.storage_dtype(p_)
    for call, (nvec, degree) in enumerate([(12, 7), (16, 6)]):   # two calls in a row
        X0 = torch.tensor(rng.standard_normal((om.n_psi, nvec)), dtype=dt, device="cuda")
        ref = X0.clone()
        m.cheb_filter(ref, degree, a, hi, lo, prec=p_)
        got = X0.clone()
        _call_static(fe, m, got, degree, a, hi, lo, p_)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), call
    # and the filter is the oracle's (the filter parity test's FP64 / FP32 bounds)
    Xg = torch.tensor(rng.standard_normal((om.n_psi, 8)), dtype=dt, device="cuda")
    ref = chefsi.cheb_filter(lambda Z: H @ Z, Xg.double().cpu().numpy(), 5, a, hi, lo)
    _call_static(fe, m, Xg, 5, a, hi, lo, p_)
    got = Xg.double().cpu().numpy()
    tol = 1e-10 if prec == "f64" else 2e-4
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


def test_static_filter_with_quadrature_potential(fe):
    """With the potential integrated by Gauss quadrature the operator adds its cell-by-cell
    term (no workspace either); both filters still agree bit for bit."""
    L, ncell, p = (5.0, 5.0, 10.0), (2, 2, 4), 4
    m = fe.Mesh(L, ncell, p)
    rng = np.random.default_rng(23)
    nq = m.n_cells * (p + 1) ** 3
    m.set_potential_quad(torch.tensor(rng.uniform(-1.0, 0.5, nq), device="cuda"))
    for prec in (fe.FE_F64, fe.FE_F32):
        X0 = torch.tensor(rng.standard_normal((m.n_psi, 20)), dtype=fe.storage_dtype(prec),
                          device="cuda")
        for _ in range(2):
            ref = X0.clone()
            m.cheb_filter(ref, 6, 3.0, 60.0, -1.0, prec=prec)
            got = X0.clone()
            _call_static(fe, m, got, 6, 3.0, 60.0, -1.0, prec)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), prec


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_static_filter_allocates_nothing(fe):
    """Free device memory around the first static call on a fresh mesh is unchanged; the
    allocating filter on the same mesh then takes at least its scratch block."""
    L, ncell, p = (16.0, 16.0, 32.0), (16, 16, 16), 2
    nvec = 512
    warm = fe.Mesh(L, ncell, p)    # loads the kernels of this shape before the measurement
    warm.set_potential(torch.zeros(warm.n_psi, dtype=torch.float64, device="cuda"))
    Xw = torch.ones((warm.n_psi, nvec), dtype=torch.float32, device="cuda")
    _call_static(fe, warm, Xw, 2, 1.0, 50.0, 0.0, fe.FE_F32)
    m = fe.Mesh(L, ncell, p)
    m.set_potential(torch.full((m.n_psi,), -0.5, dtype=torch.float64, device="cuda"))
    X = torch.ones((m.n_psi, nvec), dtype=torch.float32, device="cuda")
    need = m.n_psi * nvec * 4
    assert 32 << 20 < need <= LIMIT
    gc.collect()
    before = _free_bytes()
    _call_static(fe, m, X, 3, 1.0, 50.0, 0.0, fe.FE_F32)
    after = _free_bytes()
    assert after >= before, (before, after)
    Y = torch.ones_like(X)
    before = _free_bytes()
    m.cheb_filter(Y, 3, 1.0, 50.0, 0.0, prec=fe.FE_F32)
    after = _free_bytes()
    assert before - after >= need, (before, after, need)
    assert torch.equal(X, Y)


def test_static_filter_limit_and_arguments(fe):
    # 16 x 16 x 16 cells, p = 2, Dirichlet z faces: 31,744 psi nodes; float rows of 528
    # entries need 67,043,328 bytes (just below 64 MiB), 532 entries 67,551,232 (above)
    m = fe.Mesh((16.0, 16.0, 32.0), (16, 16, 16), 2)
    assert m.n_psi == 31744
    m.set_potential(torch.zeros(m.n_psi, dtype=torch.float64, device="cuda"))
    below = torch.zeros((m.n_psi, 528), dtype=torch.float32, device="cuda")
    below[:, :16] = 1.0
    ref = below.clone()
    m.cheb_filter(ref[:, :16], 2, 1.0, 2.0, 0.0, prec=fe.FE_F32)
    fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(below), 16, 528, 2, 1.0, 2.0, 0.0,
                 fe.FE_F32)
    torch.cuda.synchronize()
    assert torch.equal(below, ref)
    del below, ref
    above = torch.zeros((m.n_psi, 532), dtype=torch.float32, device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe._lib.call("fe_cheb_filter_static", m.handle, fe._ptr(above), 16, 532, 2, 1.0, 2.0,
                     0.0, fe.FE_F32)
    assert e.value.status == fe._lib.FE_EINVAL and "static limit" in str(e.value)
    # FE_F64: 212,400 psi nodes x 48 doubles (81.6 MB) is above the limit
    big = fe.Mesh((40.0, 40.0, 40.0), (20, 20, 20), 3)
    big.set_potential(torch.zeros(big.n_psi, dtype=torch.float64, device="cuda"))
    X = torch.zeros((big.n_psi, 48), dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        _call_static(fe, big, X, 3, 1.0, 2.0, 0.0, fe.FE_F64)
    assert e.value.status == fe._lib.FE_EINVAL and "static limit" in str(e.value)
    small = above[:64, :4].contiguous()
    with pytest.raises(fe.FeError) as e:
        _call_static(fe, m, small, 3, 1.0, 2.0, 0.0, fe.FE_BF16_F32ACC)
    assert e.value.status == fe._lib.FE_EUNSUPPORTED
    # bounds as for fe_cheb_filter: finite, a0 < a < b
    Xs = torch.zeros((m.n_psi, 4), dtype=torch.float32, device="cuda")
    for a, b, a0 in ((1.0, float("inf"), 0.0), (1.0, 2.0, float("-inf")), (1.0, 2.0, 1.5),
                     (float("nan"), 2.0, 0.0)):
        with pytest.raises(fe.FeError) as e:
            _call_static(fe, m, Xs, 3, a, b, a0, fe.FE_F32)
        assert e.value.status == fe._lib.FE_EINVAL

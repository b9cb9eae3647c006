"""Batched operator and filter over independent slabs (one launch per step for every
instance) against the oracle and against the per-instance entry points: ragged batches
(different heights, vector counts and leading dimensions), single-instance batches, the
24-slab bias sweep at full size on sampled rows, and the rejection of incompatible meshes.

Tolerances as for the single-mesh path: FP64 1e-10 relative (Frobenius) against the oracle,
FP32 2e-5; batch against the per-instance call 1e-12 (FP64) and 1e-6 (FP32), the same
arithmetic in the same order up to the compiler's scheduling of one shared kernel body.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assembly, chefsi
from oracle.mesh import Mesh as OMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


def _instances(fe, heights, p=3, nx=3, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for k, h in enumerate(heights):
        L = (2.0 * nx, 2.0 * nx, 2.0 * h)
        dirichlet = (True, True) if k % 2 == 0 else (True, False)
        om = OMesh(L, (nx, nx, h), p, dirichlet)
        V = rng.uniform(-1.0, 0.5, om.n_psi)
        m = fe.Mesh(L, (nx, nx, h), p, dirichlet)
        m.set_potential(torch.tensor(V, device="cuda"))
        out.append((om, V, m))
    return out


def _block(rng, n, nvec, ld, dtype):
    buf = torch.zeros((n, ld), dtype=dtype, device="cuda")
    X = rng.standard_normal((n, nvec))
    buf[:, :nvec] = torch.tensor(X, dtype=dtype)
    return buf, X


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_apply_H_ragged(fe, prec):
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = fe.storage_dtype(P)
    tol = 1e-10 if prec == "f64" else 2e-5
    inst = _instances(fe, [4, 7, 5, 2])
    rng = np.random.default_rng(1)
    shapes = [(5, 8), (8, 8), (12, 16), (1, 4)]
    Xs, Xh, Ys = [], [], []
    for (om, V, m), (nv, ld) in zip(inst, shapes):
        buf, X = _block(rng, om.n_psi, nv, ld, dt)
        Xs.append(buf[:, :nv])
        Xh.append(X)
        Ys.append(torch.full((om.n_psi, ld), 7.0, dtype=dt, device="cuda")[:, :nv])
    b = fe.Batch([m for _, _, m in inst])
    b.apply_H(Xs, Ys, prec=P)
    for (om, V, m), X, Xg, Y, (nv, ld) in zip(inst, Xh, Xs, Ys, shapes):
        ref = assembly.hamiltonian(om, V) @ (X.astype(np.float32).astype(np.float64)
                                             if prec == "f32" else X)
        got = Y.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
        # columns past nvec are untouched
        full = Y.as_strided((om.n_psi, ld), (ld, 1))
        assert torch.all(full[:, nv:] == 7.0)
        ys = torch.zeros((om.n_psi, ld), dtype=dt, device="cuda")
        fe._lib.call("fe_apply_H", m.handle, fe._ptr(Xg), fe._ptr(ys), nv, ld, P)
        single = ys[:, :nv].double().cpu().numpy()
        assert np.linalg.norm(got - single) / np.linalg.norm(single) <= (
            1e-12 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_filter_matches_single_and_oracle(fe, prec):
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = fe.storage_dtype(P)
    inst = _instances(fe, [6, 3, 5], seed=8)
    rng = np.random.default_rng(2)
    degree = 7
    Xs, X0s, bounds = [], [], []
    for om, V, m in inst:
        H = assembly.hamiltonian(om, V)
        ev = np.linalg.eigvalsh(H.toarray())
        a0, bb = ev[0] - 0.1, ev[-1] + 0.1
        a = a0 + 0.2 * (bb - a0)
        bounds.append((a, bb, a0))
        X = rng.standard_normal((om.n_psi, 8))
        X0s.append(X)
        Xs.append(torch.tensor(X, dtype=dt, device="cuda"))
    b = fe.Batch([m for _, _, m in inst])
    singles = [x.clone() for x in Xs]
    b.cheb_filter(Xs, degree, [t[0] for t in bounds], [t[1] for t in bounds],
                  [t[2] for t in bounds], prec=P)
    for (om, V, m), X, X0, Xb, (a, bb, a0) in zip(inst, singles, X0s, Xs, bounds):
        m.cheb_filter(X, degree, a, bb, a0, prec=P)
        got = Xb.double().cpu().numpy()
        one = X.double().cpu().numpy()
        assert np.linalg.norm(got - one) / np.linalg.norm(one) <= (1e-12 if prec == "f64" else 1e-6)
        H = assembly.hamiltonian(om, V)
        Xin = X0.astype(np.float32).astype(np.float64) if prec == "f32" else X0
        ref = chefsi.cheb_filter(lambda Z: H @ Z, Xin, degree, a, bb, a0)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= (1e-10 if prec == "f64" else 2e-4)


def test_single_instance_batch_equals_mesh(fe):
    (om, V, m), = _instances(fe, [5], p=4, nx=2, seed=3)
    rng = np.random.default_rng(4)
    X = torch.tensor(rng.standard_normal((om.n_psi, 10)), device="cuda")
    b = fe.Batch([m])
    (Y,) = b.apply_H([X])
    ref = m.apply_H(X)
    assert torch.max(torch.abs(Y - ref)) <= 1e-12 * torch.max(torch.abs(ref))


def test_batch_rejects_mixed_cell_size_and_precision(fe):
    m1 = fe.Mesh((6.0, 6.0, 8.0), (3, 3, 4), 3)
    m2 = fe.Mesh((6.0, 6.0, 9.0), (3, 3, 4), 3)      # hz differs
    with pytest.raises(fe.FeError) as e:
        fe.Batch([m1, m2])
    assert e.value.status == 7
    m3 = fe.Mesh((6.0, 6.0, 8.0), (3, 3, 4), 4)      # p differs
    with pytest.raises(fe.FeError):
        fe.Batch([m1, m3])
    m1.set_potential(torch.zeros(m1.n_psi, dtype=torch.float64, device="cuda"))
    b = fe.Batch([m1])
    X = torch.zeros((m1.n_psi, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(fe.FeError) as e:
        b.apply_H([X], prec=fe.FE_BF16_F32ACC)
    assert e.value.status == 7


def test_bias_sweep_full_size_sampled_rows(fe):
    """The 24 slabs of 8 x 8 x H cells (H in [8, 40]), p = 4, 128 float vectors each, one
    degree-20 filter over the batch; the first step's H X is checked at sampled rows of
    every instance and the filtered blocks against the per-instance filter."""
    slabs = W.config4()
    rng = np.random.default_rng(12)
    meshes, Vs, X0s = [], [], []
    for s in slabs:
        m = fe.Mesh(s.L, s.ncell, s.p, s.psi_dirichlet)
        V = rng.uniform(-1.5, 0.5, m.n_psi)
        m.set_potential(torch.tensor(V, device="cuda"))
        meshes.append(m)
        Vs.append(V)
        X0s.append(W.start_block(s))
    b = fe.Batch(meshes)
    Xs = [torch.tensor(X, device="cuda") for X in X0s]
    Ys = b.apply_H(Xs, prec=fe.FE_F32)
    for s, m, V, X0, Y in zip(slabs[::5], meshes[::5], Vs[::5], X0s[::5], Ys[::5]):
        om = OMesh(s.L, s.ncell, s.p, s.psi_dirichlet)
        nxy = om.NX * om.NY
        rows = np.unique(np.concatenate([[0, nxy - 1, nxy, om.n_psi - 1],
                                         rng.choice(om.n_psi, 12, replace=False)]))
        ref = assembly.apply_H_rows(om, V, X0, rows)
        got = Y[torch.tensor(rows, device="cuda")].double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5
    a, bb, a0 = [], [], []
    for m in meshes:
        lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device="cuda"), 20)
        a0.append(lo)
        bb.append(hi)
        a.append(lo + 0.05 * (hi - lo))
    singles = [X.clone() for X in Xs]
    b.cheb_filter(Xs, 20, a, bb, a0, prec=fe.FE_F32)
    for k in (0, 7, 23):
        meshes[k].cheb_filter(singles[k], 20, a[k], bb[k], a0[k], prec=fe.FE_F32)
        d = torch.linalg.norm((Xs[k] - singles[k]).double()) / torch.linalg.norm(singles[k].double())
        assert d <= 1e-6


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_rayleigh_ritz_matches_per_instance(fe, prec):
    """Batched Cholesky-QR + Rayleigh-Ritz (batched n x n steps) against fe_rayleigh_ritz per
    instance: same Ritz values (1e-10 in FP64; 1e-6 relative with float blocks, both through
    the FP32-accurate tensor-core products), orthonormal rotated blocks whose Rayleigh
    quotients are the Ritz values."""
    P = fe.FE_F64 if prec == "f64" else fe.FE_F32
    dt = fe.storage_dtype(P)
    inst = _instances(fe, [5, 7, 4], p=3, seed=21)
    rng = np.random.default_rng(6)
    nvec = 8
    Xs = []
    for om, V, m in inst:
        m.set_rr_products(True)
        Xs.append(torch.tensor(rng.standard_normal((om.n_psi, nvec)), dtype=dt, device="cuda"))
    singles = [X.clone() for X in Xs]
    b = fe.Batch([m for _, _, m in inst])
    eb = b.rayleigh_ritz(Xs, prec=P)
    for (om, V, m), X, Xs1, e in zip(inst, Xs, singles, eb):
        es = m.rayleigh_ritz(Xs1, prec=P)
        tol = 1e-10 if prec == "f64" else 1e-6 * float(torch.max(torch.abs(es)))
        assert torch.max(torch.abs(e - es)) <= tol
        Xd = X.double().cpu().numpy()
        G = Xd.T @ Xd
        assert np.max(np.abs(G - np.eye(nvec))) <= (1e-10 if prec == "f64" else 1e-5)
        H = assembly.hamiltonian(om, V)
        rq = np.einsum("ij,ij->j", Xd, H @ Xd)
        assert np.max(np.abs(rq - e.cpu().numpy())) <= (1e-9 if prec == "f64" else 1e-4) * max(1.0, float(np.max(np.abs(rq))))


def test_batch_rayleigh_ritz_needs_tensor_core_products_for_float(fe):
    (om, V, m), = _instances(fe, [4], seed=2)
    m.set_rr_products(False)
    b = fe.Batch([m])
    X = torch.zeros((om.n_psi, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(fe.FeError) as e:
        b.rayleigh_ritz([X], prec=fe.FE_F32)
    assert e.value.status == 7


def test_batch_launch_configurations_and_tuner(fe):
    """Every launch configuration the autotuner chooses among (z-segment length x one CTA
    per item or a persistent, counter-scheduled grid) gives the same filtered blocks bit
    for bit; the tuner times them on the first call and reports its choice."""
    inst = _instances(fe, [3, 9, 6, 2, 7], p=4, nx=2, seed=13)
    rng = np.random.default_rng(14)
    X0 = [torch.tensor(rng.standard_normal((om.n_psi, 16)), dtype=torch.float32, device="cuda")
          for om, _, _ in inst]
    a, b, a0 = [4.0] * 5, [90.0] * 5, [-1.0] * 5
    outs = []
    for zseg, pers in ((0, 0), (0, 1), (2, 0), (2, 1), (4, 1), (16, 0)):
        batch = fe.Batch([m for _, _, m in inst])
        batch.set_launch(zseg, pers)
        Xs = [x.clone() for x in X0]
        batch.cheb_filter(Xs, 5, a, b, a0, prec=fe.FE_F32)
        torch.cuda.synchronize()
        assert batch.tuning()[:2] == (zseg, pers)
        outs.append(Xs)
        batch.close()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert torch.equal(x, y)
    batch = fe.Batch([m for _, _, m in inst])
    with pytest.raises(fe.FeError):
        batch.tuning()                      # nothing chosen before the first call
    Xs = [x.clone() for x in X0]
    batch.cheb_filter(Xs, 5, a, b, a0, prec=fe.FE_F32)
    zseg, pers, ms, nc = batch.tuning()
    assert zseg >= 0 and pers in (0, 1) and ms > 0 and nc >= 4
    for x, y in zip(outs[0], Xs):
        assert torch.equal(x, y)
    batch.close()
    # a second batch of the same shape takes the cached choice without timing
    batch = fe.Batch([m for _, _, m in inst])
    batch.cheb_filter([x.clone() for x in X0], 5, a, b, a0, prec=fe.FE_F32)
    assert batch.tuning()[:2] == (zseg, pers) and batch.tuning()[3] == 0
    batch.close()

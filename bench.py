#!/usr/bin/env python3
"""Benchmark of the finite-element Kohn-Sham slab hot path on GB300.

One step = one pass of the whole hot path on the p = 5 constant-field slab (16 x 16 x 48
cells, 1,529,600 psi nodes, 256 pseudo-atoms, field 0.005 Ha/bohr, 512 vectors):
  Poisson load + Jacobi-CG solve with the CEF boundary conditions and V_eff assembly,
  the degree-30 Chebyshev filter, Cholesky-QR and Rayleigh-Ritz (one more H X).
Metric: nominal cell-matrix flops (2 n_e^2 per cell per vector per H X) of all H X
applications in the step divided by the step's device time, in TFLOP/s.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
For N > 1 run under torch.distributed.run: every rank runs an independent replica on its
own GPU (the path has no data exchange between slabs), the step time is the maximum over
ranks and the value the work of all ranks over that time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

R_FILTER = 0.03          # filter cut a = a0 + 0.03 (b - a0)
POISSON_RTOL = 1e-10
LANCZOS_STEPS = 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--prec", choices=["f32", "f64", "bf16", "f32tc"], default="f32",
                    help="filter operator: f32 (CUDA cores), f64, bf16 (dense cell matrix on "
                         "the tensor cores), f32tc (sum-factorised, split-TF32 in-plane "
                         "contractions on the tensor cores, FP32-accurate)")
    ap.add_argument("--workload", choices=["p5", "p5s", "p3", "sweep", "p5nl", "scf", "p5k",
                                           "p5q", "p5qs", "p5l"],
                    default="p5",
                    help="p5: the benchmark slab; p5s / p3: smaller slabs; sweep: the batched "
                         "bias sweep of 24 independent 8x8xH-cell p=4 slabs; p5nl: the "
                         "benchmark step with synthetic nonlocal projectors on every atom; "
                         "scf: self-consistent iterations on the benchmark slab; p5k: the "
                         "benchmark step at a Bloch wave vector (complex block of the same "
                         "size); p5q: the benchmark step with the potential integrated by "
                         "Gauss quadrature (V_bare interpolated to the Gauss points); p5qs: "
                         "p5q on the p5s slab")
    ap.add_argument("--rr", choices=["f64", "tc32"], default="tc32",
                    help="Rayleigh-Ritz block products for float storage: double GEMMs or "
                         "FP32-accurate tensor-core emulation (n x n part always double)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision-conformant step, the FP64 peak probe and the "
                         "batched-sweep summary that the default run adds to its line")
    return ap.parse_args()


def workload(name):
    """p5: the benchmark slab; p5s: the same p = 5 cells and vectors with 16 cell layers and
    256 vectors (a 0.5 GB block, above L2) for profiler captures; p3: the small CEF slab."""
    if name in ("p5", "p5nl", "scf", "p5k", "p5q"):
        return W.config2()
    if name in ("p5s", "p5qs"):
        s = W.config2()
        return W.Slab(s.name.replace("96", "32") + "-short", (s.L[0], s.L[1], 32.0),
                      (16, 16, 16), 5, s.R - np.array([0.0, 0.0, 32.0]), s.Z, s.bias, nvec=256,
                      degree=s.degree, seed=s.seed)
    return W.config1()


def nominal_flops_per_hx(slab, nvec):
    ne = (slab.p + 1) ** 3
    return 2.0 * ne * ne * slab.n_cells * nvec


def workload_desc(slab):
    nx, ny, nz = slab.ncell
    return (f"{slab.name}: {nx}x{ny}x{nz} cells, p={slab.p}, {slab.n_psi:,} psi nodes, "
            f"{slab.nvec} vectors, Chebyshev degree {slab.degree}, {len(slab.R)} atoms, "
            f"{slab.bias.kind.upper()} field {slab.bias.field}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel_key, node_vectors):
    """DRAM bytes per launch from a committed ncu summary, if the kernel is unchanged, scaled
    from the record's node-vectors to this launch's (traffic grows with them: the captures
    keep the tile shape and per-CTA sweep)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel_key]
    except Exception:
        return None
    import hashlib
    src = os.path.join(ROOT, rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != rec.get("source_sha"):
        return None
    b = rec.get("bytes_per_launch")
    ref = rec.get("node_vectors")
    return b * node_vectors / ref if (b and ref) else b


class ClockSampler:
    """nvidia-smi clock and throttle-reason sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(dev):
    import torch
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if dev.index < len(ids) and ids[dev.index].strip().isdigit():
            return int(ids[dev.index])
    return dev.index if dev.index is not None else torch.cuda.current_device()


def reduce_over_ranks(dist, device, elapsed_ms, launches):
    """Replicas: the job's time is the slowest rank's, its kernel launches the sum over
    ranks (identity without a process group)."""
    if dist is None:
        return elapsed_ms, launches
    import torch
    t = torch.tensor([float(elapsed_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([int(launches)], device=device, dtype=torch.int64)
    dist.all_reduce(n)
    return float(t.item()), int(n.item())


def aggregate_value(world, flops_per_rank_step, ms_step):
    """Whole-job throughput: the work of all ranks over the slowest rank's step time."""
    return world * flops_per_rank_step / (ms_step * 1e-3) / 1e12


def _host_threads():
    return max(1, os.cpu_count() or 1)


def oracle_hx_threaded(H, X, threads):
    """The oracle's CSR product H X, its vector columns split into one contiguous block per
    host thread (scipy's sparse kernel releases the GIL, so the blocks run in parallel)."""
    from concurrent.futures import ThreadPoolExecutor
    nvec = X.shape[1]
    edges = np.linspace(0, nvec, threads + 1).astype(int)
    blocks = [(edges[i], edges[i + 1]) for i in range(threads) if edges[i + 1] > edges[i]]
    Y = np.empty((H.shape[0], nvec))

    def one(b):
        Y[:, b[0]:b[1]] = H @ np.ascontiguousarray(X[:, b[0]:b[1]])

    with ThreadPoolExecutor(len(blocks)) as ex:
        list(ex.map(one, blocks))
    return Y, len(blocks)


def cpu_model():
    """Host CPU model (lscpu's model name, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_baseline_oracle(slab, nvec, seed=5, degree=None):
    """The oracle as it stands on a 2-cell-thick slice of the same slab (bounded CPU sample):
    one CSR Ht X (the metric's unit), the degree-m scaled Chebyshev filter built on it, the
    textbook Jacobi-CG Poisson solve (CEF, relative residual 1e-10) on the slice's phi
    system, and Householder-QR + dense-eigh Rayleigh-Ritz of the filtered block."""
    from oracle import assembly, chefsi, poisson
    from oracle.mesh import Mesh as OMesh
    degree = degree or slab.degree
    nc = (slab.ncell[0], slab.ncell[1], 2)
    L = (slab.L[0], slab.L[1], 2 * slab.L[2] / slab.ncell[2])
    om = OMesh(L, nc, slab.p, slab.psi_dirichlet)
    rng = np.random.default_rng(seed)
    K = assembly.assemble_stiffness(om)
    M = assembly.lumped_mass(om)
    H = assembly.hamiltonian(om, rng.uniform(-1, 0.5, om.n_psi), K, M)
    X = rng.standard_normal((om.n_psi, nvec))
    threads = _host_threads()
    oracle_hx_threaded(H, X[:, :2 * threads], threads)
    t0 = time.perf_counter()
    _, used = oracle_hx_threaded(H, X, threads)
    dt = time.perf_counter() - t0
    hx = lambda Z: oracle_hx_threaded(H, Z, threads)[0]
    lo, hi = chefsi.lanczos_bounds(lambda v: H @ v, np.random.default_rng(31).standard_normal(
        om.n_psi), LANCZOS_STEPS)
    t0 = time.perf_counter()
    Y = chefsi.cheb_filter(hx, X, degree, lo + R_FILTER * (hi - lo), hi, lo)
    t_filter = time.perf_counter() - t0
    t0 = time.perf_counter()
    chefsi.rayleigh_ritz(hx, Y)
    t_rr = time.perf_counter() - t0
    f = M * rng.standard_normal(om.n_phi)
    t0 = time.perf_counter()
    _, cg_iters, cg_rel = poisson.solve_cef_cg(K, f, M, rtol=POISSON_RTOL)
    t_cg = time.perf_counter() - t0
    ne = (slab.p + 1) ** 3
    flops = 2.0 * ne * ne * om.n_cells * nvec
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": used, "kind": "oracle",
            "cpu_model": cpu_model(), "host_threads": threads,
            "sample": (f"oracle on a {nc[0]}x{nc[1]}x{nc[2]}-cell slice of the slab (p={slab.p}, "
                       f"{om.n_psi:,} psi nodes x {nvec} vectors, {om.n_phi:,} phi nodes): "
                       f"scipy CSR Ht X with the vector columns split over {used} host "
                       f"threads (value), the degree-{degree} filter on it, Householder-QR + "
                       "eigh Rayleigh-Ritz, and Jacobi-CG of the CEF Poisson system (one "
                       "thread, scipy)"),
            "seconds": {"hx": dt, "filter": t_filter, "rayleigh_ritz": t_rr,
                        "poisson_cg": t_cg},
            "poisson_cg_iterations": int(cg_iters), "poisson_cg_rel_residual": float(cg_rel)}


def fp64_gemm_peak(dev, n=8192, reps=5):
    """Measured FP64 peak for the FP64 path's roofline: cuBLAS DGEMM n^3 (torch.matmul on
    float64), best of reps, CUDA events."""
    import torch
    a = torch.randn((n, n), dtype=torch.float64, device=dev)
    b = torch.randn((n, n), dtype=torch.float64, device=dev)
    c = torch.matmul(a, b)
    best = float("inf")
    st = torch.cuda.current_stream(dev)
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        torch.matmul(a, b, out=c)
        e1.record(st)
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def sumfact_flops_per_hx(slab, nvec):
    """Arithmetic of the sum-factorised operator: per node-vector seven assembled 1D
    contractions (y: M1 and K1; x: M1 on both, K1 on one; z: M1 and K1), each with the
    average tap count of an assembled GLL line (p + 1 taps at p - 1 interior nodes of a
    cell segment, 2p + 1 at the shared node: (p (p + 1) + p) / p per node), plus the
    potential and the two-term Chebyshev update: 2 flops per FMA."""
    p = slab.p
    taps = (p * (p + 1) + p) / p
    return 2.0 * (7.0 * taps + 3.0) * slab.n_psi * nvec


# ------------------------------------------------------------------------------------------
def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    slab = workload(args.workload)
    from oracle import assembly
    from oracle.mesh import Mesh as OMesh
    nc = (slab.ncell[0], slab.ncell[1], 2)
    L = (slab.L[0], slab.L[1], 2 * slab.L[2] / slab.ncell[2])
    om = OMesh(L, nc, slab.p, slab.psi_dirichlet)
    rng = np.random.default_rng(5)
    H = assembly.hamiltonian(om, rng.uniform(-1, 0.5, om.n_psi))
    nvec = slab.nvec
    X = rng.standard_normal((om.n_psi, nvec))
    ne = (slab.p + 1) ** 3
    flops = 2.0 * ne * ne * om.n_cells * nvec
    threads = _host_threads()
    for _ in range(args.warmup):
        oracle_hx_threaded(H, X, threads)
    t0 = time.perf_counter()
    used = threads
    for _ in range(args.steps):
        _, used = oracle_hx_threaded(H, X, threads)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    val = flops / dt / 1e12
    sample = (f"one oracle scipy CSR Ht X per step on a {nc[0]}x{nc[1]}x{nc[2]}-cell slice of "
              f"the slab (p={slab.p}, {om.n_psi:,} psi nodes x {nvec} vectors), vector "
              f"columns split over {used} host threads")
    line = {
        "impl": "reference", "metric": "Cheb-filter H·X nominal TFLOP/s", "value": val,
        "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(slab), "sample": sample},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def conformant_step(m, slab, X0, a, b, a0, phi_mixed, flops_step, dev, fe):
    """One step in the arithmetic the method's precision contract states: the filter's
    operator in FP32, Cholesky-QR / Rayleigh-Ritz block products in FP64 (double GEMMs on a
    double copy of the block), the Poisson CG in FP64 throughout.  Timed once from the
    benchmark's start block, after one untimed step; its Ritz values and potential are
    compared with the default (fast) configuration's from the same start block."""
    import torch
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    nvec = slab.nvec
    phi = torch.empty(m.n_phi, dtype=torch.float64, device=dev)
    vb = torch.empty(m.n_psi, dtype=torch.float64, device=dev)

    def one(rec):
        X = X0.to(dev)
        e = [ev() for _ in range(4)]
        e[0].record(st)
        _, _, info = m.poisson_solve(slab.bias, rtol=POISSON_RTOL, phi=phi, vbare=vb)
        m.set_potential(vb)
        e[1].record(st)
        m.cheb_filter(X, slab.degree, a, b, a0, prec=fe.FE_F32)
        e[2].record(st)
        eig = m.rayleigh_ritz(X, prec=fe.FE_F32)
        e[3].record(st)
        torch.cuda.synchronize(dev)
        return eig.cpu().numpy(), info, [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]),
                                         e[2].elapsed_time(e[3])]

    # the default configuration's Ritz values from the same start block
    eig_fast, _, _ = one(False)
    m.set_poisson_mixed(False)
    m.set_rr_products(False)
    try:
        one(False)
        eig_c, info, ph = one(True)
        phi_c = phi.clone()
    finally:
        m.set_poisson_mixed(True)
        m.set_rr_products(True)
    ms = sum(ph)
    k = min(int(slab.n_electrons // 2), nvec - 8)
    dphi = float((phi_c - phi_mixed).abs().max() / phi_c.abs().max())
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": flops_step / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "arithmetic": "Poisson CG in FP64; filter operator FP32; Cholesky-QR and "
                          "Rayleigh-Ritz block products and n x n part in FP64",
            "phases_ms": {"poisson_and_veff": ph[0], "cheb_filter": ph[1], "cholqr_rr": ph[2]},
            "poisson_iterations": info.iters,
            "phi_max_rel_diff_vs_mixed_cg": dphi,
            "eig_max_diff_vs_default_ha": float(np.max(np.abs(eig_c[:k] - eig_fast[:k]))),
            "eig_count": k}


def filter_variants(m, slab, X, phi, a, b, a0, dev, fe):
    """The benchmark slab's degree-m filter with the operator variants of the method, each
    timed (after one untimed filter) with CUDA events on the mesh stream: the Bloch k-point
    Hamiltonian at k = (0.1, 0.05) / bohr on the same block read as nvec / 2 complex
    vectors, and the potential integrated by Gauss quadrature.  Nominal flops as the
    metric's (the collocated operator's cell-matrix count on nvec lanes)."""
    import torch
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    nvec, degree = slab.nvec, slab.degree
    flops = nominal_flops_per_hx(slab, nvec) * degree
    out = {}

    def timed(blk):
        m.cheb_filter(blk, degree, a, b, a0, prec=fe.FE_F32)
        e0, e1 = ev(), ev()
        e0.record(st)
        m.cheb_filter(blk, degree, a, b, a0, prec=fe.FE_F32)
        e1.record(st)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    Xw = X.clone()
    try:
        m.set_kpoint(0.1, 0.05)
        ms = timed(torch.view_as_complex(Xw.view(m.n_psi, nvec // 2, 2)))
        out["kpoint_filter"] = {"ms": ms, "ms_per_hx": ms / degree,
                                "tflops": flops / (ms * 1e-3) / 1e12,
                                "workload": f"k = (0.1, 0.05) / bohr, {nvec // 2} complex vectors"}
    finally:
        m.set_kpoint(0.0, 0.0)
    vb = torch.empty(m.n_psi, dtype=torch.float64, device=dev)
    _, _, _ = m.poisson_solve(slab.bias, rtol=POISSON_RTOL, phi=phi, vbare=vb)
    try:
        m.set_potential_quad(m.interp_quad(m.vbare_phi(phi, slab.bias)))
        Xw.copy_(X)
        ms = timed(Xw)
        out["quadrature_filter"] = {"ms": ms, "ms_per_hx": ms / degree,
                                    "tflops": flops / (ms * 1e-3) / 1e12,
                                    "workload": f"V_bare at the {slab.p + 1}^3 Gauss points of "
                                                "every cell"}
    finally:
        m.set_potential(vb)
    del Xw
    torch.cuda.empty_cache()
    return out


def sweep_measure(steps, warmup):
    """Batched bias sweep: 24 independent slabs of 8 x 8 x H cells (p = 4, 128 vectors),
    half under a constant field and half under a constrained potential difference, stepped
    together.  One step = the degree-20 Chebyshev filter of every slab as batched launches
    (one kernel per filter step over all instances) and the batched Cholesky-QR /
    Rayleigh-Ritz of all slabs.  The Poisson solves that give each slab's V_eff run once
    before timing.  Returns the measurements (and the clock summary)."""
    import torch
    import paper_2504_00998_gb300 as fe

    dev = torch.device("cuda", torch.cuda.current_device())
    lib = fe.load()
    slabs = W.config4()
    meshes, Xs, bounds = [], [], []
    for sl in slabs:
        m = fe.Mesh.from_slab(sl, device=dev.index)
        m.set_rr_products(True)   # the batched Rayleigh-Ritz of float blocks needs them
        _, vb, _ = m.poisson_solve(sl.bias, rtol=POISSON_RTOL)
        m.set_potential(vb)
        lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device=dev),
                                  LANCZOS_STEPS)
        bounds.append((lo + R_FILTER * (hi - lo), hi, lo))
        meshes.append(m)
        Xs.append(torch.from_numpy(W.start_block(sl)).to(dev))
    batch = fe.Batch(meshes)
    degree = slabs[0].degree
    a = [t[0] for t in bounds]
    b = [t[1] for t in bounds]
    a0 = [t[2] for t in bounds]
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    fl, rr = [], []

    def step(rec):
        e = [ev() for _ in range(3)]
        e[0].record(st)
        batch.cheb_filter(Xs, degree, a, b, a0, prec=fe.FE_F32)
        e[1].record(st)
        batch.rayleigh_ritz(Xs, prec=fe.FE_F32)
        e[2].record(st)
        if rec:
            fl.append((e[0], e[1]))
            rr.append((e[1], e[2]))

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize(dev)
    n0 = lib.fe_kernel_launches()
    t0, t1 = ev(), ev()
    with ClockSampler(gpu_index(dev)) as clk:
        t0.record(st)
        for _ in range(steps):
            step(True)
        t1.record(st)
        torch.cuda.synchronize(dev)
    launches = lib.fe_kernel_launches() - n0
    ms_step = t0.elapsed_time(t1) / steps
    f_ms = sum(x.elapsed_time(y) for x, y in fl) / len(fl)
    r_ms = sum(x.elapsed_time(y) for x, y in rr) / len(rr)
    nvec = slabs[0].nvec
    flops_hx = sum(nominal_flops_per_hx(sl, nvec) for sl in slabs)
    value = flops_hx * (degree + 1) / (ms_step * 1e-3) / 1e12
    n_all = sum(mm.n_psi for mm in meshes)
    bytes_filter = (2 + 3 * (degree - 1)) * n_all * nvec * 4 + degree * n_all * 4
    achieved = bytes_filter / degree / (f_ms / degree * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    heights = [sl.ncell[2] for sl in slabs]
    batch.close()
    for mm in meshes:
        mm.close()
    del Xs
    torch.cuda.empty_cache()
    return {
        "value": value, "unit": "TFLOP/s", "ms_per_step": ms_step, "steps": steps,
        "warmup": warmup,
        "workload": (f"bias sweep: {len(slabs)} slabs of 8x8xH cells, H from {min(heights)} to "
                     f"{max(heights)}, p=4, {n_all:,} psi nodes in all, {nvec} vectors each, "
                     f"Chebyshev degree {degree}, 12 CEF + 12 CPD"),
        "l2": "inputs larger than L2 (blocks of %.1f GB in all)" % (n_all * nvec * 4 / 1e9),
        "phases_ms": {"batched_cheb_filter": f_ms, "batched_cholqr_rr": r_ms},
        "filter_tflops": flops_hx * degree / (f_ms * 1e-3) / 1e12,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "kernel": "kron_batch_f32_p4",
                     "algorithmic_bytes_per_launch": bytes_filter / degree,
                     "launch_ms": f_ms / degree},
        "gpu_launches": launches, "clocks": clk.summary()}


# ------------------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import paper_2504_00998_gb300 as fe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"f32": fe.FE_F32, "f64": fe.FE_F64, "bf16": fe.FE_BF16_F32ACC,
            "f32tc": fe.FE_F32_F32ACC}[args.prec]
    dtype_name = {"f32": "f32", "f64": "f64", "bf16": "bf16", "f32tc": "f32 (split tf32)"}[args.prec]
    slab = workload(args.workload)
    nvec, degree = slab.nvec, slab.degree
    lib = fe.load()

    m = fe.Mesh.from_slab(slab, device=local)
    if prec != fe.FE_F64:
        m.set_rr_products(args.rr == "tc32")
    nl_desc = ""
    if args.workload == "p5k":
        # Bloch wave vector k = (0.1, 0.05) / bohr: the block is complex (the same bytes as
        # the Gamma-point block: nvec / 2 complex vectors)
        m.set_kpoint(0.1, 0.05)
        nl_desc = f" at k = (0.1, 0.05) / bohr with {slab.nvec // 2} complex vectors"
    if args.workload == "p5nl":
        # synthetic s + p projectors on every atom (the stand-in for the pseudopotentials'
        # nonlocal part): width 0.8 bohr, cut at 2.6 bohr, D = (1.0, 0.4, 0.4, 0.4) Ha
        na = len(slab.R)
        m.set_nonlocal(slab.R, np.full(na, 0.8), np.tile([1.0, 0.4, 0.4, 0.4], (na, 1)), 2.6)
        nl_desc = f" + synthetic s,p nonlocal projectors on all {na} atoms (sigma 0.8, cut 2.6 bohr)"
    quad = args.workload in ("p5q", "p5qs")
    if quad:
        nl_desc = (f" with the potential integrated by {slab.p + 1}^3-point Gauss quadrature "
                   "(V_bare interpolated to the Gauss points)")
    phi = torch.empty(m.n_phi, dtype=torch.float64, device=dev)
    vb = torch.empty(m.n_psi, dtype=torch.float64, device=dev)

    def set_pot():
        # V_eff at the psi nodes (collocated), or at every cell's Gauss points
        if quad:
            m.set_potential_quad(m.interp_quad(m.vbare_phi(phi, slab.bias)))
        else:
            m.set_potential(vb)

    m.poisson_solve(slab.bias, rtol=POISSON_RTOL, phi=phi, vbare=vb)
    set_pot()
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device=dev), LANCZOS_STEPS)
    a0, b = lo, hi
    a = a0 + R_FILTER * (b - a0)

    X0 = torch.from_numpy(W.start_block(slab)).pin_memory()
    X = torch.empty((m.n_psi, nvec), dtype=fe.storage_dtype(prec), device=dev)
    # the block the step works on: X itself, or its complex view at a Bloch wave vector
    blk = torch.view_as_complex(X.view(m.n_psi, nvec // 2, 2)) if args.workload == "p5k" else X
    X.copy_(X0.to(X.dtype) if X.dtype != X0.dtype else X0)
    st = torch.cuda.current_stream(dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    marks = []

    pinfo = {}

    def step(rec):
        e = [ev() for _ in range(5)] if rec else None
        if rec:
            e[0].record(st)
        _, _, info = m.poisson_solve(slab.bias, rtol=POISSON_RTOL, phi=phi, vbare=vb)
        pinfo["iters"], pinfo["rel_residual"] = info.iters, info.rel_residual
        if rec:
            e[1].record(st)
        set_pot()
        if rec:
            e[2].record(st)
        m.cheb_filter(blk, degree, a, b, a0, prec=prec)
        if rec:
            e[3].record(st)
        eig = m.rayleigh_ritz(blk, prec=prec)
        if rec:
            e[4].record(st)
            marks.append(e)
        return eig

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    n0 = lib.fe_kernel_launches()
    t_start, t_end = ev(), ev()
    with ClockSampler(gpu_index(dev)) as clk:
        t_start.record(st)
        for _ in range(args.steps):
            torch.cuda.nvtx.range_push("timed_step")   # lets a profiler select one step
            eig = step(True)
            torch.cuda.nvtx.range_pop()
        t_end.record(st)
        torch.cuda.synchronize(dev)
    launches = lib.fe_kernel_launches() - n0
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms, launches = reduce_over_ranks(dist, dev, elapsed_ms, launches)
    if dist:
        dist.barrier()
    phase = np.zeros(4)
    for e in marks:
        phase += [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3]),
                  e[3].elapsed_time(e[4])]
    phase /= max(len(marks), 1)
    ms_step = elapsed_ms / args.steps
    flops_hx = nominal_flops_per_hx(slab, nvec)
    flops_step = flops_hx * (degree + 1)
    value = aggregate_value(world, flops_step, ms_step)

    # roofline of the dominant kernel: the fused Chebyshev operator launch
    eb = 8 if prec == fe.FE_F64 else 4
    n = m.n_psi
    bytes_filter = (2 + 3 * (degree - 1)) * n * nvec * eb + degree * n * eb
    bytes_per_launch = bytes_filter / degree
    launch_ms = phase[2] / degree
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    kernel_key = {fe.FE_F32: "kron_f32_p5", fe.FE_F64: "kron_f64_p5",
                  fe.FE_F32_F32ACC: "ktc_f32_p5"}.get(prec, "tc_p5")
    # (the nonlocal term adds its own kernels to the filter time: no single-kernel traffic)
    traffic = traffic_record(kernel_key, n * nvec) if not nl_desc else None

    # end to end through the public API with host buffers.  Every step copies its input block
    # in from pinned host memory (3.1 GB on the benchmark slab) and reads its result back.
    # The step's result is what a subspace iteration hands back to its caller: the Ritz values
    # (the filtered, rotated block is the iteration's device-resident state, fed to the next
    # step).  The input is the block as it stands after the timed steps (the state a device
    # step starts from, so both loops do the same numerical work); it streams in on a copy
    # stream into one of two device blocks while the previous step runs (the first step's
    # under its Poisson solve, which reads no block), and the filter waits for it.  A second
    # leg also reads the whole block back every step (two device blocks alternate; a step's
    # block leaves while the next step's filter runs, the last one after the last step, inside
    # the timed region; its input copy waits for that read-back, so it streams in under the
    # step's Poisson solve) and is reported beside it.
    Xh = X.cpu().pin_memory()
    eig_h = torch.empty(blk.shape[1], dtype=torch.float64).pin_memory()
    Xbuf = [X, torch.empty_like(X)]
    views = [torch.view_as_complex(b.view(m.n_psi, nvec // 2, 2)) if args.workload == "p5k"
             else b for b in Xbuf]
    cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_leg(read_block):
        outs = [torch.empty_like(Xh).pin_memory() for _ in range(2)] if read_block else None
        out_done = [None, None]
        pending, marks, d2h = [], [], []
        nsteps = max(1, min(args.steps, 3))

        def read_back(j, fin, eig, after=None):
            cout.wait_event(fin)
            if after is not None:
                cout.wait_event(after)
            with torch.cuda.stream(cout):
                start = ev()
                start.record(cout)
                if read_block:
                    outs[j].copy_(Xbuf[j], non_blocking=True)
                eig_h.copy_(eig, non_blocking=True)
                eig.record_stream(cout)
                done = ev()
                done.record(cout)
            out_done[j] = done
            d2h.append((start, done))

        # Without the block read-back, step k's input goes to device buffer k % 2 and is
        # copied in while step k - 1 runs: it waits only for step k - 2, the buffer's last
        # user (one copy stream, so the copies arrive in step order).
        h2d = {}
        fins = {}

        def copy_in(k):
            jj = k % 2
            if k >= 2:
                cin.wait_event(fins[k - 2])
            start, arr = ev(), ev()
            with torch.cuda.stream(cin):
                start.record(cin)
                Xbuf[jj].copy_(Xh, non_blocking=True)
                arr.record(cin)
            h2d[k] = (start, arr)

        def step(i):
            j = i % 2
            e = [ev() for _ in range(5)]
            if read_block:
                arrived = ev()
                cin.wait_stream(st)
                if out_done[j] is not None:
                    cin.wait_event(out_done[j])
                with torch.cuda.stream(cin):
                    e[0].record(cin)
                    Xbuf[j].copy_(Xh, non_blocking=True)
                    arrived.record(cin)
            else:
                if i == 0:
                    cin.wait_stream(st)
                    copy_in(0)
                if i + 1 < nsteps:
                    copy_in(i + 1)
                e[0], arrived = h2d[i]
            e[1].record(st)
            m.poisson_solve(slab.bias, rtol=POISSON_RTOL, phi=phi, vbare=vb)
            set_pot()
            e[2].record(st)
            if pending:
                pj, pfin, peig = pending.pop()
                read_back(pj, pfin, peig, after=e[2])
            st.wait_event(arrived)
            e[3].record(st)
            m.cheb_filter(views[j], degree, a, b, a0, prec=prec)
            e[4].record(st)
            eig = m.rayleigh_ritz(views[j], prec=prec)
            fin = ev()
            fin.record(st)
            fins[i] = fin
            if read_block:
                pending.append((j, fin, eig))
            else:
                read_back(j, fin, eig)
            marks.append((e, arrived, fin))

        torch.cuda.synchronize(dev)
        t0, t1 = ev(), ev()
        t0.record(st)
        for i in range(nsteps):
            step(i)
        if pending:
            pj, pfin, peig = pending.pop()
            read_back(pj, pfin, peig)
        st.wait_stream(cout)
        st.wait_stream(cin)
        t1.record(st)
        torch.cuda.synchronize(dev)
        ms = t0.elapsed_time(t1) / nsteps
        ph = {"h2d": 0.0, "poisson_and_veff": 0.0, "wait_for_input": 0.0, "cheb_filter": 0.0,
              "cholqr_rr": 0.0}
        for e, arrived, fin in marks:
            ph["h2d"] += e[0].elapsed_time(arrived)
            ph["poisson_and_veff"] += e[1].elapsed_time(e[2])
            ph["wait_for_input"] += e[2].elapsed_time(e[3])
            ph["cheb_filter"] += e[3].elapsed_time(e[4])
            ph["cholqr_rr"] += e[4].elapsed_time(fin)
        ph = {k: v / max(len(marks), 1) for k, v in ph.items()}
        ph["d2h"] = sum(x.elapsed_time(y) for x, y in d2h) / max(len(d2h), 1)
        ok = True
        if read_block:
            last = (nsteps - 1) % 2
            ok = bool(torch.equal(outs[last], Xbuf[last].cpu()))
        return ms, ph, ok

    e2e_ms, e2e_phases, _ = e2e_leg(False)
    e2e_ms, _ = reduce_over_ranks(dist, dev, e2e_ms, 0)
    e2e_val = aggregate_value(world, flops_step, e2e_ms)
    blk_ms, blk_phases, e2e_result_ok = e2e_leg(True)
    blk_ms, _ = reduce_over_ranks(dist, dev, blk_ms, 0)
    del Xbuf[1], views
    torch.cuda.empty_cache()

    extra = {}
    if (rank == 0 and world == 1 and not args.no_fp64_compare and prec != fe.FE_F64
            and args.workload != "p5k"):
        # one cycle of both paths from the same start block: Ritz-value difference and the
        # FP64 filter's throughput
        # two cycles (the second starts from an orthonormal block, as in an SCF loop)
        Xm = torch.empty((n, nvec), dtype=fe.storage_dtype(prec), device=dev)
        Xm.copy_(X0.to(Xm.dtype))
        for _ in range(2):
            m.cheb_filter(Xm, degree, a, b, a0, prec=prec)
            ev_m = m.rayleigh_ritz(Xm, prec=prec).cpu().numpy()
        del Xm
        Xd = X0.to(dev).double()
        f0, f1 = ev(), ev()
        for cyc in range(2):
            if cyc == 1:
                f0.record(st)
            m.cheb_filter(Xd, degree, a, b, a0, prec=fe.FE_F64)
            if cyc == 1:
                f1.record(st)
            ev_d = m.rayleigh_ritz(Xd, prec=fe.FE_F64).cpu().numpy()
        torch.cuda.synchronize(dev)
        fms = f0.elapsed_time(f1)
        del Xd
        k = min(int(slab.n_electrons // 2), nvec - 8)
        extra = {"fp64_filter_ms": fms,
                 "fp64_filter_tflops": flops_hx * degree / (fms * 1e-3) / 1e12,
                 "eig_err_vs_fp64_ha": float(np.max(np.abs(ev_m[:k] - ev_d[:k]))),
                 "eig_err_count": k}
        if not args.no_extras:
            # the FP64 operator is bound by the FP64 pipes: its roofline is its own
            # arithmetic (the sum-factorised flops) against a DGEMM measured here
            pk64 = fp64_gemm_peak(dev)
            hw = sumfact_flops_per_hx(slab, nvec) * degree / (fms * 1e-3) / 1e12
            extra["fp64_roofline"] = {
                "bound": "fp64", "achieved": hw, "peak": pk64, "unit": "TFLOP/s",
                "frac": hw / pk64, "peak_source": "measured in this run: cuBLAS DGEMM 8192^3",
                "flops": "sum-factorised operator arithmetic: 2 (7 (p + 2) + 3) per node-vector"}
        torch.cuda.empty_cache()

    conformant = None
    if (rank == 0 and world == 1 and not args.no_extras and prec == fe.FE_F32
            and args.workload == "p5"):
        conformant = conformant_step(m, slab, X0, a, b, a0, phi, flops_step, dev, fe)
    sweep = None
    variants = {}
    scf = None
    large = None
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "p5":
        variants = filter_variants(m, slab, X, phi, a, b, a0, dev, fe)
        sweep = sweep_measure(max(2, min(args.steps, 3)), 2)
        scf = scf_measure(2, 1)
        large = large_measure(1, 1)

    cpu = None
    if (rank == 0 and world == 1 and not args.no_cpu_baseline
            and args.workload not in ("p5k", "p5q", "p5qs")):
        cpu = cpu_baseline_oracle(slab, nvec)

    if rank == 0:
        line = {
            "metric": "Cheb-filter H·X nominal TFLOP/s", "value": value, "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
            "config": {"workload": workload_desc(slab) + nl_desc,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (block of %.1f GB)" % (n * nvec * eb / 1e9),
                       "rr_products": args.rr if prec != fe.FE_F64 else "f64",
                       "filter_bounds": {"a0": a0, "a": a, "b": b}},
            "phases_ms": {"poisson_and_veff": phase[0], "set_potential": phase[1],
                          "cheb_filter": phase[2], "cholqr_rr": phase[3]},
            "filter_tflops": flops_hx * degree / (phase[2] * 1e-3) / 1e12,
            "poisson": {"iterations": pinfo.get("iters"), "rel_residual": pinfo.get("rel_residual"),
                        "rtol": POISSON_RTOL},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src, "kernel": kernel_key,
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "launch_ms": launch_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(X0.numel() * X.element_size()),
                    "d2h_bytes_per_step": int(blk.shape[1] * 8),
                    "result": "the Ritz values read back every step (the filtered, rotated "
                              "block is the iteration's device-resident state)",
                    "phases_ms": e2e_phases,
                    "with_block_readback": {
                        "value": aggregate_value(world, flops_step, blk_ms), "unit": "TFLOP/s",
                        "ms_per_step": blk_ms,
                        "d2h_bytes_per_step": int(X0.numel() * X.element_size() + blk.shape[1] * 8),
                        "phases_ms": blk_phases, "result_matches_device": e2e_result_ok}},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        line.update(extra)
        if conformant is not None:
            line["conformant"] = conformant
        if sweep is not None:
            variants["sweep"] = sweep
        if scf is not None:
            variants["scf"] = scf
        if large is not None:
            variants["large_lcpd"] = large
        if variants:
            line["variants"] = variants
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    m.close()
    return 0


def run_sweep(args):
    """The batched bias sweep as its own benchmark line (see sweep_measure)."""
    import torch
    torch.cuda.set_device(0)
    r = sweep_measure(args.steps, args.warmup)
    line = {
        "metric": "Cheb-filter H·X nominal TFLOP/s", "value": r["value"], "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": r["workload"],
                   "parallelism": "single GPU, one batched launch per filter step",
                   "l2": r["l2"], "rr_products": "tc32"},
        "phases_ms": r["phases_ms"], "filter_tflops": r["filter_tflops"],
        "roofline": r["roofline"], "cpu_baseline": None, "e2e": None,
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
    }
    print(json.dumps(line))
    return 0


def scf_measure(steps, warmup):
    """Self-consistent iterations on the benchmark slab (Hartree level, CEF bias): the time
    of one iteration (Poisson, V_eff, Lanczos bounds, one filter + Rayleigh-Ritz cycle,
    occupations, density, Anderson mixing).  A run of 1 + K iterations and a run of one
    iteration are timed (after warm-up runs); their difference over K excludes each run's
    set-up (model density, mixer)."""
    import torch
    import paper_2504_00998_gb300 as fe
    from paper_2504_00998_gb300 import scf as fscf
    dev = torch.device("cuda", 0)
    slab = W.config2()
    m = fe.Mesh.from_slab(slab, device=0)
    m.set_rr_products(True)
    X = torch.tensor(W.start_block(slab), device=dev)
    n_e = float(np.sum(slab.Z))
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(iters):
        t0, t1 = ev(), ev()
        torch.cuda.synchronize(dev)
        t0.record(st)
        out = fscf.scf_run(m, slab.bias, n_e, X, iters=iters, degree=slab.degree,
                           prec=fe.FE_F32, rtol=POISSON_RTOL, first_cycles=1)
        t1.record(st)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1), out

    for _ in range(max(warmup, 1)):
        timed(1)
    t1_ms, _ = timed(1)
    tk_ms, out = timed(1 + steps)
    ms = (tk_ms - t1_ms) / steps
    m.close()
    return {"ms_per_iteration": ms, "steps": steps, "warmup": max(warmup, 1),
            "workload": workload_desc(slab) + "; Hartree-level self-consistent iterations",
            "run_ms": {"1": t1_ms, str(1 + steps): tk_ms},
            "mixing_residuals": out["res"], "mu": out["mu"]}


def run_scf(args):
    """The SCF iteration time as its own benchmark line (see scf_measure)."""
    import torch
    torch.cuda.set_device(0)
    r = scf_measure(args.steps, args.warmup)
    print(json.dumps({
        "metric": "SCF iteration time", "value": r["ms_per_iteration"], "unit": "ms",
        "n_gpus": 1, "steps": r["steps"], "warmup": r["warmup"],
        "ms_per_step": r["ms_per_iteration"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "parallelism": "single GPU"},
        "run_ms": r["run_ms"], "mixing_residuals": r["mixing_residuals"], "mu": r["mu"]}))
    return 0


def large_measure(steps, warmup):
    """The large L-CPD slab (48 x 48 x 144 bohr, 24 x 24 x 72 cells, p = 5, 2048 atoms,
    1024 vectors).  One step = the L-CPD Poisson solve and V_eff, the degree-40 Chebyshev
    filter of the 1024-wide float array as four 256-vector blocks (each block a column slice,
    leading dimension 1024), and Rayleigh-Ritz over all 1024 vectors.  Returns the
    measurements."""
    import torch
    import paper_2504_00998_gb300 as fe

    dev = torch.device("cuda", torch.cuda.current_device())
    lib = fe.load()
    slab = W.config5()
    nvec, degree, nb = slab.nvec, slab.degree, 256
    m = fe.Mesh.from_slab(slab, device=dev.index)
    m.set_rr_products(True)
    phi = torch.empty(m.n_phi, dtype=torch.float64, device=dev)
    vb = torch.empty(m.n_psi, dtype=torch.float64, device=dev)
    m.poisson_solve(slab.bias, rtol=POISSON_RTOL, max_iter=40000, phi=phi, vbare=vb)
    m.set_potential(vb)
    lo, hi = m.lanczos_bounds(torch.tensor(W.lanczos_start(m.n_psi), device=dev), LANCZOS_STEPS)
    a = lo + R_FILTER * (hi - lo)
    X = torch.empty((m.n_psi, nvec), dtype=torch.float32, device=dev)
    for j in range(nvec // nb):
        X[:, nb * j:nb * (j + 1)].copy_(
            torch.from_numpy(W.start_block(slab, nvec=nb, seed=2005 + j)))
    blocks = [X[:, nb * j:nb * (j + 1)] for j in range(nvec // nb)]
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    marks, pinfo = [], {}

    def step(rec):
        e = [ev() for _ in range(4)]
        e[0].record(st)
        _, _, info = m.poisson_solve(slab.bias, rtol=POISSON_RTOL, max_iter=40000, phi=phi,
                                     vbare=vb)
        pinfo["iters"], pinfo["rel_residual"] = info.iters, info.rel_residual
        m.set_potential(vb)
        e[1].record(st)
        for xb in blocks:
            m.cheb_filter(xb, degree, a, hi, lo, prec=fe.FE_F32)
        e[2].record(st)
        eig = m.rayleigh_ritz(X, prec=fe.FE_F32)
        e[3].record(st)
        if rec:
            marks.append(e)
        return eig

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize(dev)
    n0 = lib.fe_kernel_launches()
    t0, t1 = ev(), ev()
    with ClockSampler(gpu_index(dev)) as clk:
        t0.record(st)
        for _ in range(steps):
            eig = step(True)
        t1.record(st)
        torch.cuda.synchronize(dev)
    launches = lib.fe_kernel_launches() - n0
    ms_step = t0.elapsed_time(t1) / steps
    ph = np.mean([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
                  for e in marks], axis=0)
    n = m.n_psi
    flops_hx = nominal_flops_per_hx(slab, nvec)
    value = flops_hx * (degree + 1) / (ms_step * 1e-3) / 1e12
    # the dominant kernel: one fused operator launch on one 256-vector block
    bytes_launch = ((2 + 3 * (degree - 1)) * n * nb * 4 + degree * n * 4) / degree
    launch_ms = ph[1] / (degree * len(blocks))
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    theta = eig.cpu().numpy()
    out = {
        "value": value, "unit": "TFLOP/s", "ms_per_step": ms_step, "steps": steps,
        "warmup": warmup,
        "workload": (workload_desc(slab) + f"; the 1024-wide float array filtered as "
                     f"{len(blocks)} blocks of {nb} vectors (leading dimension {nvec}), "
                     f"Rayleigh-Ritz over all {nvec}"),
        "l2": "inputs larger than L2 (a %.1f GB array, %.1f GB per block)"
              % (n * nvec * 4 / 1e9, n * nb * 4 / 1e9),
        "phases_ms": {"poisson_and_veff": ph[0], "cheb_filter_4_blocks": ph[1],
                      "cholqr_rr": ph[2]},
        "poisson": {"iterations": pinfo["iters"], "rel_residual": pinfo["rel_residual"],
                    "rtol": POISSON_RTOL, "bias": "L-CPD (constrained 12 x 12 bohr patch)"},
        "filter_tflops": flops_hx * degree / (ph[1] * 1e-3) / 1e12,
        "ritz_range_ha": [float(theta[0]), float(theta[-1])],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "kernel": "kron_f32_p5 (256-vector block, leading dimension 1024)",
                     "algorithmic_bytes_per_launch": bytes_launch, "launch_ms": launch_ms},
        "gpu_launches": launches, "clocks": clk.summary()}
    m.close()
    del X, blocks
    torch.cuda.empty_cache()
    return out


def run_large(args):
    """The large L-CPD slab as its own benchmark line (see large_measure)."""
    import torch
    torch.cuda.set_device(0)
    r = large_measure(args.steps, args.warmup)
    print(json.dumps({
        "metric": "Cheb-filter H·X nominal TFLOP/s", "value": r["value"], "unit": "TFLOP/s",
        "n_gpus": 1, "steps": r["steps"], "warmup": r["warmup"],
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "parallelism": "single GPU", "l2": r["l2"],
                   "rr_products": "tc32"},
        "phases_ms": r["phases_ms"], "poisson": r["poisson"],
        "filter_tflops": r["filter_tflops"], "ritz_range_ha": r["ritz_range_ha"],
        "roofline": r["roofline"], "cpu_baseline": None, "e2e": None,
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "scf":
        return run_scf(args)
    if args.workload == "p5l":
        return run_large(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

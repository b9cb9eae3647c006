"""Seeded synthetic slab workloads shared by the oracle, the tests and the benchmark.

This module only lays out inputs: box and mesh sizes, pseudo-atom positions and
charges, bias settings and random start blocks.  It contains none of the finite-element
arithmetic, so the CPU oracle and the CUDA path can both draw from it without sharing
any of the method.

The slabs stand in for the paper's LLZO / GaAs / Al systems (Section 3), which need
real structures and ONCV pseudopotentials: each slab is a stack of jittered square or
rectangular pseudo-atom lattices centred in a vacuum-padded box, periodic in x/y and
finite in z.  Units are Hartree atomic units (bohr, Ha).

Recipe (all positions from ``numpy.random.default_rng(1000 + config index)``, jitter
uniform in [-0.2, 0.2] bohr per coordinate; random start blocks from
``default_rng(2000 + config index)`` as float32 N(0, 1) draws):

==== ================ ====== =================================================== =====================
cfg  box (bohr)       cells  layers                                              bias
==== ================ ====== =================================================== =====================
1    12 x 12 x 36     6x6x16 2 x (4x2, 3 x 6 bohr), z = 16.5, 19.5               CEF E = 0.01
2    32 x 32 x 96     16^2x48 4 x (8x8, 4 bohr), 2.5 bohr apart, centred          CEF E = 0.005
3    24 x 24 x 80     12^2x40 4 x (8x4, 3 x 6 bohr), 2.5 bohr apart, centred      CPD dV = 0.5 V
4    16 x 16 x 2H     8x8xH  L x (4x4, 4 bohr), 2 bohr apart, 24 instances        12 CEF + 12 CPD
5    48 x 48 x 144    24^2x72 8 x (16x16, 3 bohr), 2.5 bohr apart, Z in {1,3,4,5} L-CPD 12x12 patch
==== ================ ====== =================================================== =====================
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

HARTREE_PER_VOLT = 1.0 / 27.211386245988  # 1 V expressed in Ha/e

JITTER = 0.2


@dataclass(frozen=True)
class Bias:
    """External bias setup of the paper's Section 2.2.

    kind: "cef" (constant electric field, sawtooth V_app, zero-Neumann Poisson) or
    "cpd" (constrained potential difference; with ``patch`` set it is L-CPD).
    field: the constant field E in Ha/bohr (CEF); dV: the potential difference in Ha
    (CPD); zA, zB: conductor interfaces (CPD); patch: ((xlo, ylo), (xhi, yhi)) in bohr.
    """

    kind: str = "cef"
    field: float = 0.0
    dV: float = 0.0
    zA: float = 0.0
    zB: float = 0.0
    patch: Optional[Tuple[Tuple[float, float], Tuple[float, float]]] = None


@dataclass(frozen=True)
class Slab:
    """One seeded synthetic slab: box, mesh, basis order, atoms and bias."""

    name: str
    L: Tuple[float, float, float]
    ncell: Tuple[int, int, int]
    p: int
    R: np.ndarray = field(repr=False)
    Z: np.ndarray = field(repr=False)
    bias: Bias = Bias()
    nvec: int = 0
    degree: int = 0
    psi_dirichlet: Tuple[bool, bool] = (True, True)
    seed: int = 0

    @property
    def n_phi(self) -> int:
        nx, ny, nz = self.ncell
        p = self.p
        return (nx * p) * (ny * p) * (nz * p + 1)

    @property
    def n_psi(self) -> int:
        nx, ny, nz = self.ncell
        p = self.p
        nzp = nz * p + 1 - int(self.psi_dirichlet[0]) - int(self.psi_dirichlet[1])
        return (nx * p) * (ny * p) * nzp

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.ncell))

    @property
    def n_electrons(self) -> float:
        return float(np.sum(self.Z))


def _layers(rng, L, nlat, spacing, z_layers, Zval, stagger=True):
    """Stack of jittered in-plane lattices; odd layers shifted by half a lattice cell."""
    R = []
    for li, z in enumerate(z_layers):
        off = 0.5 if (stagger and li % 2 == 1) else 0.0
        for j in range(nlat[1]):
            for i in range(nlat[0]):
                x = (i + 0.5 + off) * spacing[0]
                y = (j + 0.5 + off) * spacing[1]
                R.append((x, y, z))
    R = np.asarray(R, dtype=np.float64)
    R += rng.uniform(-JITTER, JITTER, size=R.shape)
    R[:, 0] %= L[0]
    R[:, 1] %= L[1]
    if np.isscalar(Zval):
        Z = np.full(len(R), float(Zval))
    else:
        Z = np.asarray(Zval, dtype=np.float64)
    return R, Z


def _centred_layers(Lz, n, gap):
    return [Lz / 2 + (k - (n - 1) / 2) * gap for k in range(n)]


def config1() -> Slab:
    """Plain FP64 constant-field slab (12x12x36 bohr, 6x6x16 cells, p=3, 16 atoms)."""
    rng = np.random.default_rng(1001)
    L = (12.0, 12.0, 36.0)
    R, Z = _layers(rng, L, (4, 2), (3.0, 6.0), [16.5, 19.5], 3.0)
    return Slab("cef-12x12x36-p3", L, (6, 6, 16), 3, R, Z,
                Bias("cef", field=0.01), nvec=32, degree=10, seed=1)


def config2() -> Slab:
    """Mixed-precision filter slab (32x32x96 bohr, 16x16x48 cells, p=5, 256 atoms)."""
    rng = np.random.default_rng(1002)
    L = (32.0, 32.0, 96.0)
    R, Z = _layers(rng, L, (8, 8), (4.0, 4.0), _centred_layers(L[2], 4, 2.5), 3.0)
    return Slab("cef-32x32x96-p5", L, (16, 16, 48), 5, R, Z,
                Bias("cef", field=0.005), nvec=512, degree=30, seed=2)


def config3() -> Slab:
    """Constrained-potential slab for differentiation (24x24x80 bohr, 12x12x40, p=4)."""
    rng = np.random.default_rng(1003)
    L = (24.0, 24.0, 80.0)
    R, Z = _layers(rng, L, (8, 4), (3.0, 6.0), _centred_layers(L[2], 4, 2.5), 3.0)
    return Slab("cpd-24x24x80-p4", L, (12, 12, 40), 4, R, Z,
                Bias("cpd", dV=0.5 * HARTREE_PER_VOLT, zA=2.0, zB=L[2] - 2.0), seed=3)


def config4(n_instances: int = 24):
    """Batched bias sweep: slabs of 8x8xH cells (H ~ U{8..40}), p=4, 128 vectors."""
    rng = np.random.default_rng(1004)
    H = rng.integers(8, 41, size=n_instances)
    fields = np.linspace(0.0, 0.02, n_instances // 2)
    dVs = np.linspace(0.0, 1.0, n_instances - n_instances // 2) * HARTREE_PER_VOLT
    out = []
    for k in range(n_instances):
        h = int(H[k])
        L = (16.0, 16.0, 2.0 * h)
        nl = int(np.clip((2 * h - 12) // 2 + 1, 3, 12))
        R, Z = _layers(rng, L, (4, 4), (4.0, 4.0), _centred_layers(L[2], nl, 2.0), 3.0)
        if k < n_instances // 2:
            b = Bias("cef", field=float(fields[k]))
        else:
            b = Bias("cpd", dV=float(dVs[k - n_instances // 2]), zA=2.0, zB=L[2] - 2.0)
        out.append(Slab(f"sweep{k:02d}-8x8x{h}-p4", L, (8, 8, h), 4, R, Z, b,
                        nvec=128, degree=20, seed=4))
    return out


def config5() -> Slab:
    """Large L-CPD slab (48x48x144 bohr, 24x24x72 cells, p=5, 2048 atoms)."""
    rng = np.random.default_rng(1005)
    L = (48.0, 48.0, 144.0)
    nat = 8 * 16 * 16
    Zval = rng.choice(np.array([1.0, 3.0, 4.0, 5.0]), size=nat)
    R, Z = _layers(rng, L, (16, 16), (3.0, 3.0), _centred_layers(L[2], 8, 2.5), Zval)
    c = (L[0] / 2, L[1] / 2)
    patch = ((c[0] - 6.0, c[1] - 6.0), (c[0] + 6.0, c[1] + 6.0))
    return Slab("lcpd-48x48x144-p5", L, (24, 24, 72), 5, R, Z,
                Bias("cpd", dV=0.5 * HARTREE_PER_VOLT, zA=2.0, zB=L[2] - 2.0, patch=patch),
                nvec=1024, degree=40, seed=5)


def small_slab(ncell=(2, 2, 4), p=3, L=(4.0, 4.0, 9.0), natoms=2, bias=None,
               psi_dirichlet=(True, True), seed=7, nvec=8, degree=6) -> Slab:
    """A tiny slab for tests that the oracle handles in well under a second."""
    rng = np.random.default_rng(seed)
    R = np.column_stack([rng.uniform(0, L[0], natoms), rng.uniform(0, L[1], natoms),
                         L[2] / 2 + rng.uniform(-1.0, 1.0, natoms)])
    Z = np.full(natoms, 1.0)
    return Slab(f"small-{ncell[0]}x{ncell[1]}x{ncell[2]}-p{p}", L, ncell, p, R, Z,
                bias or Bias("cef", field=0.01), nvec=nvec, degree=degree,
                psi_dirichlet=psi_dirichlet, seed=seed)


def start_block(slab: Slab, nvec: Optional[int] = None, seed: Optional[int] = None,
                n_rows: Optional[int] = None) -> np.ndarray:
    """Random start block X0 [n_psi][nvec], float32 N(0,1) draws from default_rng(2000+cfg)."""
    rng = np.random.default_rng(2000 + slab.seed if seed is None else seed)
    n = slab.n_psi if n_rows is None else n_rows
    return rng.standard_normal((n, nvec or slab.nvec), dtype=np.float32)


def lanczos_start(n: int, seed: int = 31) -> np.ndarray:
    """Start vector for the spectral-bound Lanczos run (float64 N(0,1))."""
    return np.random.default_rng(seed).standard_normal(n)


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}

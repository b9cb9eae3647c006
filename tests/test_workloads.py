"""Sizes of the seeded workloads (node counts follow from the mesh definition)."""
import numpy as np

import workloads as W


def test_config_sizes():
    c1 = W.config1()
    assert (c1.n_phi, c1.n_psi, c1.n_cells) == (15876, 15228, 576)
    assert len(c1.R) == 16 and c1.n_electrons == 48
    c2 = W.config2()
    assert (c2.n_phi, c2.n_psi) == (1542400, 1529600) and len(c2.R) == 256
    c3 = W.config3()
    assert (c3.n_phi, c3.n_psi) == (370944, 366336) and len(c3.R) == 128
    c5 = W.config5()
    assert c5.n_phi == 5198400 and len(c5.R) == 2048


def test_sweep_instances():
    sw = W.config4()
    assert len(sw) == 24
    assert all(8 <= s.ncell[2] <= 40 for s in sw)
    assert all(48 <= len(s.R) <= 192 for s in sw)
    assert sum(s.bias.kind == "cef" for s in sw) == 12


def test_seeded_and_in_box():
    a, b = W.config1(), W.config1()
    assert np.array_equal(a.R, b.R)
    for c in (W.config1(), W.config3()):
        assert np.all(c.R[:, 0] >= 0) and np.all(c.R[:, 0] < c.L[0])
        assert np.all(np.abs(c.R[:, 2] - c.L[2] / 2) < 0.25 * c.L[2])
    x0 = W.start_block(W.config1())
    assert x0.shape == (15228, 32) and x0.dtype == np.float32

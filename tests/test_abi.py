"""The C-ABI library builds, loads and exports every entry point of include/fe.h (no GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fe.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00998_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fe_mesh_create", "fe_apply_H", "fe_cheb_filter", "fe_poisson_solve",
              "fe_rayleigh_ritz", "fe_set_potential", "fe_lanczos_bounds"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_00998_gb300 import _lib
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(_lib.EXPORTS) == _declared()


def test_host_side_validation_without_gpu(lib):
    """Invalid descriptors are rejected on the host before any CUDA call."""
    from paper_2504_00998_gb300 import _lib
    d = _lib.FeMeshDesc()
    for k in range(3):
        d.L[k] = 1.0
        d.ncell[k] = 2
    h = C.c_void_p()
    for p in (0, 7):
        d.p = p
        assert lib.fe_mesh_create(C.byref(d), C.byref(h)) == _lib.FE_EINVAL
        assert b"p =" in lib.fe_last_error()
    d.p = 3
    d.L[1] = -1.0
    assert lib.fe_mesh_create(C.byref(d), C.byref(h)) == _lib.FE_EINVAL
    assert lib.fe_mesh_create(None, C.byref(h)) == _lib.FE_EINVAL
    assert lib.fe_apply_H(None, None, None, 1, 1, 0) == _lib.FE_EINVAL
    assert lib.fe_poisson_solve(None, None, None, None, None, None) == _lib.FE_EINVAL
    assert lib.fe_mesh_destroy(None) == _lib.FE_OK
    # the variants' entry points reject null meshes and arrays before any CUDA call
    assert lib.fe_set_potential_quad(None, None) == _lib.FE_EINVAL
    assert lib.fe_interp_quad(None, None, None) == _lib.FE_EINVAL
    assert lib.fe_set_kpoint(None, 0.1, 0.2) == _lib.FE_EINVAL
    assert lib.fe_rayleigh_ritz(None, None, 4, 4, None, 0) == _lib.FE_EINVAL
    assert lib.fe_lda_exchange(None, None, None, None) == _lib.FE_EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2504_00998_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved

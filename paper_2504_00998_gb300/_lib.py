"""ctypes binding of libfe's C ABI (include/fe.h).

Argument marshalling only: every function here forwards to the C function of the same name.
Loading fails loudly when the library has not been built; there is no fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfe.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_ENOCONV, FE_EBREAKDOWN, FE_ETIMEOUT, FE_EUNSUPPORTED = range(8)
FE_F64, FE_F32, FE_BF16_F32ACC, FE_F32_F32ACC = range(4)
FE_FACE_NEUMANN, FE_FACE_DIRICHLET = 0, 1
FE_BIAS_CEF, FE_BIAS_CPD = 0, 1
FE_OPT_RR_PRODUCTS, FE_OPT_POISSON_PRECOND, FE_OPT_POISSON_ARITH, FE_OPT_RR_EIGEN = 0, 1, 2, 3
FE_OPT_POISSON_ITER, FE_OPT_TEST_CG_STALL = 4, 5
FE_POISSON_ITER_PERSISTENT, FE_POISSON_ITER_LAUNCHES = 0, 1
FE_POISSON_F64, FE_POISSON_MIXED = 0, 1
FE_RR_PRODUCTS_F64, FE_RR_PRODUCTS_TC32 = 0, 1
FE_PRECOND_JACOBI, FE_PRECOND_JACOBI_PLANES, FE_PRECOND_JACOBI_PLANES_MODES = 0, 1, 2
FE_RR_EIGEN_SYEVD, FE_RR_EIGEN_SYEVJ = 0, 1

STATUS_NAMES = {0: "FE_OK", 1: "FE_EINVAL", 2: "FE_ENOMEM", 3: "FE_ECUDA", 4: "FE_ENOCONV",
                5: "FE_EBREAKDOWN", 6: "FE_ETIMEOUT", 7: "FE_EUNSUPPORTED"}

# every entry point declared in include/fe.h
EXPORTS = [
    "fe_mesh_create", "fe_mesh_destroy", "fe_mesh_info", "fe_mesh_set_stream", "fe_set_option",
    "fe_node_coords",
    "fe_lumped_mass", "fe_set_atoms", "fe_set_potential", "fe_apply_H", "fe_cheb_filter",
    "fe_cheb_filter_static",
    "fe_poisson_solve", "fe_poisson_solve_load", "fe_poisson_constraints",
    "fe_poisson_apply_K", "fe_poisson_apply_K_f32", "fe_poisson_rhs",
    "fe_rayleigh_ritz", "fe_atom_fields", "fe_energy", "fe_atom_fields_vjp",
    "fe_lanczos_bounds", "fe_kernel_launches", "fe_last_error",
    "fe_batch_create", "fe_batch_destroy", "fe_batch_apply_H", "fe_batch_cheb_filter",
    "fe_batch_rayleigh_ritz", "fe_density", "fe_occupations", "fe_mixer_create",
    "fe_mixer_destroy", "fe_mixer_step", "fe_lda_exchange", "fe_planar", "fe_dipole", "fe_vbare_phi",
    "fe_set_nonlocal", "fe_set_kpoint", "fe_set_potential_quad", "fe_interp_quad",
    "fe_potential_vjp", "fe_batch_tuning", "fe_batch_set_launch",
]


class FeMeshDesc(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("ncell", C.c_int * 3), ("p", C.c_int),
                ("psi_z", C.c_int * 2), ("device", C.c_int), ("stream", C.c_void_p)]


class FePoissonBC(C.Structure):
    _fields_ = [("kind", C.c_int), ("field", C.c_double), ("dV", C.c_double), ("zA", C.c_double),
                ("zB", C.c_double), ("has_patch", C.c_int), ("patch_lo", C.c_double * 2),
                ("patch_hi", C.c_double * 2), ("rtol", C.c_double), ("max_iter", C.c_int)]


class FeSolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_residual", C.c_double), ("status", C.c_int)]


class FeError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path=LIB_PATH):
    """Load libfe.so (raises if it is missing: build it with paper_2504_00998_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libfe is not built ({path} missing); run "
                          "python -m paper_2504_00998_gb300.build")
    lib = C.CDLL(path)
    P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
    sig = {
        "fe_mesh_create": ([C.POINTER(FeMeshDesc), C.POINTER(C.c_void_p)], I),
        "fe_mesh_destroy": ([P], I),
        "fe_mesh_info": ([P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)], I),
        "fe_mesh_set_stream": ([P, P], I),
        "fe_set_option": ([P, I, I64], I),
        "fe_node_coords": ([P, P], I),
        "fe_lumped_mass": ([P, P], I),
        "fe_set_atoms": ([P, I, P, P, D, D, D], I),
        "fe_set_potential": ([P, P], I),
        "fe_apply_H": ([P, P, P, I64, I64, I], I),
        "fe_potential_vjp": ([P, P, P, I64, I64, P, I], I),
        "fe_cheb_filter": ([P, P, I64, I64, I, D, D, D, I], I),
        "fe_cheb_filter_static": ([P, P, I64, I64, I, D, D, D, I], I),
        "fe_poisson_solve": ([P, P, C.POINTER(FePoissonBC), P, P, C.POINTER(FeSolveInfo)], I),
        "fe_poisson_solve_load": ([P, P, C.POINTER(FePoissonBC), P, P, C.POINTER(FeSolveInfo)], I),
        "fe_poisson_constraints": ([P, C.POINTER(FePoissonBC), P, P], I),
        "fe_poisson_apply_K": ([P, P, P], I),
        "fe_poisson_apply_K_f32": ([P, P, P], I),
        "fe_lda_exchange": ([P, P, P, C.POINTER(D)], I),
        "fe_set_kpoint": ([P, D, D], I),
        "fe_set_potential_quad": ([P, P], I),
        "fe_interp_quad": ([P, P, P], I),
        "fe_poisson_rhs": ([P, P, P, P, P], I),
        "fe_rayleigh_ritz": ([P, P, I64, I64, P, I], I),
        "fe_lanczos_bounds": ([P, P, I, C.POINTER(D), C.POINTER(D)], I),
        "fe_atom_fields": ([P, P, P, P], I),
        "fe_energy": ([P, C.POINTER(FePoissonBC), P, C.POINTER(D), C.POINTER(D), C.POINTER(D),
                       P, P, P], I),
        "fe_atom_fields_vjp": ([P, P, P, P, P], I),
        "fe_batch_create": ([P, I, C.POINTER(C.c_void_p)], I),
        "fe_batch_destroy": ([P], I),
        "fe_batch_apply_H": ([P, P, P, P, P, I], I),
        "fe_batch_cheb_filter": ([P, P, P, P, I, P, P, P, I], I),
        "fe_batch_rayleigh_ritz": ([P, P, I64, P, P, I], I),
        "fe_batch_tuning": ([P, C.POINTER(I), C.POINTER(I), C.POINTER(D), C.POINTER(I)], I),
        "fe_batch_set_launch": ([P, I, I], I),
        "fe_density": ([P, P, I64, I64, P, P, I], I),
        "fe_occupations": ([P, I, D, D, P, C.POINTER(D)], I),
        "fe_mixer_create": ([P, I, D, C.POINTER(C.c_void_p)], I),
        "fe_mixer_destroy": ([P], I),
        "fe_mixer_step": ([P, P, P, C.POINTER(D)], I),
        "fe_planar": ([P, P, I, P], I),
        "fe_dipole": ([P, P, C.POINTER(D)], I),
        "fe_vbare_phi": ([P, P, C.POINTER(FePoissonBC), P], I),
        "fe_set_nonlocal": ([P, I, P, P, P, D], I),
        "fe_kernel_launches": ([], I64),
        "fe_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def check(status, func):
    if status != FE_OK:
        msg = load().fe_last_error().decode(errors="replace")
        raise FeError(status, func, msg)
    return status


def call(name, *args):
    """Call ``name`` and raise FeError on a non-FE_OK status."""
    return check(getattr(load(), name)(*args), name)

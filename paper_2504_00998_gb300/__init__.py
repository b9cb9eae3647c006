"""GB300 finite-element Kohn-Sham slab hot path: a thin torch-facing binding of libfe.

PyTorch provides device memory and streams only; every step runs in libfe's CUDA kernels
through the C ABI declared in include/fe.h (see ``_lib.py`` for the raw binding).  If
libfe has not been built, importing the binding raises instead of falling back.
"""
import ctypes as C

import torch

from . import _lib
from ._lib import (FE_BF16_F32ACC, FE_BIAS_CEF, FE_BIAS_CPD, FE_F32, FE_F32_F32ACC, FE_F64,
                   FE_FACE_DIRICHLET, FE_FACE_NEUMANN, FeError, FePoissonBC, FeSolveInfo, call)

__all__ = ["Mesh", "Batch", "FeError", "FE_F64", "FE_F32", "FE_BF16_F32ACC", "FE_F32_F32ACC",
           "FE_BIAS_CEF", "FE_BIAS_CPD", "storage_dtype", "load"]

load = _lib.load


def storage_dtype(prec, complex_=False):
    if complex_:
        return torch.complex128 if prec == FE_F64 else torch.complex64
    return torch.float64 if prec == FE_F64 else torch.float32


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Mesh:
    """Owns one fe_mesh handle (Section 2.3 slab mesh, periodic x/y, bounded z)."""

    def __init__(self, L, ncell, p, psi_dirichlet=(True, True), device=0, stream=None):
        load()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        d = _lib.FeMeshDesc()
        for k in range(3):
            d.L[k] = float(L[k])
            d.ncell[k] = int(ncell[k])
        d.p = int(p)
        d.psi_z[0] = FE_FACE_DIRICHLET if psi_dirichlet[0] else FE_FACE_NEUMANN
        d.psi_z[1] = FE_FACE_DIRICHLET if psi_dirichlet[1] else FE_FACE_NEUMANN
        d.device = device
        d.stream = C.c_void_p(stream.cuda_stream)
        h = C.c_void_p()
        call("fe_mesh_create", C.byref(d), C.byref(h))
        self._h = h
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        call("fe_mesh_info", h, C.byref(a), C.byref(b), C.byref(c))
        self.n_phi, self.n_psi, self.n_cells = a.value, b.value, c.value
        self.L, self.ncell, self.p = tuple(L), tuple(ncell), p

    @classmethod
    def from_slab(cls, slab, device=0, stream=None, with_atoms=True):
        m = cls(slab.L, slab.ncell, slab.p, slab.psi_dirichlet, device, stream)
        if with_atoms:
            m.set_atoms(slab.R, slab.Z)
        return m

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().fe_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f64(self, n):
        return torch.empty(n, dtype=torch.float64, device=self.device)

    def set_rr_products(self, tensor_core):
        """Rayleigh-Ritz block products for float storage: double GEMMs (False) or
        FP32-accurate tensor-core emulation (True)."""
        call("fe_set_option", self._h, _lib.FE_OPT_RR_PRODUCTS,
             _lib.FE_RR_PRODUCTS_TC32 if tensor_core else _lib.FE_RR_PRODUCTS_F64)

    def set_rr_eigensolver(self, jacobi):
        """Dense eigensolver of the projected matrix in Rayleigh-Ritz: divide-and-conquer
        (False, the default) or cyclic Jacobi (True); double precision either way."""
        call("fe_set_option", self._h, _lib.FE_OPT_RR_EIGEN,
             _lib.FE_RR_EIGEN_SYEVJ if jacobi else _lib.FE_RR_EIGEN_SYEVD)

    def set_poisson_precond(self, planes, modes=False):
        """Poisson CG preconditioner: Jacobi (planes False), Jacobi plus the z-plane coarse
        solve (planes True), and with modes True also the in-plane Fourier modes of
        wavenumber one on every plane (persistent float iteration, meshes without
        constrained phi nodes)."""
        v = (_lib.FE_PRECOND_JACOBI_PLANES_MODES if modes else _lib.FE_PRECOND_JACOBI_PLANES) \
            if planes else _lib.FE_PRECOND_JACOBI
        call("fe_set_option", self._h, _lib.FE_OPT_POISSON_PRECOND, v)

    def planar(self, f, average=False):
        """Per phi plane: the planar integral (rho0) or average (V0) of a phi-node field."""
        out = self._f64(self.ncell[2] * self.p + 1)
        call("fe_planar", self._h, _ptr(f.contiguous()), 1 if average else 0, _ptr(out))
        return out

    def dipole(self, rho=None):
        """mu_z = int (b + rho)(z - Lz/2) (rho None: the atoms' model density)."""
        mu = C.c_double()
        call("fe_dipole", self._h, _ptr(rho.contiguous() if rho is not None else None),
             C.byref(mu))
        return mu.value

    def vbare_phi(self, phi, bias):
        """V_bare = phi + V_loc - V_sm + V_app on every phi node."""
        out = self._f64(self.n_phi)
        bc = self.make_bc(bias)
        call("fe_vbare_phi", self._h, _ptr(phi.contiguous()), C.byref(bc), _ptr(out))
        return out

    def set_poisson_mixed(self, mixed):
        """Poisson arithmetic: double CG (False) or float corrections refined against the
        double residual (True, the default); both stop at the same double residual."""
        call("fe_set_option", self._h, _lib.FE_OPT_POISSON_ARITH,
             _lib.FE_POISSON_MIXED if mixed else _lib.FE_POISSON_F64)

    def set_poisson_persistent(self, persistent):
        """Float CG iterations in one cooperative kernel between reliable updates (True, the
        default) or one launch per step from CUDA graphs (False)."""
        call("fe_set_option", self._h, _lib.FE_OPT_POISSON_ITER,
             _lib.FE_POISSON_ITER_PERSISTENT if persistent else _lib.FE_POISSON_ITER_LAUNCHES)

    def node_coords(self):
        out = self._f64((self.n_phi, 3))
        call("fe_node_coords", self._h, _ptr(out))
        return out

    def lumped_mass(self):
        out = self._f64(self.n_phi)
        call("fe_lumped_mass", self._h, _ptr(out))
        return out

    def set_atoms(self, R, Z, sigma_b=0.5, rc_loc=1.0, sigma_rho=1.0):
        R = torch.as_tensor(R, dtype=torch.float64).contiguous().cpu()
        Z = torch.as_tensor(Z, dtype=torch.float64).contiguous().cpu()
        call("fe_set_atoms", self._h, int(Z.numel()), _ptr(R), _ptr(Z), float(sigma_b),
             float(rc_loc), float(sigma_rho))

    def set_nonlocal(self, R, sigma, D, rc):
        """Nonlocal term with synthetic s + p projectors (R [n][3], sigma [n], D [n][4])."""
        R = torch.as_tensor(R, dtype=torch.float64).contiguous().cpu()
        sg = torch.as_tensor(sigma, dtype=torch.float64).contiguous().cpu()
        Dt = torch.as_tensor(D, dtype=torch.float64).contiguous().cpu()
        call("fe_set_nonlocal", self._h, int(sg.numel()), _ptr(R), _ptr(sg), _ptr(Dt), float(rc))

    def set_kpoint(self, kx, ky):
        """Bloch wave vector (fe_set_kpoint); blocks are then complex tensors."""
        call("fe_set_kpoint", self._h, float(kx), float(ky))
        self.kpoint = (float(kx), float(ky))

    def _block_dtype(self, prec):
        k = getattr(self, "kpoint", (0.0, 0.0))
        return storage_dtype(prec, complex_=(k != (0.0, 0.0)))

    def set_potential(self, veff):
        assert veff.dtype == torch.float64 and veff.is_cuda and veff.numel() == self.n_psi
        call("fe_set_potential", self._h, _ptr(veff.contiguous()))

    def set_potential_quad(self, vq):
        """V_eff at every cell's Gauss points, [n_cells, (p+1)^3] float64 on the device
        (fe_set_potential_quad): the potential term integrated by Gauss quadrature."""
        assert vq.dtype == torch.float64 and vq.is_cuda
        assert vq.numel() == self.n_cells * (self.p + 1) ** 3
        call("fe_set_potential_quad", self._h, _ptr(vq.contiguous()))

    def interp_quad(self, f_phi):
        """Values at every cell's Gauss points of the phi-node field f_phi (fe_interp_quad)."""
        assert f_phi.dtype == torch.float64 and f_phi.is_cuda and f_phi.numel() == self.n_phi
        out = torch.empty((self.n_cells, (self.p + 1) ** 3), dtype=torch.float64,
                          device=f_phi.device)
        call("fe_interp_quad", self._h, _ptr(f_phi.contiguous()), _ptr(out))
        return out

    def apply_H(self, X, Y=None, prec=FE_F64):
        n, nvec = X.shape[0], X.shape[1]
        assert n == self.n_psi and X.dtype == self._block_dtype(prec) and X.is_cuda
        if Y is None:
            Y = torch.empty_like(X)
        call("fe_apply_H", self._h, _ptr(X), _ptr(Y), nvec, X.stride(0), int(prec))
        return Y

    def potential_vjp(self, X, Ybar, prec=FE_F64):
        """dL/dV_eff = sum_v Ybar_Iv X_Iv for Y = Ht X (fe_potential_vjp)."""
        assert X.dtype == Ybar.dtype == self._block_dtype(prec)
        assert X.shape == Ybar.shape and X.stride(0) == Ybar.stride(0) and X.shape[0] == self.n_psi
        g = self._f64(self.n_psi)
        call("fe_potential_vjp", self._h, _ptr(X), _ptr(Ybar), X.shape[1], X.stride(0), _ptr(g),
             int(prec))
        return g

    def cheb_filter(self, X, degree, a, b, a0, prec=FE_F64):
        assert X.dtype == self._block_dtype(prec) and X.shape[0] == self.n_psi
        call("fe_cheb_filter", self._h, _ptr(X), X.shape[1], X.stride(0), int(degree), float(a),
             float(b), float(a0), int(prec))
        return X

    def rayleigh_ritz(self, X, prec=FE_F64):
        eig = self._f64(X.shape[1])
        call("fe_rayleigh_ritz", self._h, _ptr(X), X.shape[1], X.stride(0), _ptr(eig), int(prec))
        return eig

    def lanczos_bounds(self, v0, steps=20):
        lo, hi = C.c_double(), C.c_double()
        call("fe_lanczos_bounds", self._h, _ptr(v0), int(steps), C.byref(lo), C.byref(hi))
        return lo.value, hi.value

    def poisson_apply_K(self, x, y=None):
        """y = K x; float64 through fe_poisson_apply_K, float32 through fe_poisson_apply_K_f32."""
        y = torch.empty_like(x) if y is None else y
        name = "fe_poisson_apply_K_f32" if x.dtype == torch.float32 else "fe_poisson_apply_K"
        call(name, self._h, _ptr(x), _ptr(y))
        return y

    def poisson_rhs(self, rho=None):
        f, r, b = self._f64(self.n_phi), self._f64(self.n_phi), self._f64(self.n_phi)
        call("fe_poisson_rhs", self._h, _ptr(rho), _ptr(f), _ptr(r), _ptr(b))
        return f, r, b

    @staticmethod
    def make_bc(bias, rtol=1e-10, max_iter=20000):
        bc = FePoissonBC()
        bc.kind = FE_BIAS_CEF if bias.kind == "cef" else FE_BIAS_CPD
        bc.field = float(bias.field)
        bc.dV = float(bias.dV)
        bc.zA = float(bias.zA)
        bc.zB = float(bias.zB)
        if bias.patch is not None:
            bc.has_patch = 1
            (bc.patch_lo[0], bc.patch_lo[1]), (bc.patch_hi[0], bc.patch_hi[1]) = bias.patch
        bc.rtol = float(rtol)
        bc.max_iter = int(max_iter)
        return bc

    def poisson_solve_load(self, f, bias, phic=None, rtol=1e-10, max_iter=20000, phi=None):
        phi = self._f64(self.n_phi) if phi is None else phi
        info = FeSolveInfo()
        bc = self.make_bc(bias, rtol, max_iter)
        call("fe_poisson_solve_load", self._h, _ptr(f.contiguous()), C.byref(bc),
             _ptr(phic.contiguous() if phic is not None else None), _ptr(phi), C.byref(info))
        return phi, info

    def poisson_constraints(self, bias):
        mask = torch.empty(self.n_phi, dtype=torch.uint8, device=self.device)
        vals = self._f64(self.n_phi)
        bc = self.make_bc(bias)
        call("fe_poisson_constraints", self._h, C.byref(bc), _ptr(mask), _ptr(vals))
        return mask.bool(), vals

    def atom_fields(self):
        r, b, v = self._f64(self.n_phi), self._f64(self.n_phi), self._f64(self.n_phi)
        call("fe_atom_fields", self._h, _ptr(r), _ptr(b), _ptr(v))
        return r, b, v

    def energy(self, bias, phi):
        """(E, dE/dfield, dE/ddV, dE/drho, dE/db, dE/dvlms) at the solved phi."""
        E, df, dv = C.c_double(), C.c_double(), C.c_double()
        gr, gb, gv = self._f64(self.n_phi), self._f64(self.n_phi), self._f64(self.n_phi)
        bc = self.make_bc(bias)
        call("fe_energy", self._h, C.byref(bc), _ptr(phi), C.byref(E), C.byref(df), C.byref(dv),
             _ptr(gr), _ptr(gb), _ptr(gv))
        return E.value, df.value, dv.value, gr, gb, gv

    def atom_fields_vjp(self, g_rho, g_b, g_vlms, natoms):
        out = torch.empty((natoms, 3), dtype=torch.float64)
        call("fe_atom_fields_vjp", self._h, _ptr(g_rho), _ptr(g_b), _ptr(g_vlms), _ptr(out))
        return out

    def poisson_solve(self, bias, rho=None, rtol=1e-10, max_iter=20000, phi=None, vbare=True):
        phi = self._f64(self.n_phi) if phi is None else phi
        vb = self._f64(self.n_psi) if vbare is True else (vbare if vbare is not False else None)
        info = FeSolveInfo()
        bc = self.make_bc(bias, rtol, max_iter)
        call("fe_poisson_solve", self._h, _ptr(rho), C.byref(bc), _ptr(phi), _ptr(vb),
             C.byref(info))
        return phi, vb, info


class Batch:
    """Independent slabs with a common p and cell size, stepped together (fe_batch_*): each
    operator application is one kernel launch over every instance."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (C.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        h = C.c_void_p()
        call("fe_batch_create", arr, len(self.meshes), C.byref(h))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().fe_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _blocks(self, Xs, prec):
        assert len(Xs) == len(self.meshes)
        for X, m in zip(Xs, self.meshes):
            assert X.dtype == storage_dtype(prec) and X.is_cuda and X.shape[0] == m.n_psi
        n = len(Xs)
        ptrs = (C.c_void_p * n)(*[X.data_ptr() for X in Xs])
        nvec = (C.c_int64 * n)(*[X.shape[1] for X in Xs])
        ld = (C.c_int64 * n)(*[X.stride(0) for X in Xs])
        return ptrs, nvec, ld

    def apply_H(self, Xs, Ys=None, prec=FE_F64):
        Ys = [torch.empty_like(X) for X in Xs] if Ys is None else Ys
        xp, nvec, ld = self._blocks(Xs, prec)
        yp, _, _ = self._blocks(Ys, prec)
        call("fe_batch_apply_H", self._h, xp, yp, nvec, ld, int(prec))
        return Ys

    def tuning(self):
        """(zseg, persistent, best_ms, candidates timed) of the batched launches
        (fe_batch_tuning)."""
        z, pers, ms, nc = C.c_int(), C.c_int(), C.c_double(), C.c_int()
        call("fe_batch_tuning", self._h, C.byref(z), C.byref(pers), C.byref(ms), C.byref(nc))
        return z.value, pers.value, ms.value, nc.value

    def set_launch(self, zseg, persistent):
        call("fe_batch_set_launch", self._h, int(zseg), int(persistent))

    def cheb_filter(self, Xs, degree, a, b, a0, prec=FE_F64):
        xp, nvec, ld = self._blocks(Xs, prec)
        n = len(Xs)
        dd = [(C.c_double * n)(*[float(v) for v in arr]) for arr in (a, b, a0)]
        call("fe_batch_cheb_filter", self._h, xp, nvec, ld, int(degree), dd[0], dd[1], dd[2],
             int(prec))
        return Xs

    def rayleigh_ritz(self, Xs, prec=FE_F64):
        """Cholesky-QR + Rayleigh-Ritz of every block (equal widths); returns the Ritz values
        per instance."""
        xp, nvec, ld = self._blocks(Xs, prec)
        n = Xs[0].shape[1]
        assert all(X.shape[1] == n for X in Xs)
        eigs = [torch.empty(n, dtype=torch.float64, device=X.device) for X in Xs]
        ep = (C.c_void_p * len(eigs))(*[e.data_ptr() for e in eigs])
        call("fe_batch_rayleigh_ritz", self._h, xp, int(n), ld, ep, int(prec))
        return eigs

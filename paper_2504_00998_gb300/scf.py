"""Self-consistent iterations of the slab driven through libfe (Hartree level, optionally
with local-density exchange, fe_lda_exchange): Poisson with the bias (fe_poisson_solve with
the current density), V_eff,
Lanczos bounds, Chebyshev-filtered subspace iteration, Fermi-Dirac occupations
(fe_occupations), the density of the block (fe_density) and Anderson mixing
(fe_mixer_step).  Every step runs in the library; this module only sequences the calls.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import call


class Mixer:
    """Owns an fe_mixer (Anderson / Pulay density mixing on phi nodes)."""

    def __init__(self, mesh, history=4, alpha=0.3):
        h = C.c_void_p()
        call("fe_mixer_create", mesh.handle, int(history), float(alpha), C.byref(h))
        self._h = h

    def step(self, rho_in, rho_out):
        r = C.c_double()
        call("fe_mixer_step", self._h, C.c_void_p(rho_in.data_ptr()),
             C.c_void_p(rho_out.data_ptr()), C.byref(r))
        return r.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.load().fe_mixer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def occupations(eig, n_electrons, kT):
    """(occ = 2 f, mu) of Ritz values (host) by fe_occupations."""
    e = np.ascontiguousarray(np.asarray(eig, dtype=np.float64))
    occ = np.empty_like(e)
    mu = C.c_double()
    call("fe_occupations", C.c_void_p(e.ctypes.data), len(e), float(n_electrons), float(kT),
         C.c_void_p(occ.ctypes.data), C.byref(mu))
    return occ, mu.value


def lda_exchange(mesh, rho, veff=None):
    """E_x of the phi-node density rho (fe_lda_exchange); adds v_x to veff (psi nodes, in
    place) when given."""
    ex = C.c_double()
    call("fe_lda_exchange", mesh.handle, C.c_void_p(rho.data_ptr()),
         C.c_void_p(veff.data_ptr()) if veff is not None else None, C.byref(ex))
    return ex.value


def density(mesh, X, occ, prec):
    """rho on phi nodes from the block X and occupations occ (device or host)."""
    o = torch.as_tensor(occ, dtype=torch.float64).to(X.device).contiguous()
    rho = torch.empty(mesh.n_phi, dtype=torch.float64, device=X.device)
    call("fe_density", mesh.handle, C.c_void_p(X.data_ptr()), X.shape[1], X.stride(0),
         C.c_void_p(o.data_ptr()), C.c_void_p(rho.data_ptr()), int(prec))
    return rho


def scf_run(mesh, bias, n_electrons, X, iters, kT=0.01, alpha=0.3, history=4, degree=10,
            first_cycles=4, lanczos_steps=20, v0=None, prec=0, rtol=1e-12, max_iter=50000,
            xc=None):
    """Self-consistent iterations from the atoms' model density (the same sequence as the
    CPU oracle's scf_run): per iteration the Poisson solve with the load 4 pi M (rho_in + b)
    and the bias, V_eff, Lanczos bounds (lo, hi) from v0, filter + Rayleigh-Ritz cycles
    (first_cycles on the first iteration, then one) with a0 = lo, b = hi and the cut
    a = lo + 0.1 (hi - lo) for the very first cycle, else the previous largest Ritz value
    when it lies in (lo, hi) (else the first-cycle rule again);
    occupations, rho_out, Anderson mixing.  xc = "lda_x" adds the local-density exchange
    potential of rho_in to V_eff.  X (the block, updated in place) holds the start vectors.
    Returns dict(rho, mu, eig, res) (and ex, E_x of the final rho_in, with xc)."""
    if xc not in (None, "lda_x"):
        raise ValueError("xc must be None or 'lda_x'")
    dev = X.device
    rho_in, _, _ = mesh.atom_fields()
    rho_in = rho_in.clone()
    mixer = Mixer(mesh, history, alpha)
    v0 = torch.ones(mesh.n_psi, dtype=torch.float64, device=dev) if v0 is None else v0
    cut, eig, mu, res = None, None, None, []
    try:
        for k in range(iters):
            _, vbare, _ = mesh.poisson_solve(bias, rho=rho_in, rtol=rtol, max_iter=max_iter)
            if xc == "lda_x":
                lda_exchange(mesh, rho_in, vbare)
            mesh.set_potential(vbare)
            lo, hi = mesh.lanczos_bounds(v0, lanczos_steps)
            for _ in range(first_cycles if k == 0 else 1):
                # the previous largest Ritz value when it lies inside the new interval, else
                # the first-cycle rule (the potential can move the spectrum between iterations)
                a = cut if cut is not None and lo < cut < hi else lo + 0.1 * (hi - lo)
                mesh.cheb_filter(X, degree, a, hi, lo, prec=prec)
                eig = mesh.rayleigh_ritz(X, prec=prec).cpu().numpy()
                cut = float(eig[-1])
            occ, mu = occupations(eig, n_electrons, kT)
            rho_out = density(mesh, X, occ, prec)
            res.append(mixer.step(rho_in, rho_out))
    finally:
        mixer.close()
    out = {"rho": rho_in, "mu": mu, "eig": eig, "res": res}
    if xc == "lda_x":
        out["ex"] = lda_exchange(mesh, rho_in)
    return out

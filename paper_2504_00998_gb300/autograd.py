"""torch.autograd wrappers of the biased-slab electrostatics (differentiation form).

* ``PoissonSolve``: phi = solve(f, phi_c) for the CEF or CPD / L-CPD setup
  (Eq. governing_equations CEF / APD).  Backward is the adjoint solve: K is symmetric, so
  dL/df = solve(dL/dphi, phi_c = 0) on the free nodes and
  dL/dphi_c = (dL/dphi)_c - (K lambda)_c on the constrained nodes.
* ``HamiltonianApply``: Y = Ht(V_eff) X (Eq. Veff and Hloc).  Ht is symmetric (Hermitian
  for a Bloch wave vector), so dL/dX = Ht Ybar (one more fe_apply_H); V_eff enters only
  through diag(V_eff), so dL/dV_eff = sum_v Ybar_Iv X_Iv (fe_potential_vjp; for complex
  blocks the real part of Ybar conj(X), the sum over the (re, im) lanes).
* ``SlabEnergy``: E(R, field, dV) of the slab (Eq. electrostatics Energy with the local
  pseudopotential and V_app terms).  The potential maximises E over the free nodes, so the
  gradient needs no adjoint solve (envelope theorem); the position gradient is the
  vector-Jacobian product of the atom fields computed by libfe.

All arithmetic runs in libfe's kernels; this module only orders the calls.
"""
import dataclasses

import torch

from . import FE_BIAS_CEF, FE_F64, Mesh


class PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, phic, mesh, bias, rtol):
        phi, info = mesh.poisson_solve_load(f.detach(), bias, phic=None if phic is None else phic.detach(),
                                            rtol=rtol)
        ctx.mesh, ctx.bias, ctx.rtol = mesh, bias, rtol
        ctx.has_phic = phic is not None
        return phi

    @staticmethod
    def backward(ctx, g):
        mesh, bias = ctx.mesh, ctx.bias
        g = g.contiguous()
        if bias.kind == "cef":
            lam, _ = mesh.poisson_solve_load(g, bias, rtol=ctx.rtol)
            return lam, None, None, None, None
        zero = torch.zeros_like(g)
        lam, _ = mesh.poisson_solve_load(g, bias, phic=zero, rtol=ctx.rtol)
        mask, _ = mesh.poisson_constraints(bias)
        grad_f = torch.where(mask, zero, lam)
        grad_phic = None
        if ctx.has_phic:
            klam = mesh.poisson_apply_K(grad_f)
            grad_phic = torch.where(mask, g - klam, zero)
        return grad_f, grad_phic, None, None, None


class HamiltonianApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, V, mesh, prec):
        X = X.detach().contiguous()
        V = V.detach().contiguous()
        mesh.set_potential(V)
        Y = mesh.apply_H(X, prec=prec)
        ctx.save_for_backward(X, V)
        ctx.mesh, ctx.prec = mesh, prec
        return Y

    @staticmethod
    def backward(ctx, gY):
        X, V = ctx.saved_tensors
        mesh, prec = ctx.mesh, ctx.prec
        gY = gY.contiguous().to(X.dtype)
        gX = gV = None
        mesh.set_potential(V)   # the operator of the forward pass
        if ctx.needs_input_grad[0]:
            gX = mesh.apply_H(gY, prec=prec)
        if ctx.needs_input_grad[1]:
            gV = mesh.potential_vjp(X, gY, prec=prec)
        return gX, gV, None, None


def apply_H(mesh, X, V, prec=FE_F64):
    """Y = Ht(V) X, differentiable in X and in the collocated potential V (float64 [n_psi])."""
    return HamiltonianApply.apply(X, V, mesh, prec)


class SlabEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, field, dV, mesh, Z, bias, rtol):
        Rn = R.detach().cpu().double()
        mesh.set_atoms(Rn, Z)
        b = dataclasses.replace(bias, field=float(field), dV=float(dV))
        phi, _, info = mesh.poisson_solve(b, rtol=rtol, vbare=False)
        E, dEf, dEdV, gr, gb, gv = mesh.energy(b, phi)
        dR = mesh.atom_fields_vjp(gr, gb, gv, Rn.shape[0])
        ctx.save_for_backward(dR.to(R.device), torch.tensor(dEf), torch.tensor(dEdV))
        ctx.cef = b.kind == "cef"
        return torch.tensor(E, dtype=torch.float64, device=R.device)

    @staticmethod
    def backward(ctx, gE):
        dR, dEf, dEdV = ctx.saved_tensors
        gE = gE.to(torch.float64)
        return (gE * dR, (gE.cpu() * dEf).to(torch.float64), (gE.cpu() * dEdV).to(torch.float64),
                None, None, None, None)


def slab_energy(mesh, R, Z, bias, field=None, dV=None, rtol=1e-12):
    """E(R, field, dV) as a differentiable torch scalar (float64)."""
    field = torch.tensor(bias.field, dtype=torch.float64) if field is None else field
    dV = torch.tensor(bias.dV, dtype=torch.float64) if dV is None else dV
    return SlabEnergy.apply(R, field, dV, mesh, Z, bias, rtol)


def poisson_solve(mesh, f, bias, phic=None, rtol=1e-12):
    return PoissonSolve.apply(f, phic, mesh, bias, rtol)

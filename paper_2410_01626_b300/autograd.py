"""torch.autograd.Function around the FMM energy with a hand-written adjoint.

E(x, qA, qB, lambda) is the Coulomb energy of the interpolated charges
q_i = qA_i + lambda_{s(i)} (qB_i - qA_i) (Sec. 2.1, Eq. 1).  Its gradient
needs no second pass through the tree: dE/dx_i = -F_i and, because E is
quadratic in the charges, dE/dq_i = k_e phi_i, which the chain rule turns into
dE/dqA_i = k_e phi_i (1 - lambda_s), dE/dqB_i = k_e phi_i lambda_s and
dE/dlambda_k = dV/dlambda_k (the lambda-particle force of Sec. 2.1).  The
forward saves F, phi and dV/dlambda; backward is one elementwise kernel
(fmm_adjoint) scaled by the incoming gradient.
"""
from __future__ import annotations

import torch


class FMMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, qA, qB, site, lam, solver):
        key = (qA.data_ptr(), qB.data_ptr(), site.data_ptr(), qA._version, qB._version, site._version, qA.numel())
        if getattr(solver, "_charge_key", None) != key:
            solver.set_charges(qA.detach().contiguous(), qB.detach().contiguous(), site.contiguous(),
                               lam.detach().contiguous())
            solver._charge_key = key
        elif lam.numel():
            solver.set_lambda(lam.detach().contiguous())
        E, F, dV, phi = solver.eval(x.detach().contiguous(), phi=True)
        ctx.solver = solver
        ctx.save_for_backward(F, phi, dV)
        ctx.needs = ctx.needs_input_grad
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        F, phi, dV = ctx.saved_tensors
        solver = ctx.solver
        g = gE.detach().reshape(1).to(torch.float64).contiguous()
        nx, na, nb, _, nl, _ = ctx.needs
        gx, ga, gb, gl = solver.adjoint(g, F, phi, dV, grad_x=nx, grad_qA=na, grad_qB=nb, grad_lam=nl)
        return gx, ga, gb, None, gl, None


def fmm_energy(x, qA, qB, site, lam, solver):
    """E as a differentiable function of positions, both charge forms and lambda."""
    return FMMEnergy.apply(x, qA, qB, site, lam, solver)


class FMMEnergy4(torch.autograd.Function):
    """The same for sites with two lambda coordinates over four charge forms (Sec. 2.1, Eq. 2):
    dE/dq^X_i = k_e phi_i w_X with the bilinear weights w_X of the atom's site."""

    @staticmethod
    def forward(ctx, x, qA, qB, qC, qD, site, lam, solver):
        key = tuple(t.data_ptr() for t in (qA, qB, qC, qD, site)) + tuple(t._version for t in (qA, qB, qC, qD, site))
        if getattr(solver, "_charge_key", None) != key:
            solver.set_charges4(*(t.detach().contiguous() for t in (qA, qB, qC, qD)), site.contiguous(),
                                lam.detach().contiguous())
            solver._charge_key = key
        elif lam.numel():
            solver.set_lambda(lam.detach().contiguous())
        E, F, dV, phi = solver.eval(x.detach().contiguous(), phi=True)
        ctx.solver = solver
        ctx.save_for_backward(F, phi, dV)
        ctx.needs = ctx.needs_input_grad
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        F, phi, dV = ctx.saved_tensors
        g = gE.detach().reshape(1).to(torch.float64).contiguous()
        nx, na, nb, nc, nd, _, nl, _ = ctx.needs
        gx, gq, gl = ctx.solver.adjoint4(g, F, phi, dV, grad_x=nx, grad_q=(na, nb, nc, nd), grad_lam=nl)
        return (gx, *gq, None, gl, None)


def fmm_energy4(x, qA, qB, qC, qD, site, lam, solver):
    """E of four-form sites as a differentiable function of positions, the four forms and lambda."""
    return FMMEnergy4.apply(x, qA, qB, qC, qD, site, lam, solver)

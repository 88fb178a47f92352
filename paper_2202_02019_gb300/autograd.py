"""Differentiable ladder energy E(L, tau, tbar) = sum_ijab tbar_ij^ab Omega_ij^ab.

Omega_ij^ab = sum_cd g_acbd tau_ij^cd with g_acbd = sum_J L^J_ac L^J_bd
(arXiv:2202.02019, Sec. II.A Cholesky form, Sec. II.B ladder).  The
gradients are the library's own contractions, each rebuilding its g or
Gamma tiles instead of storing them (the storage policy of App. A):

  dE/dL^J_ac    = 2 D^J_ac     (cc_ladder_density; Eq. integral_contraction
                                 carries the factor 2, D the V^4 part of W-tilde)
  dE/dtau_ij^cd = sum_ab tbar_ij^ab g_acbd   (cc_ladder_residual_adjoint)
  dE/dtbar      = Omega                      (cc_ladder_residual)

dE/dL = 2D holds for pair-symmetric tau and tbar (tau_ij^cd = tau_ji^dc), the
precondition of the library's packed algorithm; a perturbation direction
that breaks the pair symmetry of tau or tbar is outside that domain.
Nothing V^4-sized is saved for backward: only the three inputs.  The
chain-rule factors (2 and the incoming gradient of E) are applied by the
library (cc_ladder_scale_by), so this module does no arithmetic itself.
"""
from __future__ import annotations

import torch

from . import ladder as lad


class LadderEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, L_vv, tau, tbar2, prec="mixed"):
        sysd = lad.System(L_vv=L_vv.contiguous(), t2=tau.contiguous(), tbar2=tbar2.contiguous())
        E = lad.cc_ladder_lagrangian([sysd], omega=None, prec=prec)
        ctx.save_for_backward(sysd.L_vv, sysd.t2, sysd.tbar2)
        ctx.prec = prec
        return E[0]

    @staticmethod
    def backward(ctx, gE):
        L_vv, tau, tbar2 = ctx.saved_tensors
        sysd = lad.System(L_vv=L_vv, t2=tau, tbar2=tbar2)
        dL = dtau = dtbar = None
        g = gE.detach().to(device=L_vv.device, dtype=torch.float64).contiguous()
        if ctx.needs_input_grad[0]:
            dL = lad.cc_ladder_scale_by(lad.cc_ladder_density([sysd], prec=ctx.prec)[0], 2.0, g)
        if ctx.needs_input_grad[1]:
            dtau = lad.cc_ladder_scale_by(lad.cc_ladder_residual_adjoint([sysd], prec=ctx.prec)[0], 1.0, g)
        if ctx.needs_input_grad[2]:
            dtbar = lad.cc_ladder_scale_by(lad.cc_ladder_residual([sysd], prec=ctx.prec)[0], 1.0, g)
        return dL, dtau, dtbar, None


def ladder_energy(L_vv, tau, tbar2, prec="mixed"):
    """E(L, tau, tbar) with the hand-written backward above."""
    return LadderEnergy.apply(L_vv, tau, tbar2, prec)

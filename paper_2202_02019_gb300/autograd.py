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

The forward runs the work the backward can reuse: when dE/dL is wanted it is
one cc_ladder_step (Omega, D and E from one preparation, the residual and
density chains side by side), and Omega and D, both of input size (O^2 V^2 and
N_J V^2), are kept for backward; nothing V^4-sized is ever stored.  The
backward then only runs the adjoint ladder for dE/dtau.  The chain-rule
factors (2 and the incoming gradient of E) are applied by the library
(cc_ladder_scale_by), so this module does no arithmetic itself.
"""
from __future__ import annotations

import torch

from . import ladder as lad


class LadderEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, L_vv, tau, tbar2, prec="mixed"):
        sysd = lad.System(L_vv=L_vv.contiguous(), t2=tau.contiguous(), tbar2=tbar2.contiguous())
        need_L, need_tau, need_tbar = ctx.needs_input_grad[:3]
        if need_L:
            om, D, E = lad.cc_ladder_step([sysd], prec=prec)
            om, D = om[0], D[0]
        else:
            om = lad.cc_ladder_residual([sysd], prec=prec)[0]
            E = lad.cc_ladder_lagrangian([sysd], omega=[om], prec=prec)   # reduction over the given Omega
            D = None
        ctx.save_for_backward(sysd.L_vv if need_tau else None, sysd.t2 if need_tau else None,
                              sysd.tbar2 if need_tau else None, om if need_tbar else None, D)
        ctx.prec = prec
        return E[0]

    @staticmethod
    def backward(ctx, gE):
        L_vv, tau, tbar2, om, D = ctx.saved_tensors
        dL = dtau = dtbar = None
        dev = next(t for t in (D, om, L_vv) if t is not None).device
        g = gE.detach().to(device=dev, dtype=torch.float64).contiguous()
        if ctx.needs_input_grad[0]:
            dL = lad.cc_ladder_scale_by(D, 2.0, g)
        if ctx.needs_input_grad[1]:
            sysd = lad.System(L_vv=L_vv, t2=tau, tbar2=tbar2)
            dtau = lad.cc_ladder_scale_by(lad.cc_ladder_residual_adjoint([sysd], prec=ctx.prec)[0], 1.0, g)
        if ctx.needs_input_grad[2]:
            dtbar = lad.cc_ladder_scale_by(om, 1.0, g)
        return dL, dtau, dtbar, None


def ladder_energy(L_vv, tau, tbar2, prec="mixed"):
    """E(L, tau, tbar) with the hand-written backward above."""
    return LadderEnergy.apply(L_vv, tau, tbar2, prec)

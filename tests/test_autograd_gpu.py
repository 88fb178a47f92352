"""Differentiable ladder energy: autograd gradients vs the FP64 oracle's
gradients and vs central finite differences of the library's own E.

Size o=8, v=48, N_J=160 (the finite-difference workload).  Directions along
tau and tbar perturb a pair-symmetric couple (ij,cd) and (ji,dc) together:
the packed algorithm is defined on pair-symmetric amplitudes.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth
from paper_2202_02019_gb300.autograd import ladder_energy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 1e-6, "fp16x2": 1e-6}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fd_case():
    s, tb1, tb2 = synth.make_pair(8, 48, 160, 160 / 6.0, seed=2202)
    tt = O.tau(s.t1, s.t2)
    return s, tt, tb2


def _grads(s, tt, tb2, prec):
    d = torch.device("cuda")
    L = torch.tensor(s.L_vv, device=d, requires_grad=True)
    tau = torch.tensor(tt, device=d, requires_grad=True)
    tbar = torch.tensor(tb2, device=d, requires_grad=True)
    E = ladder_energy(L, tau, tbar, prec)
    E.backward()
    torch.cuda.synchronize()
    return float(E.detach()), L.grad.cpu().numpy(), tau.grad.cpu().numpy(), tbar.grad.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_gradients_match_oracle(fd_case, prec):
    s, tt, tb2 = fd_case
    E, gL, gT, gB = _grads(s, tt, tb2, prec)
    E_ref = O.lagrangian(tb2, O.residual_dense(s.L_vv, tt))
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert rel(gL, O.dE_dL_general(s.L_vv, tb2, tt)) < TOL[prec]
    assert rel(gT, O.dE_dtau(s.L_vv, tb2)) < TOL[prec]
    assert rel(gB, O.residual_dense(s.L_vv, tt)) < TOL[prec]


def test_central_differences_fp64(fd_case):
    s, tt, tb2 = fd_case
    d = torch.device("cuda")
    E0, gL, gT, gB = _grads(s, tt, tb2, "fp64")

    def E_of(L, t, b):
        sysd = lad.System(L_vv=torch.tensor(L, device=d), t2=torch.tensor(t, device=d),
                          tbar2=torch.tensor(b, device=d))
        e = lad.cc_ladder_lagrangian([sysd], omega=None, prec="fp64")
        torch.cuda.synchronize()
        return float(e[0])

    rng = np.random.default_rng(3)
    # E is quadratic in L (central differences exact) and linear in tau and
    # tbar (forward differences exact): h only trades against roundoff.
    h = 1e-3
    for _ in range(4):                                   # single L entries (L need not be symmetric)
        J, x, y = rng.integers(160), rng.integers(48), rng.integers(48)
        Lp = s.L_vv.copy(); Lp[J, x, y] += h
        Lm = s.L_vv.copy(); Lm[J, x, y] -= h
        fd = (E_of(Lp, tt, tb2) - E_of(Lm, tt, tb2)) / (2 * h)
        assert abs(fd - gL[J, x, y]) <= 1e-6 * max(1.0, abs(gL[J, x, y])), (fd, gL[J, x, y])
    for _ in range(3):                                   # pair-symmetric tau / tbar directions
        i, j, c, dd = rng.integers(8), rng.integers(8), rng.integers(48), rng.integers(48)
        for which in ("tau", "tbar"):
            t, b = tt.copy(), tb2.copy()
            arr = t if which == "tau" else b
            arr[i, j, c, dd] += h
            if (i, j, c, dd) != (j, i, dd, c):
                arr[j, i, dd, c] += h
            fd = (E_of(s.L_vv, t, b) - E0) / h            # E is linear in tau and in tbar
            g = gT if which == "tau" else gB
            an = g[i, j, c, dd] + (g[j, i, dd, c] if (i, j, c, dd) != (j, i, dd, c) else 0.0)
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (which, fd, an)


@pytest.mark.parametrize("which", ["L", "tau", "tbar"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_input_gradients(fd_case, prec, which):
    """Only one input requires grad: the forward takes the residual route when dE/dL is not
    wanted, and the gradient still matches the oracle."""
    s, tt, tb2 = fd_case
    d = torch.device("cuda")
    L = torch.tensor(s.L_vv, device=d, requires_grad=which == "L")
    tau = torch.tensor(tt, device=d, requires_grad=which == "tau")
    tbar = torch.tensor(tb2, device=d, requires_grad=which == "tbar")
    E = ladder_energy(L, tau, tbar, prec)
    E.backward()
    torch.cuda.synchronize()
    E_ref = O.lagrangian(tb2, O.residual_dense(s.L_vv, tt))
    assert abs(float(E.detach()) - E_ref) <= TOL[prec] * abs(E_ref)
    got = {"L": L, "tau": tau, "tbar": tbar}[which].grad.cpu().numpy()
    ref = {"L": lambda: O.dE_dL_general(s.L_vv, tb2, tt), "tau": lambda: O.dE_dtau(s.L_vv, tb2),
           "tbar": lambda: O.residual_dense(s.L_vv, tt)}[which]()
    assert rel(got, ref) < TOL[prec]
    for name, t in (("L", L), ("tau", tau), ("tbar", tbar)):
        if name != which:
            assert t.grad is None

"""GPU parity of the amplitude iteration (MP2-like driver + ladder + Jacobi step)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import iterate as I
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 1e-6, "fp16x2": 1e-6}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("o,v,nj", [(4, 20, 60), (5, 37, 70), (8, 48, 160)])
def test_driver_matches_oracle(o, v, nj, prec):
    s, _, _ = synth.make_pair(o, v, nj, nj / 6.0, seed=2202)
    ref = I.mp2_driver(s.L_ov)
    g = lad.cc_ladder_mp2_driver(dev(s.L_ov), prec=prec)
    gc = g.cpu().numpy()
    assert rel(gc, ref) < (1e-13 if prec == "fp64" else 1e-6)
    assert np.array_equal(gc, gc.transpose(1, 0, 3, 2))       # exactly pair symmetric
    # divided by the denominators it is the generator's MP2 guess
    assert rel(gc / I.denominators(s.eps, o), s.t2) < (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_iterations_match_oracle(prec):
    o, v, nj = 8, 48, 160
    s, _, _ = synth.make_pair(o, v, nj, nj / 6.0, seed=2202)
    L = 0.1 * s.L_vv
    g = I.mp2_driver(s.L_ov)
    t_ref, dn_ref = I.jacobi(L, s.t1, s.t2, g, s.eps, 3)
    sd = lad.System(L_vv=dev(L), t2=dev(s.t2), t1=dev(s.t1), eps=dev(s.eps))
    t, dn = lad.cc_ladder_iterate(sd, dev(g), 3, prec=prec)
    # each step adds at most the per-call error of the ladder (TOL, relative, divided by the
    # denominators), and the Jacobi map is contractive here, so after n steps the bound is n * TOL
    assert rel(t.cpu(), t_ref) < 3 * TOL[prec]
    assert np.allclose(dn.cpu().numpy(), dn_ref, rtol=1e-4 if prec != "fp64" else 1e-9, atol=0)
    # in place (t2_out = the starting amplitudes) gives the same result: the same bits on the split
    # paths; the FP64 path adds split-K partial sums with atomics, so only the summation order differs
    t0 = dev(s.t2)
    sd2 = lad.System(L_vv=dev(L), t2=t0, t1=dev(s.t1), eps=dev(s.eps))
    t_in, _ = lad.cc_ladder_iterate(sd2, dev(g), 3, prec=prec, out=t0)
    if prec == "fp64":
        assert rel(t_in.cpu(), t.cpu()) < 1e-14
    else:
        assert torch.equal(t_in, t)


def test_iteration_converges_to_the_direct_solution():
    o, v, nj = 4, 20, 60
    s, _, _ = synth.make_pair(o, v, nj, 12.0, seed=2202)
    L = 0.1 * s.L_vv
    g = I.mp2_driver(s.L_ov)
    t_star = I.fixed_point(L, s.t1, g, s.eps)
    sd = lad.System(L_vv=dev(L), t2=dev(np.zeros_like(s.t2)), t1=dev(s.t1), eps=dev(s.eps))
    t, dn = lad.cc_ladder_iterate(sd, dev(g), 40, prec="fp64")
    assert rel(t.cpu(), t_star) < 1e-10
    d = dn.cpu().numpy()
    assert d[-1] < 1e-20 * d[0]

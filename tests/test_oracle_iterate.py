"""Pins for the amplitude-iteration oracle (CPU only).

The MP2-like driver divided by the denominators must reproduce the
generator's MP2 guess (computed there in its own way); the Jacobi iteration
must converge to the direct solution of the fixed-point linear systems, and
that solution must zero the doubles residual written out in full.
"""
import numpy as np
import pytest

import oracle as O
from oracle import iterate as I
from paper_2202_02019_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def tiny():
    s, tb1, tb2 = synth.make_pair(*synth.CONFIGS["tiny"], seed=2202)
    return s


def test_driver_over_denominator_is_the_mp2_guess(tiny):
    s = tiny
    g = I.mp2_driver(s.L_ov)
    assert rel(g / I.denominators(s.eps, s.t2.shape[0]), s.t2) < 1e-13
    # pair symmetry g_aibj = g_bjai holds exactly
    assert np.array_equal(g, g.transpose(1, 0, 3, 2))


def test_first_step_without_ladder_is_mp2(tiny):
    s = tiny
    g = I.mp2_driver(s.L_ov)
    t, dn = I.jacobi(np.zeros_like(s.L_vv), None, np.zeros_like(s.t2), g, s.eps, 1)
    assert rel(t, s.t2) < 1e-13
    assert abs(dn[0] - np.sum(s.t2 ** 2)) < 1e-12 * np.sum(s.t2 ** 2)


def test_jacobi_converges_to_the_direct_solution(tiny):
    s = tiny
    L = 0.1 * s.L_vv          # keep the ladder small against the denominators: Jacobi contracts
    g = I.mp2_driver(s.L_ov)
    t_star = I.fixed_point(L, s.t1, g, s.eps)
    o = s.t2.shape[0]
    D = I.denominators(s.eps, o)
    # the direct solution zeroes the residual written out in full
    res = g + O.residual_dense(L, O.tau(s.t1, t_star)) - D * t_star
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(g))
    t, dn = I.jacobi(L, s.t1, np.zeros_like(s.t2), g, s.eps, 60)
    assert rel(t, t_star) < 1e-12
    assert np.all(np.diff(np.log(dn[:20])) < 0)       # monotone geometric decrease

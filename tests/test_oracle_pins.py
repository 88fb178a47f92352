"""Pins for the oracle functions that the ladder pins do not reach (CPU only).

Each function is tied to hand-computed values in
tests/golden/hand_update_es_ov3.json (worked from the paper's definitions, not
from the oracle) and, where one exists, to a second route:

* ``update_t2`` (the Jacobi step with orbital-energy denominators) equals one
  step of ``iterate.jacobi`` when it is given the full doubles residual
  g + ladder - Delta t, and leaves the amplitudes of ``iterate.fixed_point``
  unchanged;
* ``t1.es_amplitudes`` (U = T2 R0 + R2, App. A) through the V^4 density;
* ``ov3.density_abic_gs`` (d^gs_abic = L^a_m t~^cb_im R0) and
  ``ov3.density_abci_es`` (d^es_abci = L_ji^ac R_j^b).

Each golden case is built so that the plausible slips fail it: a swapped
occupied pair or swapped virtual pair in t~ or L2, R0 on the wrong term, a
denominator with the wrong sign or with occupied and virtual energies mixed
up.  ``test_planted_*`` plant those slips in copies of the oracle code and
check that the golden values reject them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import iterate as I
from oracle import ov3 as V
from oracle import t1 as T
from paper_2202_02019_gb300 import synth

HERE = os.path.dirname(__file__)
G = json.load(open(os.path.join(HERE, "golden", "hand_update_es_ov3.json")))
A = lambda x: np.array(x, dtype=np.float64)


# ------------------------------------------------------------------ update_t2
@pytest.mark.parametrize("case", G["update"], ids=lambda c: c["name"])
def test_update_t2_hand_values(case):
    got = O.update_t2(A(case["t2"]), A(case["omega"]), A(case["eps"]), case["o"])
    assert np.array_equal(got, A(case["t_new"]))


def test_update_t2_is_one_jacobi_step_and_fixes_the_fixed_point():
    s = synth.make_system(2, 5, 7, 4.0, seed=13)
    o = s.o
    g = I.mp2_driver(s.L_ov)
    Delta = I.denominators(s.eps, o)
    t = s.t2
    # the full doubles residual of the model: driver + ladder - Delta t
    resid = g + O.residual_dense(s.L_vv, O.tau(s.t1, t)) - Delta * t
    t_step, _ = I.jacobi(s.L_vv, s.t1, t, g, s.eps, 1)
    assert np.allclose(O.update_t2(t, resid, s.eps, o), t_step, rtol=1e-13, atol=1e-15)
    # at the fixed point the residual vanishes and the step changes nothing
    tf = I.fixed_point(s.L_vv, s.t1, g, s.eps)
    rf = g + O.residual_dense(s.L_vv, O.tau(s.t1, tf)) - Delta * tf
    assert np.max(np.abs(rf)) < 1e-11 * np.max(np.abs(g))
    assert np.allclose(O.update_t2(tf, rf, s.eps, o), tf, rtol=1e-12, atol=1e-15)


def test_planted_update_mistakes_fail_the_golden_values():
    def wrong_sign(t2, om, eps, o):
        eo, ev = eps[:o], eps[o:]
        den = ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None]
        return t2 + om / den

    def occ_virt_mixed(t2, om, eps, o):
        # occupied energies indexed by the virtual indices and vice versa
        v = t2.shape[2]
        e1, e2 = eps[:v], eps[v:]
        den = (e2[:, None, None, None] + e2[None, :, None, None]
               - e1[None, None, :, None] - e1[None, None, None, :])
        return t2 + om / den

    for wrong in (wrong_sign, occ_virt_mixed):
        caught = False
        for case in G["update"]:
            try:
                got = wrong(A(case["t2"]), A(case["omega"]), A(case["eps"]), case["o"])
            except ValueError:
                caught = True
                continue
            caught |= not np.allclose(got, A(case["t_new"]))
        assert caught, wrong.__name__


# ------------------------------------------------------------------ es_amplitudes
def test_es_amplitudes_hand_values_through_the_density():
    c = G["es_density"]
    U = T.es_amplitudes(A(c["t2"]), A(c["R2"]), c["R0"])
    assert np.array_equal(U, A(c["U"]))
    D = O.density_dense(A(c["L_vv"]), A(c["L2"]), U)
    assert np.allclose(D, A(c["D"]), rtol=0, atol=1e-12)
    assert abs(O.euler_lagrangian(A(c["L_vv"]), D) - 57.0) < 1e-12


def test_planted_es_amplitude_mistakes_fail_the_golden_values():
    c = G["es_density"]
    wrong = {
        "R0 on R2": lambda t2, r2, r0: t2 + r0 * r2,
        "R0 dropped": lambda t2, r2, r0: t2 + r2,
        "R2 dropped": lambda t2, r2, r0: r0 * t2,
    }
    for name, f in wrong.items():
        D = O.density_dense(A(c["L_vv"]), A(c["L2"]), f(A(c["t2"]), A(c["R2"]), c["R0"]))
        assert not np.allclose(D, A(c["D"])), name


# ------------------------------------------------------------------ OV^3 density blocks
def test_density_abic_gs_hand_values():
    c = G["ov3_gs_abic"]
    d = V.density_abic_gs(A(c["tbar1"]), A(c["t2"]), c["R0"])
    assert np.allclose(d, A(c["d"]), rtol=0, atol=1e-14)


def test_density_abci_es_hand_values():
    c = G["ov3_es_abci"]
    d = V.density_abci_es(A(c["L2"]), A(c["R1"]))
    assert np.allclose(d, A(c["d"]), rtol=0, atol=1e-14)


def test_planted_ov3_transpositions_fail_the_golden_values():
    c = G["ov3_gs_abic"]
    tb1, t2, R0 = A(c["tbar1"]), A(c["t2"]), c["R0"]
    tt = 2.0 * t2 - t2.transpose(1, 0, 2, 3)
    wrong_gs = {
        "t~ virtual pair swapped (imbc)": R0 * np.einsum("ma,imbc->abic", tb1, tt),
        "t~ occupied pair swapped (micb)": R0 * np.einsum("ma,micb->abic", tb1, tt),
        "t instead of t~": R0 * np.einsum("ma,imcb->abic", tb1, t2),
        "t~ exchange term with the wrong sign (2t + t_ji)": R0 * np.einsum(
            "ma,imcb->abic", tb1, 2.0 * t2 + t2.transpose(1, 0, 2, 3)),
        "R0 dropped": np.einsum("ma,imcb->abic", tb1, tt),
    }
    for name, bad in wrong_gs.items():
        assert not np.allclose(bad, A(c["d"])), name
    e = G["ov3_es_abci"]
    L2, R1 = A(e["L2"]), A(e["R1"])
    wrong_es = {
        "L2 occupied pair swapped (ijac)": np.einsum("ijac,jb->abci", L2, R1),
        "L2 virtual pair swapped (jica)": np.einsum("jica,jb->abci", L2, R1),
        "R1 on the wrong occupied index": np.einsum("jiac,ib->abci", L2, R1),
    }
    for name, bad in wrong_es.items():
        assert not np.allclose(bad, A(e["d"])), name

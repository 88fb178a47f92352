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


# ------------------------------------------------------------------ excited-state d_abic (App. A)
def _dense(entries, shape):
    x = np.zeros(shape)
    for e in entries:
        x[tuple(e[:-1])] = e[-1]
    return x


def test_density_abic_es_hand_values():
    c = G["ov3_es_abic_Rtilde"]
    z2 = np.zeros((2, 2, 2, 2))
    d = V.density_abic_es(A(c["tbar1"]), z2, z2, 0.0, np.zeros((2, 2)), A(c["R2"]))
    assert np.allclose(d, A(c["d"]), rtol=0, atol=1e-14)
    c = G["ov3_es_abic_R1_sparse"]
    L2 = _dense(c["L2_nonzero"], (2, 2, 2, 2))
    t2 = _dense(c["t2_nonzero"], (2, 2, 2, 2))
    R1 = _dense(c["R1_nonzero"], (2, 2))
    assert np.array_equal(L2, L2.transpose(1, 0, 3, 2)) and np.array_equal(t2, t2.transpose(1, 0, 3, 2))
    d = V.density_abic_es(np.zeros((2, 2)), L2, t2, 0.0, R1, np.zeros((2, 2, 2, 2)))
    assert np.allclose(d, _dense(c["d_nonzero"], (2, 2, 2, 2)), rtol=0, atol=1e-14)


def _es_case(o, v, seed):
    s, tb1, L2 = synth.make_pair(o, v, 5, 4.0, seed=seed)
    rng = np.random.default_rng(seed)
    R1 = rng.standard_normal((o, v))
    R2 = rng.standard_normal((o, o, v, v))
    R2 = 0.5 * (R2 + R2.transpose(1, 0, 3, 2))
    return s, tb1, L2, R1, R2


def test_density_abic_es_reduces_to_the_ground_state_and_cancels_in_one_orbital_spaces():
    s, tb1, L2, R1, R2 = _es_case(3, 6, 21)
    # no excitation: the ground-state block (itself pinned by hand values)
    assert np.allclose(V.density_abic_es(tb1, L2, s.t2, 0.8, 0 * R1, 0 * R2), V.density_abic_gs(tb1, s.t2, 0.8),
                       rtol=0, atol=1e-15)
    # one occupied or one virtual orbital (pair-symmetric inputs): the six R1 terms cancel exactly,
    # 2 X - X - X and -2 (V + Y) + (L t~ R) + Y~ pair off term by term
    for o, v in ((1, 6), (5, 1)):
        s1, tb, L2b, R1b, _ = _es_case(o, v, 5)
        d = V.density_abic_es(np.zeros_like(tb), L2b, s1.t2, 0.0, R1b, np.zeros_like(s1.t2))
        assert np.max(np.abs(d)) < 1e-13 * max(1.0, np.max(np.abs(L2b)) * np.max(np.abs(s1.t2)))


def test_w_ov3_es_abic_factorised_and_finite_differences():
    s, tb1, L2, R1, R2 = _es_case(3, 7, 9)
    d = V.density_abic_es(tb1, L2, s.t2, 0.6, R1, R2)
    We, Wo = V.w_from_abic(d, s.L_vv, s.L_ov)
    Fe, Fo = V.w_ov3_es_abic(tb1, L2, s.t2, 0.6, R1, R2, s.L_vv, s.L_ov)
    assert np.linalg.norm(Fe - We) < 1e-13 * np.linalg.norm(We)
    assert np.linalg.norm(Fo - Wo) < 1e-13 * np.linalg.norm(Wo)

    def energy(Lvv, Lov):       # sum_abic d_abic (ab|ic), (ab|ic) = sum_K L^K_ab L^K_ic
        return float(np.einsum("abic,Kab,Kic->", d, Lvv, Lov))

    h = 1e-6
    for (K, a, b) in [(0, 1, 2), (4, 6, 0)]:
        Lp = s.L_vv.copy(); Lp[K, a, b] += h
        Lm = s.L_vv.copy(); Lm[K, a, b] -= h
        fd = (energy(Lp, s.L_ov) - energy(Lm, s.L_ov)) / (2 * h)
        assert abs(fd - Fe[K, a, b]) < 1e-7 * max(1.0, abs(fd))
    for (K, i, c) in [(1, 0, 3), (3, 2, 6)]:
        Lp = s.L_ov.copy(); Lp[K, i, c] += h
        Lm = s.L_ov.copy(); Lm[K, i, c] -= h
        fd = (energy(s.L_vv, Lp) - energy(s.L_vv, Lm)) / (2 * h)
        assert abs(fd - Fo[K, i, c]) < 1e-7 * max(1.0, abs(fd))


def test_planted_es_abic_mistakes_fail_the_pins():
    c = G["ov3_es_abic_R1_sparse"]
    L2 = _dense(c["L2_nonzero"], (2, 2, 2, 2))
    t2 = _dense(c["t2_nonzero"], (2, 2, 2, 2))
    R1 = _dense(c["R1_nonzero"], (2, 2))
    ref = _dense(c["d_nonzero"], (2, 2, 2, 2))
    good = V.density_abic_es(np.zeros((2, 2)), L2, t2, 0.0, R1, np.zeros((2, 2, 2, 2)))
    tt = V.t_tilde(t2)
    wrong = {
        "t~ virtual pair swapped in the W_am term": good - np.einsum("mkad,mibc,kd->abic", L2, tt, R1)
        + np.einsum("mkad,micb,kd->abic", L2, tt, R1),
        "sign of the B t term": good + 2 * np.einsum("mnad,mnbc,id->abic", L2, t2, R1),
        "2 Y in place of Y~ (the Sec. II.C variant)": good - np.einsum("akci,kb->abic", V.ytilde_djak(L2, t2), R1)
        + 2 * np.einsum("akci,kb->abic", V.y_ajbi(L2, t2), R1),
        "X_ab R^c_i without its 2": good - np.einsum("ab,ic->abic", V.x_ab(L2, t2), R1),
    }
    for name, bad in wrong.items():
        assert not np.allclose(bad, ref), name
    c = G["ov3_es_abic_Rtilde"]
    z2 = np.zeros((2, 2, 2, 2))
    Rt = V.t_tilde(A(c["R2"]))
    plain = np.einsum("ma,imcb->abic", A(c["tbar1"]), Rt)   # the U-tilde reading, L^a_m R~^cb_im
    assert not np.allclose(plain, A(c["d"]))

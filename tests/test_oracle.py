"""Pins for the FP64 oracle (CPU only).

Each test ties the oracle to something other than itself: hand-computed
values, matrix closed forms, finite differences, algebraic identities, or a
second formulation with different arithmetic.  A plausible slip in the
oracle (dropped term, swapped index, wrong sign, transposed operand) fails
at least one of these; ``test_planted_mistakes_are_caught`` checks that on
purpose-built wrong variants.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2202_02019_gb300 import synth

HERE = os.path.dirname(__file__)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def tiny():
    s, tb1, tb2 = synth.make_pair(*synth.CONFIGS["tiny"], seed=2202)
    return s, tb2, O.tau(s.t1, s.t2)


@pytest.fixture(scope="module")
def odd():
    # ragged odd sizes, o = 3, v = 7, nj = 5
    s, tb1, tb2 = synth.make_pair(3, 7, 5, 4.0, seed=7)
    return s, tb2, O.tau(s.t1, s.t2)


# ------------------------------------------------------------------ generator
def test_generator_deterministic_and_structured():
    a = synth.make_system(3, 5, 4, 12.0, seed=11)
    b = synth.make_system(3, 5, 4, 12.0, seed=11)
    c = synth.make_system(3, 5, 4, 12.0, seed=12)
    assert np.array_equal(a.L_vv, b.L_vv) and np.array_equal(a.t2, b.t2)
    assert not np.array_equal(a.L_vv, c.L_vv)
    # symmetric Cholesky slices, pair-symmetric t2 (bit exact)
    assert np.array_equal(a.L_vv, a.L_vv.transpose(0, 2, 1))
    assert np.array_equal(a.t2, a.t2.transpose(1, 0, 3, 2))
    # energy windows
    assert np.all(a.eps[:3] < -0.3) and np.all(a.eps[:3] >= -2)
    assert np.all(a.eps[3:] > 0.1) and np.all(a.eps[3:] <= 5)
    # lambda_J decay of the slice norms: ||L^J|| ~ sqrt(lambda_J) * O(n)
    s = synth.make_system(2, 30, 40, 12.0, seed=3)
    norms = np.linalg.norm(s.L_vv.reshape(40, -1), axis=1)
    ratio = norms[30:].mean() / norms[:10].mean()
    expect = np.exp(-30 / 24.0) / np.exp(-4.5 / 24.0)   # sqrt(lambda) ratio, roughly
    assert 0.3 * expect < ratio < 3 * expect


def test_mp2_guess_formula():
    s = synth.make_system(2, 3, 5, 12.0, seed=5)
    i, j, a, b = 1, 0, 2, 1
    g = np.sum(s.L_ov[:, i, a] * s.L_ov[:, j, b])
    den = s.eps[i] + s.eps[j] - s.eps[2 + a] - s.eps[2 + b]
    assert abs(s.t2[i, j, a, b] - g / den) < 1e-14 * abs(g / den) + 1e-300


def test_batch_sizes():
    sz = synth.batch_sizes()
    assert len(sz) == 24
    for o, v, nj in sz:
        assert 6 <= o <= 40 and 50 <= v <= 300 and nj == 5 * v
    assert sz == synth.batch_sizes()


# ------------------------------------------------------------------ golden
def test_hand_computed_golden():
    d = json.load(open(os.path.join(HERE, "golden", "hand_o1_v2.json")))
    for c in d["cases"]:
        L = np.array(c["L_vv"], float)
        t1 = np.array(c["t1"], float)
        t2 = np.array(c["t2"], float)
        tb = np.array(c["tbar2"], float)
        tt = O.tau(t1, t2)
        om = O.residual_dense(L, tt)
        D = O.density_dense(L, tb, tt)
        assert np.allclose(om, np.array(c["omega"]), rtol=0, atol=1e-12), c["name"]
        assert np.allclose(D, np.array(c["D"]), rtol=0, atol=1e-12), c["name"]
        assert abs(O.lagrangian(tb, om) - c["E"]) < 1e-12
        assert abs(O.euler_lagrangian(L, D) - c["E"]) < 1e-12
        assert np.allclose(O.residual_rows(L, tt), om, atol=1e-12)
        assert np.allclose(O.density_rows(L, tb, tt), D, atol=1e-12)


# ------------------------------------------------------------------ formulations agree
@pytest.mark.parametrize("fx", ["tiny", "odd"])
def test_three_formulations_agree(fx, request):
    s, tb, tt = request.getfixturevalue(fx)
    om_d = O.residual_dense(s.L_vv, tt)
    om_r = O.residual_rows(s.L_vv, tt)
    om_p = O.residual_pm(s.L_vv, tt)
    assert rel(om_r, om_d) < 1e-13
    assert rel(om_p, om_d) < 1e-13
    D_d = O.density_dense(s.L_vv, tb, tt)
    D_r = O.density_rows(s.L_vv, tb, tt)
    D_p = O.density_pm(s.L_vv, tb, tt)
    assert rel(D_r, D_d) < 1e-13
    assert rel(D_p, D_d) < 1e-13


def test_rows_subset(tiny):
    s, tb, tt = tiny
    rows = [0, 7, 19]
    om, D = O.sampled_rows(s.L_vv, s.t1, s.t2, tb, rows)
    om_d = O.residual_dense(s.L_vv, tt)
    D_d = O.density_dense(s.L_vv, tb, tt)
    assert rel(om, om_d[:, :, rows, :]) < 1e-13
    assert rel(D, D_d[:, rows, :]) < 1e-13
    cols = [3, 4, 11, 18]
    om2, D2 = O.sampled_rows(s.L_vv, s.t1, s.t2, tb, rows, cols)
    assert rel(om2, om_d[:, :, rows, :][:, :, :, cols]) < 1e-13
    assert rel(D2, D_d[:, rows, :][:, :, cols]) < 1e-13


# ------------------------------------------------------------------ symmetries
def test_pair_symmetries(tiny):
    s, tb, tt = tiny
    g = O.g_vvvv(s.L_vv)                                   # [a,c,b,d]
    assert rel(g, g.transpose(2, 3, 0, 1)) < 1e-15         # g_acbd = g_bdac
    om = O.residual_dense(s.L_vv, tt)
    assert rel(om, om.transpose(1, 0, 3, 2)) < 1e-13       # Omega_ij^ab = Omega_ji^ba
    G = O.gamma_dense(tb, tt)
    assert rel(G, G.transpose(1, 0, 3, 2)) < 1e-13         # Gamma_abcd = Gamma_badc


# ------------------------------------------------------------------ identities
@pytest.mark.parametrize("fx", ["tiny", "odd"])
def test_euler_identity(fx, request):
    s, tb, tt = request.getfixturevalue(fx)
    om = O.residual_dense(s.L_vv, tt)
    D = O.density_dense(s.L_vv, tb, tt)
    E = O.lagrangian(tb, om)
    assert abs(O.euler_lagrangian(s.L_vv, D) - E) < 1e-12 * abs(E)


def test_homogeneity_and_linearity(tiny):
    s, tb, tt = tiny
    L = s.L_vv
    om = O.residual_dense(L, tt)
    D = O.density_dense(L, tb, tt)
    al = 1.7
    assert rel(O.residual_dense(al * L, tt), al ** 2 * om) < 1e-13
    # with tau and tbar held fixed, D is linear in L (Gamma does not involve L)
    assert rel(O.density_dense(al * L, tb, tt), al * D) < 1e-13
    rng = np.random.default_rng(0)
    t2b = rng.standard_normal(tt.shape)
    t2b = 0.5 * (t2b + t2b.transpose(1, 0, 3, 2))
    assert rel(O.residual_dense(L, tt + 2 * t2b),
               om + 2 * O.residual_dense(L, t2b)) < 1e-12
    assert rel(O.density_dense(L, 3 * tb, tt), 3 * D) < 1e-13


# ------------------------------------------------------------------ closed forms
def test_closed_form_nj1():
    s, tb1, tb = synth.make_pair(3, 6, 1, 12.0, seed=21)
    L = s.L_vv
    tt = O.tau(s.t1, s.t2)
    om = O.residual_dense(L, tt)
    D = O.density_dense(L, tb, tt)
    L1 = L[0]
    for i in range(3):
        for j in range(3):
            assert np.allclose(om[i, j], L1 @ tt[i, j] @ L1.T, rtol=1e-13, atol=1e-14)
    Dm = sum(tb[i, j] @ L1 @ tt[i, j].T for i in range(3) for j in range(3))
    assert np.allclose(D[0], Dm, rtol=1e-12, atol=1e-14)


def test_closed_form_one_hot():
    v, o = 4, 2
    nj = v * v
    L = np.zeros((nj, v, v))
    for a in range(v):
        for c in range(v):
            L[a * v + c, a, c] = 1.0                 # L^J_ac = delta_{J,(a,c)}
    rng = np.random.default_rng(1)
    t2 = rng.standard_normal((o, o, v, v))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    g = O.g_vvvv(L)
    eye = np.eye(v)
    assert np.array_equal(g, np.einsum("ab,cd->acbd", eye, eye))   # g_acbd = d_ab d_cd
    om = O.residual_dense(L, t2)
    tr = np.einsum("ijcc->ij", t2)
    assert np.allclose(om, np.einsum("ab,ij->ijab", eye, tr), atol=1e-14)


def test_t1_zero_and_o1():
    s, tb1, tb = synth.make_pair(1, 5, 3, 12.0, seed=4)
    assert np.array_equal(O.tau(None, s.t2), s.t2)
    assert np.array_equal(O.tau(np.zeros_like(s.t1), s.t2), s.t2)
    # o = 1: tau is a single symmetric v x v matrix; check tau explicitly
    tt = O.tau(s.t1, s.t2)
    assert np.allclose(tt[0, 0], s.t2[0, 0] + np.outer(s.t1[0], s.t1[0]), atol=0)
    om = O.residual_dense(s.L_vv, tt)
    ref = sum(s.L_vv[J] @ tt[0, 0] @ s.L_vv[J].T for J in range(3))
    assert np.allclose(om[0, 0], ref, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ finite differences
def _E(L, tt, tb):
    return O.lagrangian(tb, O.residual_dense(L, tt))


def test_fd_dE_dL_equals_2D():
    s, tb1, tb = synth.make_pair(2, 6, 3, 4.0, seed=31)
    tt = O.tau(s.t1, s.t2)
    L = s.L_vv.copy()
    D = O.density_dense(L, tb, tt)
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(12):
        J, x, y = rng.integers(3), rng.integers(6), rng.integers(6)
        Lp = L.copy(); Lp[J, x, y] += h
        Lm = L.copy(); Lm[J, x, y] -= h
        fd = (_E(Lp, tt, tb) - _E(Lm, tt, tb)) / (2 * h)
        assert abs(fd - 2 * D[J, x, y]) < 1e-7 * max(1.0, abs(fd)), (J, x, y, fd, 2 * D[J, x, y])


def test_fd_general_gradient_without_pair_symmetry():
    rng = np.random.default_rng(9)
    o, v, nj = 2, 4, 3
    L = rng.standard_normal((nj, v, v))           # non-symmetric L
    tt = rng.standard_normal((o, o, v, v))        # no pair symmetry
    tb = rng.standard_normal((o, o, v, v))
    G = O.dE_dL_general(L, tb, tt)
    h = 1e-6
    for J, x, y in [(0, 1, 2), (2, 3, 0), (1, 0, 0)]:
        Lp = L.copy(); Lp[J, x, y] += h
        Lm = L.copy(); Lm[J, x, y] -= h
        fd = (_E(Lp, tt, tb) - _E(Lm, tt, tb)) / (2 * h)
        assert abs(fd - G[J, x, y]) < 1e-7 * max(1.0, abs(fd))


def test_fd_dE_dtau():
    rng = np.random.default_rng(10)
    o, v, nj = 2, 4, 3
    L = rng.standard_normal((nj, v, v))
    tt = rng.standard_normal((o, o, v, v))
    tb = rng.standard_normal((o, o, v, v))
    G = O.dE_dtau(L, tb)
    # E is linear in tau: a single difference is exact up to rounding
    for idx in [(0, 1, 2, 3), (1, 1, 0, 0)]:
        tp = tt.copy(); tp[idx] += 1.0
        assert abs((_E(L, tp, tb) - _E(L, tt, tb)) - G[idx]) < 1e-11 * max(1.0, abs(G[idx]))
    # with symmetric L the transposed ladder is the ladder applied to tbar
    Ls = 0.5 * (L + L.transpose(0, 2, 1))
    assert rel(O.dE_dtau(Ls, tb), O.residual_dense(Ls, tb)) < 1e-13


def test_update_step():
    s = synth.make_system(2, 3, 4, 12.0, seed=8)
    om = np.ones_like(s.t2)
    t = O.update_t2(s.t2, om, s.eps, 2)
    i, j, a, b = 1, 0, 2, 0
    den = s.eps[i] + s.eps[j] - s.eps[2 + a] - s.eps[2 + b]
    assert abs(t[i, j, a, b] - (s.t2[i, j, a, b] + 1.0 / den)) < 1e-15


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistakes_are_caught(tiny):
    """Wrong variants of the residual/density fail the independent pins."""
    s, tb, tt = tiny
    L = s.L_vv
    good_om = O.residual_dense(L, tt)
    wrong_residuals = {
        "swapped g pairing": np.einsum("abcd,ijcd->ijab", O.g_vvvv(L), tt),
        "transposed tau": np.einsum("acbd,ijdc->ijab", O.g_vvvv(L), tt),
        "dropped t1 term": O.residual_dense(L, s.t2),
    }
    d = json.load(open(os.path.join(HERE, "golden", "hand_o1_v2.json")))["cases"][2]
    Lh = np.array(d["L_vv"], float)
    tth = O.tau(np.array(d["t1"], float), np.array(d["t2"], float))
    for name, bad in wrong_residuals.items():
        assert rel(bad, good_om) > 1e-6, name
    # the golden case catches the dropped-t1 slip on its own
    assert not np.allclose(O.residual_dense(Lh, np.array(d["t2"], float)), np.array(d["omega"]))
    # a density with the wrong L index fails the Euler identity
    G = O.gamma_dense(tb, tt)
    D_bad = np.einsum("abcd,Jdb->Jac", G, L + 0.1 * np.eye(L.shape[1]))
    E = O.lagrangian(tb, good_om)
    assert abs(O.euler_lagrangian(L, D_bad) - E) > 1e-6 * abs(E)

"""Pins for the T1-transformed-basis and excited-state oracle (CPU only).

The T1 transformation (Sec. II.C) is pinned to results that follow from its
definition but are computed another way: the four-index transform of the
integrals against the three-index transform of the Cholesky vectors, the
textbook property that the occupied-virtual block (the one that builds the
(ia|jb) integrals) is left unchanged while the occupied-occupied block picks
up L_ia t_j^a, the inverse transform, the adjoint relation that fixes the
back-transformation of W, and central finite differences of the T1-form
Lagrangian with respect to the MO occupied-virtual Cholesky block.
"""
import numpy as np
import pytest

import oracle as O
from oracle import t1 as T


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def rnd():
    rng = np.random.default_rng(11)
    o, v, nj = 2, 3, 4
    n = o + v
    L = rng.standard_normal((nj, n, n))            # not symmetric on purpose
    t1 = 0.3 * rng.standard_normal((o, v))
    return o, v, nj, L, t1


def test_zero_singles_is_identity(rnd):
    o, v, nj, L, t1 = rnd
    z = np.zeros_like(t1)
    assert np.array_equal(T.t1_transform_full(L, z), L)
    assert np.array_equal(T.w_backtransform_full(L, z), L)


def test_four_index_transform_matches_cholesky_transform(rnd):
    o, v, nj, L, t1 = rnd
    g_mo = np.einsum("Jpq,Jrs->pqrs", L, L)
    Lt = T.t1_transform_full(L, t1)
    assert rel(np.einsum("Jpq,Jrs->pqrs", Lt, Lt), T.g_t1_full(g_mo, t1)) < 1e-14


def test_textbook_blocks(rnd):
    # ov block unchanged; oo block L_ij + sum_a L_ia t_j^a; vv block L_ac - sum_i t_i^a L_ic
    o, v, nj, L, t1 = rnd
    Lt = T.t1_transform_full(L, t1)
    assert np.allclose(Lt[:, :o, o:], L[:, :o, o:], rtol=0, atol=1e-15)
    assert rel(Lt[:, :o, :o], L[:, :o, :o] + np.einsum("Jia,ja->Jij", L[:, :o, o:], t1)) < 1e-14
    assert rel(Lt[:, o:, o:], L[:, o:, o:] - np.einsum("ia,Jic->Jac", t1, L[:, :o, o:])) < 1e-14


def test_inverse_transform(rnd):
    o, v, nj, L, t1 = rnd
    assert rel(T.t1_transform_full(T.t1_transform_full(L, t1), -t1), L) < 1e-14


def test_backtransform_is_the_adjoint(rnd):
    # sum W^MO . L^MO = sum W . L^T1: the chain rule that defines W^MO
    o, v, nj, L, t1 = rnd
    W = np.random.default_rng(5).standard_normal(L.shape)
    lhs = np.sum(T.w_backtransform_full(W, t1) * L)
    rhs = np.sum(W * T.t1_transform_full(L, t1))
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)


def test_backtransform_of_a_vv_only_w(rnd):
    # W nonzero in the vv block only: W^MO keeps vv and gains ov = -sum_a t_i^a W_ac
    o, v, nj, L, t1 = rnd
    W = np.zeros_like(L)
    W[:, o:, o:] = np.random.default_rng(6).standard_normal((nj, v, v))
    Wm = T.w_backtransform_full(W, t1)
    assert np.allclose(Wm[:, o:, o:], W[:, o:, o:], rtol=0, atol=1e-15)
    assert rel(Wm[:, :o, o:], -np.einsum("ia,Jac->Jic", t1, W[:, o:, o:])) < 1e-14
    assert np.allclose(Wm[:, :, :o], 0.0, rtol=0, atol=1e-15)


def _t1_energy(L_full, t1, t2, tb2):
    o = t1.shape[0]
    Lt = T.t1_transform_vv(L_full, t1)
    return O.lagrangian(tb2, O.residual_dense(Lt, t2))


def test_fd_t1_form_gradient_wrt_mo_ov_block():
    # E(L^MO) = tbar . ladder(L^T1_vv(L^MO), t2): dE/dL^MO_ic = 2 (W^MO)_ic with W = D in the vv block
    rng = np.random.default_rng(3)
    o, v, nj = 2, 4, 3
    n = o + v
    L = rng.standard_normal((nj, n, n))
    t1 = 0.2 * rng.standard_normal((o, v))
    t2 = rng.standard_normal((o, o, v, v)); t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    tb = rng.standard_normal((o, o, v, v)); tb = 0.5 * (tb + tb.transpose(1, 0, 3, 2))
    Lt = T.t1_transform_vv(L, t1)
    D = O.density_dense(Lt, tb, t2)
    W = np.zeros_like(L)
    W[:, o:, o:] = D
    grad = 2.0 * T.w_backtransform_full(W, t1)
    h = 1e-5
    for (J, i, c) in [(0, 0, 0), (1, 1, 2), (2, 0, 3)]:
        Lp = L.copy(); Lp[J, i, o + c] += h
        Lm = L.copy(); Lm[J, i, o + c] -= h
        fd = (_t1_energy(Lp, t1, t2, tb) - _t1_energy(Lm, t1, t2, tb)) / (2 * h)
        assert abs(fd - grad[J, i, o + c]) < 1e-7 * max(1.0, abs(fd))
    # and the vv block: dE/dL^MO_ac = 2 D_ac
    for (J, a, c) in [(0, 1, 2), (2, 3, 0)]:
        Lp = L.copy(); Lp[J, o + a, o + c] += h
        Lm = L.copy(); Lm[J, o + a, o + c] -= h
        fd = (_t1_energy(Lp, t1, t2, tb) - _t1_energy(Lm, t1, t2, tb)) / (2 * h)
        assert abs(fd - 2.0 * D[J, a, c]) < 1e-7 * max(1.0, abs(fd))


def test_es_amplitudes():
    rng = np.random.default_rng(4)
    t2 = rng.standard_normal((2, 2, 3, 3)); r2 = rng.standard_normal((2, 2, 3, 3))
    assert np.array_equal(T.es_amplitudes(t2, r2, 0.0), r2)
    assert np.array_equal(T.es_amplitudes(t2, np.zeros_like(r2), 1.0), t2)
    assert rel(T.es_amplitudes(t2, r2, -0.5), r2 - 0.5 * t2) < 1e-16


def test_planted_t1_mistakes_are_caught(rnd):
    # a transposed singles block and a flipped sign both break the textbook-block pin
    o, v, nj, L, t1 = rnd
    n = o + v
    for bad in ("transpose", "sign"):
        Tm = np.zeros((n, n))
        if bad == "transpose":
            Tm[:o, o:] = t1
        else:
            Tm[o:, :o] = -t1.T
        x, y = np.eye(n) - Tm, np.eye(n) + Tm.T
        Lt = np.einsum("pr,Jrs,qs->Jpq", x, L, y)
        ok_ov = np.allclose(Lt[:, :o, o:], L[:, :o, o:], rtol=0, atol=1e-15)
        ok_vv = rel(Lt[:, o:, o:], L[:, o:, o:] - np.einsum("ia,Jic->Jac", t1, L[:, :o, o:])) < 1e-14
        assert not (ok_ov and ok_vv), bad

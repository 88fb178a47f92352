"""Pins for the OV^3 contribution oracle (CPU only): the explicit density route
against the factorised one, finite differences of the OV^3 energy term
sum d_abic (ab|ic) with (ab|ic) = sum_K L^K_ab L^K_ic, and the symmetry of
the t~ matrix that the GPU path relies on."""
import numpy as np

from oracle import ov3 as V
from paper_2202_02019_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def case(seed=3):
    s, tb1, tb2 = synth.make_pair(3, 7, 5, 4.0, seed=seed)
    return s, tb1


def test_explicit_matches_factorised():
    s, tb1 = case()
    d = V.density_abic_gs(tb1, s.t2, 0.8)
    We, Wo = V.w_from_abic(d, s.L_vv, s.L_ov)
    Fe, Fo = V.w_ov3_gs(tb1, s.t2, 0.8, s.L_vv, s.L_ov)
    assert rel(Fe, We) < 1e-14 and rel(Fo, Wo) < 1e-14


def test_fd_of_the_ov3_energy():
    s, tb1 = case(5)
    R0 = 1.0
    d = V.density_abic_gs(tb1, s.t2, R0)

    def energy(Lvv, Lov):
        return float(np.einsum("abic,Kab,Kic->", d, Lvv, Lov))

    Wv, Wo = V.w_ov3_gs(tb1, s.t2, R0, s.L_vv, s.L_ov)
    h = 1e-6
    for (K, a, b) in [(0, 1, 2), (3, 6, 0)]:
        Lp = s.L_vv.copy(); Lp[K, a, b] += h
        Lm = s.L_vv.copy(); Lm[K, a, b] -= h
        fd = (energy(Lp, s.L_ov) - energy(Lm, s.L_ov)) / (2 * h)
        assert abs(fd - Wv[K, a, b]) < 1e-7 * max(1.0, abs(fd))
    for (K, i, c) in [(1, 0, 3), (4, 2, 6)]:
        Lp = s.L_ov.copy(); Lp[K, i, c] += h
        Lm = s.L_ov.copy(); Lm[K, i, c] -= h
        fd = (energy(s.L_vv, Lp) - energy(s.L_vv, Lm)) / (2 * h)
        assert abs(fd - Wo[K, i, c]) < 1e-7 * max(1.0, abs(fd))


def test_t_tilde_matrix_is_symmetric_for_pair_symmetric_t2():
    # T~[(i,c),(m,b)] = t~^cb_im equals T~[(m,b),(i,c)] = t~^bc_mi when t_ij^ab = t_ji^ba
    s, _ = case()
    o, v = s.t2.shape[0], s.t2.shape[2]
    tt = V.t_tilde(s.t2)                                 # [i, m, c, b]
    M = tt.transpose(0, 2, 1, 3).reshape(o * v, o * v)   # rows (i,c), cols (m,b)
    assert np.allclose(M, M.T, rtol=0, atol=1e-15)
    assert rel(V.t_tilde(s.t2)[0, 1], 2 * s.t2[0, 1] - s.t2[1, 0]) < 1e-16


def test_es_abci_explicit_matches_factorised_and_fd():
    s, tb1, L2 = V_case_es()
    R1 = np.random.default_rng(8).standard_normal(s.t1.shape)
    d = V.density_abci_es(L2, R1)
    We, Wo = V.w_from_abci(d, s.L_vv, s.L_ov)
    Fe, Fo = V.w_ov3_es_abci(L2, R1, s.L_vv, s.L_ov)
    assert rel(Fe, We) < 1e-14 and rel(Fo, Wo) < 1e-14

    def energy(Lvv, Lov):
        return float(np.einsum("abci,Kab,Kic->", d, Lvv, Lov))

    h = 1e-6
    for (K, a, b) in [(0, 2, 5), (2, 6, 1)]:
        Lp = s.L_vv.copy(); Lp[K, a, b] += h
        Lm = s.L_vv.copy(); Lm[K, a, b] -= h
        fd = (energy(Lp, s.L_ov) - energy(Lm, s.L_ov)) / (2 * h)
        assert abs(fd - Fe[K, a, b]) < 1e-7 * max(1.0, abs(fd))
    for (K, i, c) in [(1, 1, 4), (3, 2, 0)]:
        Lp = s.L_ov.copy(); Lp[K, i, c] += h
        Lm = s.L_ov.copy(); Lm[K, i, c] -= h
        fd = (energy(s.L_vv, Lp) - energy(s.L_vv, Lm)) / (2 * h)
        assert abs(fd - Fo[K, i, c]) < 1e-7 * max(1.0, abs(fd))


def V_case_es():
    # a pair-symmetric L2 (left doubles) from the generator's second system
    s, tb1, tb2 = synth.make_pair(3, 7, 5, 4.0, seed=9)
    return s, tb1, tb2

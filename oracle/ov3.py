"""FP64 oracle for the OV^3 ground-state density contributions to the
three-index intermediates (test infrastructure only, like the rest of
``oracle``).

Ground state, App. A:  d_abci = 0  and  d_abic = L^a_m t~^cb_im R0  with
t~_ij^ab = 2 t_ij^ab - t_ji^ab (Table I) and L^a_m the singles multipliers.
Sec. II.C builds the OV^3 blocks' contributions to W^K_pq = sum_rs d_pqrs
Z^K_rs directly, never storing the density:

    W_ab^K = sum_ic d_abic Z^K_ic = R0 L^a_m Y~^K_bm,   Y~^K_bm = t~^cb_im Z^K_ic   (Table I)
    W_ic^K = sum_ab d_abic Z^K_ab = R0 t~^cb_im O^K_bm,  O^K_bm = L^a_m Z^K_ab

with L^K in place of Z^K, as for the V^4 part (D).  ``density_*`` forms the
OV^3 density; ``w_ov3_*`` is the factorised form.  Pins: the two density
blocks against hand-computed o = 2, v = 2 values (tests/golden/
hand_update_es_ov3.json, built so that a swapped occupied or virtual pair
fails them), the factorised forms against the explicit ones, and central
finite differences of the OV^3 energy term (tests/test_oracle_ov3.py,
tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

__all__ = ["t_tilde", "density_abic_gs", "w_from_abic", "w_ov3_gs", "density_abci_es", "w_from_abci",
           "w_ov3_es_abci"]


def t_tilde(t2):
    """t~_ij^ab = 2 t_ij^ab - t_ji^ab."""
    t2 = np.asarray(t2, dtype=np.float64)
    return 2.0 * t2 - t2.transpose(1, 0, 2, 3)


def density_abic_gs(tbar1, t2, R0):
    """d[a, b, i, c] = R0 sum_m L^a_m t~^cb_im (tbar1[m, a] = L^a_m)."""
    tt = t_tilde(t2)                                    # tt[i, m, c, b] = t~^cb_im
    return R0 * np.einsum("ma,imcb->abic", np.asarray(tbar1, dtype=np.float64), tt)


def w_from_abic(d, L_vv, L_ov):
    """(W_vv[K, a, b], W_ov[K, i, c]) = (sum_ic d_abic L^K_ic, sum_ab d_abic L^K_ab)."""
    return np.einsum("abic,Kic->Kab", d, L_ov), np.einsum("abic,Kab->Kic", d, L_vv)


def w_ov3_gs(tbar1, t2, R0, L_vv, L_ov):
    """The factorised form through Y~ and O (no OV^3 array)."""
    tt = t_tilde(t2)
    Y = np.einsum("imcb,Kic->Kbm", tt, L_ov)           # Y~^K_bm
    W_vv = R0 * np.einsum("ma,Kbm->Kab", tbar1, Y)
    Om = np.einsum("ma,Kab->Kbm", tbar1, L_vv)         # O^K_bm
    W_ov = R0 * np.einsum("imcb,Kbm->Kic", tt, Om)
    return W_vv, W_ov


# --------------------------------------------------------------------------
# excited state, the d_abci block (App. A): d^es_abci = L_ji^ac R_j^b
# --------------------------------------------------------------------------
def density_abci_es(L2, R1):
    """d[a, b, c, i] = sum_j L_ji^ac R_j^b (L2[j, i, a, c] = L_ji^ac, R1[j, b] = R_j^b)."""
    return np.einsum("jiac,jb->abci", np.asarray(L2, dtype=np.float64), np.asarray(R1, dtype=np.float64))


def w_from_abci(d, L_vv, L_ov):
    """(W_vv[K, a, b], W_vo[K, i, c]) = (sum_ci d_abci L^K_ci, sum_ab d_abci L^K_ab), L_ci = L_ov[K, i, c]."""
    return np.einsum("abci,Kic->Kab", d, L_ov), np.einsum("abci,Kab->Kic", d, L_vv)


def w_ov3_es_abci(L2, R1, L_vv, L_ov):
    """The factorised form of Sec. II.C: W_ab^K = R_j^b X^K_aj with X^K_aj = L_ji^ac Z^K_ci, and
    W_ci^K = L_ji^ac P^K_aj with P^K_aj = R_j^b Z^K_ab (Table I), L^K in place of Z^K."""
    L2 = np.asarray(L2, dtype=np.float64)
    X = np.einsum("jiac,Kic->Kaj", L2, L_ov)
    W_vv = np.einsum("jb,Kaj->Kab", R1, X)
    P = np.einsum("jb,Kab->Kaj", R1, L_vv)
    W_vo = np.einsum("jiac,Kaj->Kic", L2, P)
    return W_vv, W_vo

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
           "w_ov3_es_abci", "x_ab", "y_ajbi", "v_ajbi", "ytilde_djak", "density_abic_es", "w_ov3_es_abic"]


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


# --------------------------------------------------------------------------
# excited state, the d_abic block (App. A), eight terms
# --------------------------------------------------------------------------
# Index layouts: L2[i, j, a, b] = L_ij^ab (left doubles), t2[i, j, a, b] = t_ij^ab,
# R2 likewise, R1[i, a] = R_i^a, tbar1[m, a] = L^a_m (left singles).  The
# intermediates of Table I / App. A with C2 = T2:

def x_ab(L2, C2):
    """X_ab(L2, C2) = L_kl^ad C_kl^bd."""
    return np.einsum("klad,klbd->ab", L2, C2)


def y_ajbi(L2, C2):
    """Y_ajbi(L2, C2) = L_jl^ad C_il^bd, as [a, j, b, i]."""
    return np.einsum("jlad,ilbd->ajbi", L2, C2)


def v_ajbi(L2, C2):
    """V_ajbi(L2, C2) = L_kj^ac C_ki^bc, as [a, j, b, i]."""
    return np.einsum("kjac,kibc->ajbi", L2, C2)


def ytilde_djak(L2, t2):
    """Y~_djak(L2, T2) = L_mj^ed t~_mk^ea, as [d, j, a, k]."""
    return np.einsum("mjed,mkea->djak", L2, t_tilde(t2))


def density_abic_es(tbar1, L2, t2, R0, R1, R2):
    """d^es_abic of App. A as printed, [a, b, i, c]:

        L^a_m t~^cb_im R0 + L^a_m (2 R~^bc_mi - R~^cb_mi) + 2 X_ab R^c_i
        - (V_akbi + Y_akbi) R^c_k + L^ad_mk t~^bc_mi R^d_k - L^ad_mn t^bc_mn R^d_i
        + Y~_akci R^b_k - X_ac R^b_i

    with X, Y, V, Y~ of (L2, T2) and R~ built from R2 as t~ from T2 (Table I's
    caption: C~_ij^ab = 2 C_ij^ab - C_ji^ab)."""
    tbar1 = np.asarray(tbar1, dtype=np.float64)
    L2 = np.asarray(L2, dtype=np.float64)
    t2 = np.asarray(t2, dtype=np.float64)
    R1 = np.asarray(R1, dtype=np.float64)
    tt, Rt = t_tilde(t2), t_tilde(R2)
    X = x_ab(L2, t2)
    VY = v_ajbi(L2, t2) + y_ajbi(L2, t2)                     # [a, k, b, i]
    Yt = ytilde_djak(L2, t2)                                 # [a, k, c, i] read as Y~_akci
    d = R0 * np.einsum("ma,imcb->abic", tbar1, tt)                                   # L^a_m t~^cb_im R0
    d += np.einsum("ma,mibc->abic", tbar1, 2.0 * Rt) - np.einsum("ma,micb->abic", tbar1, Rt)
    d += 2.0 * np.einsum("ab,ic->abic", X, R1)                                       # 2 X_ab R^c_i
    d -= np.einsum("akbi,kc->abic", VY, R1)                                          # -(V + Y)_akbi R^c_k
    d += np.einsum("mkad,mibc,kd->abic", L2, tt, R1)                                 # L^ad_mk t~^bc_mi R^d_k
    d -= np.einsum("mnad,mnbc,id->abic", L2, t2, R1)                                 # -L^ad_mn t^bc_mn R^d_i
    d += np.einsum("akci,kb->abic", Yt, R1)                                          # Y~_akci R^b_k
    d -= np.einsum("ac,ib->abic", X, R1)                                             # -X_ac R^b_i
    return d


def w_ov3_es_abic(tbar1, L2, t2, R0, R1, R2, L_vv, L_ov):
    """(W_vv[K, a, b], W_ov[K, i, c]) = (sum_ic d_abic L^K_ic, sum_ab d_abic L^K_ab) for d^es_abic,
    term by term through three-index intermediates, never the OV^3 array (Sec. II.C), with L^K in
    place of Z^K.  The pair matrix of the first two terms is P^cb_im = R0 t~^cb_im + 2 R~^bc_mi -
    R~^cb_mi; the others go through X, V + Y, Y~, W_am = L^ad_mk R^d_k and B_iamn = L^ad_mn R^d_i."""
    tbar1 = np.asarray(tbar1, dtype=np.float64)
    L2 = np.asarray(L2, dtype=np.float64)
    t2 = np.asarray(t2, dtype=np.float64)
    R1 = np.asarray(R1, dtype=np.float64)
    tt, Rt = t_tilde(t2), t_tilde(R2)
    P = R0 * tt + 2.0 * Rt.transpose(1, 0, 3, 2) - Rt.transpose(1, 0, 2, 3)   # P[i, m, c, b] = P^cb_im
    X = x_ab(L2, t2)
    VY = v_ajbi(L2, t2) + y_ajbi(L2, t2)
    Yt = ytilde_djak(L2, t2)
    Wam = np.einsum("mkad,kd->am", L2, R1)
    B = np.einsum("mnad,id->iamn", L2, R1)
    # terms 1-2: L^a_m P^cb_im
    W_vv = np.einsum("ma,Kbm->Kab", tbar1, np.einsum("imcb,Kic->Kbm", P, L_ov))
    W_ov = np.einsum("imcb,Kbm->Kic", P, np.einsum("ma,Kab->Kbm", tbar1, L_vv))
    # term 3: 2 X_ab R^c_i
    W_vv += 2.0 * np.einsum("ab,K->Kab", X, np.einsum("ic,Kic->K", R1, L_ov))
    W_ov += 2.0 * np.einsum("ic,K->Kic", R1, np.einsum("ab,Kab->K", X, L_vv))
    # term 4: -(V + Y)_akbi R^c_k
    W_vv -= np.einsum("akbi,Kik->Kab", VY, np.einsum("kc,Kic->Kik", R1, L_ov))
    W_ov -= np.einsum("kc,Kik->Kic", R1, np.einsum("akbi,Kab->Kik", VY, L_vv))
    # term 5: W_am t~^bc_mi
    W_vv += np.einsum("am,Kbm->Kab", Wam, np.einsum("mibc,Kic->Kbm", tt, L_ov))
    W_ov += np.einsum("mibc,Kbm->Kic", tt, np.einsum("am,Kab->Kbm", Wam, L_vv))
    # term 6: -B_iamn t^bc_mn
    W_vv -= np.einsum("iamn,Kbimn->Kab", B, np.einsum("mnbc,Kic->Kbimn", t2, L_ov))
    W_ov -= np.einsum("iamn,mnbc,Kab->Kic", B, t2, L_vv)
    # term 7: Y~_akci R^b_k
    W_vv += np.einsum("kb,Kak->Kab", R1, np.einsum("akci,Kic->Kak", Yt, L_ov))
    W_ov += np.einsum("akci,Kak->Kic", Yt, np.einsum("kb,Kab->Kak", R1, L_vv))
    # term 8: -X_ac R^b_i
    W_vv -= np.einsum("ib,Kai->Kab", R1, np.einsum("ac,Kic->Kai", X, L_ov))
    W_ov -= np.einsum("ac,Kai->Kic", X, np.einsum("ib,Kab->Kai", R1, L_vv))
    return W_vv, W_ov

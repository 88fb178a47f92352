"""FP64 oracle for the T1-transformed form of the ladder and for the excited-state
V^4 density (test infrastructure only, like the rest of ``oracle``).

T1-transformed basis, Sec. II.C of arXiv:2202.02019: with the singles matrix
T1 over all n = o + v orbitals (T1[o + a, i] = t_i^a, the only non-zero
block is virtual row / occupied column),

    x = I - T1,   y = I + T1^T,
    h_pq = sum_rs x_pr y_qs h^MO_rs,
    g_pqrs = sum_tumn x_pt y_qu x_rm y_sn g^MO_tumn,
    L^J_pq = sum_rs x_pr y_qs (L^J_rs)^MO,

and the three-index density intermediate goes back to the MO basis as

    (W^J_pq)^MO = sum_rs x_rp y_sq W^J_rs.

In that basis the ladder uses t2 itself (no t1 t1 term: the singles live in
the integrals) and the densities do not depend on T1.

Excited-state V^4 density, App. A: d^es_abcd = O^(2)_abcd(L2, U) with
U = T2 R0 + R2, where O^(2)_abcd(L2, C2) is the same contraction as the
ground-state density with C2 = U in place of tau.

Everything below is the plain definition over the full n x n matrices, for
small sizes; the CUDA path uses only the blocks that contribute.
"""
from __future__ import annotations

import numpy as np

__all__ = ["t1_matrices", "t1_transform_full", "t1_transform_vv", "g_t1_full",
           "w_backtransform_full", "es_amplitudes"]


def t1_matrices(t1):
    """x = I - T1 and y = I + T1^T for singles t1[i, a] = t_i^a (Sec. II.C)."""
    t1 = np.asarray(t1, dtype=np.float64)
    o, v = t1.shape
    n = o + v
    T = np.zeros((n, n))
    T[o:, :o] = t1.T          # T[o + a, i] = t_i^a
    eye = np.eye(n)
    return eye - T, eye + T.T


def t1_transform_full(L_full, t1):
    """L^J -> x L^J y^T for every J: L_full[J, p, q] over all n orbitals."""
    x, y = t1_matrices(t1)
    L_full = np.asarray(L_full, dtype=np.float64)
    return np.einsum("pr,Jrs,qs->Jpq", x, L_full, y)


def t1_transform_vv(L_full, t1):
    """The virtual-virtual block of the T1-transformed Cholesky vectors."""
    o = np.asarray(t1).shape[0]
    return np.ascontiguousarray(t1_transform_full(L_full, t1)[:, o:, o:])


def g_t1_full(g_mo, t1):
    """g_pqrs = sum x_pt y_qu x_rm y_sn g^MO_tumn, the four-index transform."""
    x, y = t1_matrices(t1)
    return np.einsum("pt,qu,rm,sn,tumn->pqrs", x, y, x, y, np.asarray(g_mo, dtype=np.float64))


def w_backtransform_full(W_full, t1):
    """(W^J)^MO = x^T W^J y for every J (the back-transformation of Sec. II.C)."""
    x, y = t1_matrices(t1)
    return np.einsum("rp,Jrs,sq->Jpq", x, np.asarray(W_full, dtype=np.float64), y)


def es_amplitudes(t2, r2, r0):
    """U = T2 R0 + R2, the doubles that pair with L2 in the excited-state V^4
    density (App. A).  Pinned through that density by a hand-computed o = 1,
    v = 2 case with R0 = 2 (tests/golden/hand_update_es_ov3.json)."""
    return float(r0) * np.asarray(t2, dtype=np.float64) + np.asarray(r2, dtype=np.float64)

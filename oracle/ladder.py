"""Plain FP64 NumPy oracle for the CD-CCSD vvvv ladder and its V^4 density.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke`` and the CPU
baseline of ``bench.py`` use it.  Nothing here is shared with, or imported by,
the CUDA library.

Definitions (arXiv:2202.02019, closed shell, Mulliken notation):

* Cholesky integrals, Sec. II.A (Cholesky expansion of (pq|rs)):
      g_acbd = (ac|bd) = sum_J L^J_ac L^J_bd
* amplitudes entering the ladder:  tau_ij^cd = t_ij^cd + t_i^c t_j^d
* ladder ("A2") residual term, Sec. II.B (Scuseria's A2 term of Omega):
      Omega_ij^ab = sum_cd g_acbd tau_ij^cd
* V^4 density, Eq. (v4density) / App. A (O^(2)_abcd(L2, C2) with L2 = tbar2
  and C2 = tau; index map: the paper's (a,c | b,d) pairing is (a,b | c,d) here):
      Gamma_abcd = sum_ij tbar_ij^ab tau_ij^cd
* its three-index contraction, the V^4 part of W^J_pq built with L in place
  of Z (the W-tilde intermediate of Sec. II.C):
      D^J_ac = sum_bd Gamma_abcd L^J_bd
  D carries no factor 2; Eq. (integral_contraction) puts the 2 in front, so
  dE/dL = 2 D for pair-symmetric tbar and tau.
* ladder slice of the Lagrangian, Eq. (lagrangian) (the zeta-bar . Omega
  term):  E = sum_ijab tbar_ij^ab Omega_ij^ab

Three independent formulations are provided: dense explicit-V^4 einsums
(``*_dense``), row-blocked matmuls over the first virtual index that never
form V^4 (``*_rows``), and the paper's symmetric/antisymmetric packed
algorithm (``*_pm``, Sec. II.B: X^pm = X_ij +- X_ji, restricted loops
i>=j, a>=b, c>=d, net four-fold saving).

Pins (tests/test_oracle.py): brute force vs rows vs packed, pair
symmetries, the Euler identity sum L.D = E, central finite differences of E
(dE/dL = 2D, dE/dtau = transposed ladder), closed forms for nj = 1, one-hot
L, t1 = 0 and o = 1, homogeneity in L, and a hand-computed example under
tests/golden/.  ``update_t2`` is pinned by hand values and by one step of
``oracle.iterate.jacobi`` (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tau", "g_vvvv", "residual_dense", "residual_rows", "residual_pm",
    "gamma_dense", "density_dense", "density_rows", "density_pm",
    "dE_dL_general", "dE_dtau", "gamma_pm", "lagrangian", "euler_lagrangian", "update_t2",
    "sampled_rows",
]


def tau(t1, t2):
    """tau_ij^cd = t_ij^cd + t_i^c t_j^d (t1 None: tau = t2)."""
    t2 = np.asarray(t2, dtype=np.float64)
    if t1 is None:
        return t2.copy()
    return t2 + np.einsum("ic,jd->ijcd", t1, t1)


# --------------------------------------------------------------------------
# dense (explicit V^4) formulation: small sizes only
# --------------------------------------------------------------------------
def g_vvvv(L_vv):
    """g_acbd = sum_J L^J_ac L^J_bd, returned as [a, c, b, d] (Sec. II.A)."""
    return np.einsum("Jac,Jbd->acbd", L_vv, L_vv)


def residual_dense(L_vv, tau_):
    """Omega_ij^ab = sum_cd g_acbd tau_ij^cd, explicit V^4 (Sec. II.B)."""
    return np.einsum("acbd,ijcd->ijab", g_vvvv(L_vv), tau_)


def gamma_dense(tbar2, tau_):
    """Gamma_abcd = sum_ij tbar_ij^ab tau_ij^cd (Eq. v4density)."""
    return np.einsum("ijab,ijcd->abcd", tbar2, tau_)


def density_dense(L_vv, tbar2, tau_):
    """D^J_ac = sum_bd Gamma_abcd L^J_bd (W-tilde, Sec. II.C)."""
    return np.einsum("abcd,Jbd->Jac", gamma_dense(tbar2, tau_), L_vv)


def dE_dL_general(L_vv, tbar2, tau_):
    """dE/dL^J_xy without assuming pair symmetry:
    sum_bd Gamma_xbyd L^J_bd + sum_ac Gamma_axcy L^J_ac."""
    G = gamma_dense(tbar2, tau_)
    return (np.einsum("xbyd,Jbd->Jxy", G, L_vv)
            + np.einsum("axcy,Jac->Jxy", G, L_vv))


def dE_dtau(L_vv, tbar2):
    """dE/dtau_ij^cd = sum_ab tbar_ij^ab g_acbd."""
    return np.einsum("ijab,acbd->ijcd", tbar2, g_vvvv(L_vv))


# --------------------------------------------------------------------------
# row-blocked formulation: one virtual row a at a time, no V^4 array
# --------------------------------------------------------------------------
def residual_rows(L_vv, tau_, rows=None, cols=None):
    """Omega[:, :, a, b] for a in ``rows`` and b in ``cols`` (all if None).

    For a fixed a:  G^a[c, (b,d)] = sum_J L^J_ac L^J_bd  (a v x v^2 block of
    g, never the whole V^4), then Omega_ij^ab = sum_{c,d} G^a[c,b,d] tau_ij^cd.
    """
    nj, v, _ = L_vv.shape
    o = tau_.shape[0]
    rows = range(v) if rows is None else rows
    cols = np.arange(v) if cols is None else np.asarray(cols)
    nb = len(cols)
    Lb = L_vv[:, cols, :].reshape(nj, nb * v)
    T = tau_.reshape(o * o, v * v)
    out = np.empty((o, o, len(rows), nb))
    for k, a in enumerate(rows):
        Ga = (L_vv[:, a, :].T @ Lb).reshape(v, nb, v)         # [c, b, d]
        Gb = Ga.transpose(1, 0, 2).reshape(nb, v * v)          # [b, (c,d)]
        out[:, :, k, :] = (Gb @ T.T).T.reshape(o, o, nb)
    return out


def density_rows(L_vv, tbar2, tau_, rows=None, cols=None):
    """D[:, a, c] for a in ``rows`` and c in ``cols`` (all if None).

    For a fixed a:  Gamma^a[b, (c,d)] = sum_ij tbar_ij^ab tau_ij^cd, then
    D^J_ac = sum_{b,d} Gamma^a[b,c,d] L^J_bd.
    """
    nj, v, _ = L_vv.shape
    o = tau_.shape[0]
    rows = range(v) if rows is None else rows
    cols = np.arange(v) if cols is None else np.asarray(cols)
    nc = len(cols)
    Lf = L_vv.reshape(nj, v * v)
    Tc = tau_[:, :, cols, :].reshape(o * o, nc * v)
    out = np.empty((nj, len(rows), nc))
    for k, a in enumerate(rows):
        Ta = tbar2[:, :, a, :].reshape(o * o, v)              # [(ij), b]
        Ga = (Ta.T @ Tc).reshape(v, nc, v)                     # [b, c, d]
        Gc = Ga.transpose(1, 0, 2).reshape(nc, v * v)          # [c, (b,d)]
        out[:, k, :] = (Gc @ Lf.T).T
    return out


def sampled_rows(L_vv, t1, t2, tbar2, rows, cols=None):
    """(Omega[:, :, rows, cols], D[:, rows, cols]) for lists of virtual indices."""
    tt = tau(t1, t2)
    return residual_rows(L_vv, tt, rows, cols), density_rows(L_vv, tbar2, tt, rows, cols)


# --------------------------------------------------------------------------
# symmetric / antisymmetric packed formulation (Sec. II.B)
# --------------------------------------------------------------------------
def _pm(X):
    """X^+- _ij = X_ij +- X_ji over the two leading (occupied) indices."""
    Xt = X.transpose(1, 0, 2, 3)
    return X + Xt, X - Xt


def _expand(X, n1, n2, s1, s2):
    """Packed X[(p<=q or p<q), (r<=s or r<s)] -> full F[p, q, r, s] using
    F[q,p,.,.] = s1 F[p,q,.,.] and F[.,.,s,r] = s2 F[.,.,r,s]
    (s = +1: symmetric, pairs with p<=q; s = -1: antisymmetric, p<q)."""
    p, q = np.triu_indices(n1, 0 if s1 > 0 else 1)
    r, s = np.triu_indices(n2, 0 if s2 > 0 else 1)
    inner = np.zeros((len(p), n2, n2))
    inner[:, r, s] = X
    inner[:, s, r] = s2 * X
    F = np.zeros((n1, n1, n2, n2))
    F[p, q] = inner
    F[q, p] = s1 * inner
    return F


def residual_pm(L_vv, tau_):
    """Packed ladder (Sec. II.B).  With X^pm_ij = X_ij +- X_ji:

        Omega^+[ab, ij] = sum_{c<=d} g+[ab, cd] tau+_ij^cd     (a<=b, i<=j)
        Omega^-[ab, ij] = sum_{c<d}  g-[ab, cd] tau-_ij^cd     (a<b,  i<j)
        g+[ab, cd] = (g_acbd + g_adbc) (1/2 if c = d),  g- = g_acbd - g_adbc

    Omega^pm_ij^ab = Omega_ij^ab +- Omega_ji^ab; Omega^+ is symmetric and
    Omega^- antisymmetric under a<->b and under i<->j, and
    Omega = (Omega^+ + Omega^-)/2.  Requires tau_ij^cd = tau_ji^dc."""
    o = tau_.shape[0]
    v = L_vv.shape[1]
    Gab = g_vvvv(L_vv).transpose(0, 2, 1, 3)      # G^{ab}_{cd} = g_acbd
    tp, tm = _pm(tau_)                            # [i, j, c, d]
    au, bu = np.triu_indices(v, 0)
    iu, ju = np.triu_indices(o, 0)
    gp = Gab[au, bu][:, au, bu] + Gab[au, bu][:, bu, au]          # [ab, cd]
    gp[:, au == bu] *= 0.5
    Op = gp @ tp[iu, ju][:, au, bu].T                              # [ab, ij]
    as_, bs = np.triu_indices(v, 1)
    is_, js = np.triu_indices(o, 1)
    gm = Gab[as_, bs][:, as_, bs] - Gab[as_, bs][:, bs, as_]
    Om = gm @ tm[is_, js][:, as_, bs].T
    full = 0.5 * (_expand(Op, v, o, +1, +1) + _expand(Om, v, o, -1, -1))
    return full.transpose(2, 3, 0, 1).copy()      # [a,b,i,j] -> [i,j,a,b]


def gamma_pm(tbar2, tau_):
    """Packed Gamma (Eq. v4density with the A2 trick of Sec. II.B):
    Gamma_abcd = (Gamma+ + Gamma-)/4 with
    Gamma+[ab,cd] = sum_{i<=j} w_ij tbar+_ij^ab tau+_ij^cd  (w_ii=1, w_i<j=2)
    Gamma-[ab,cd] = sum_{i<j} 2 tbar-_ij^ab tau-_ij^cd,
    X^pm_ij = X_ij +- X_ji.  Returns the full [a, b, c, d] array."""
    o, _, v, _ = tau_.shape
    bp, bm = _pm(tbar2)
    tp, tm = _pm(tau_)
    au, bu = np.triu_indices(v, 0)
    as_, bs = np.triu_indices(v, 1)
    iu, ju = np.triu_indices(o, 0)
    is_, js = np.triu_indices(o, 1)
    w = np.where(iu == ju, 1.0, 2.0)
    Gp = (bp[iu, ju][:, au, bu] * w[:, None]).T @ tp[iu, ju][:, au, bu]
    Gm = (2.0 * bm[is_, js][:, as_, bs]).T @ tm[is_, js][:, as_, bs]
    return 0.25 * (_expand(Gp, v, v, +1, +1) + _expand(Gm, v, v, -1, -1))


def density_pm(L_vv, tbar2, tau_):
    """D^J_ac = sum_bd Gamma_abcd L^J_bd with Gamma from the packed form."""
    return np.einsum("abcd,Jbd->Jac", gamma_pm(tbar2, tau_), L_vv)


# --------------------------------------------------------------------------
# reductions and the amplitude step
# --------------------------------------------------------------------------
def lagrangian(tbar2, omega):
    """E = sum_ijab tbar_ij^ab Omega_ij^ab (plain sum, no spin factors)."""
    return float(np.sum(np.asarray(tbar2, np.float64) * np.asarray(omega, np.float64)))


def euler_lagrangian(L_vv, D):
    """sum_J,ac L^J_ac D^J_ac; equals E because E is quadratic in L."""
    return float(np.sum(L_vv * D))


def update_t2(t2, omega, eps, o):
    """t'_ij^ab = t_ij^ab + Omega_ij^ab / (eps_i + eps_j - eps_a - eps_b)."""
    eo, ev = eps[:o], eps[o:]
    den = (eo[:, None, None, None] + eo[None, :, None, None]
           - ev[None, None, :, None] - ev[None, None, None, :])
    return t2 + omega / den

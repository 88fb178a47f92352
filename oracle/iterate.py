"""FP64 oracle for a doubles amplitude iteration driven by the ladder (test
infrastructure only, like the rest of ``oracle``).

The CC amplitude equations Omega_mu = <mu| exp(-T) H exp(T) |HF> = 0
(Sec. II.A) are solved by the usual quasi-Newton (Jacobi) step with the
orbital-energy denominators; the paper leaves the solver to its CC program.
The model kept here is the part of the doubles equations that the ladder
path owns, with the MP2-like driver term that starts it:

    g_aibj      = sum_J L^J_ai L^J_bj                       (Cholesky integrals, Sec. II.A)
    Omega_ij^ab = g_aibj + sum_cd g_acbd tau_ij^cd - Delta_ijab t_ij^ab
    Delta_ijab  = eps_i + eps_j - eps_a - eps_b              (eps_a + eps_b - eps_i - eps_j is the
                                                              diagonal Fock part of Omega)
    t' = t + Omega / Delta = (g_aibj + sum_cd g_acbd tau_ij^cd) / Delta,

with tau = t2 + t1 (x) t1 for fixed singles t1.  At t = 0 and no ladder the
step gives the MP2 guess.  The fixed point solves, for every occupied pair
(i, j), the linear system (Delta_ij - G) t_ij = g_ij + G (t1_i (x) t1_j) with
G[(a,b),(c,d)] = g_acbd; ``fixed_point`` solves it directly.
"""
from __future__ import annotations

import numpy as np

from .ladder import residual_dense, tau, g_vvvv

__all__ = ["mp2_driver", "denominators", "jacobi", "fixed_point"]


def mp2_driver(L_ov):
    """g[i, j, a, b] = g_aibj = sum_J L^J_ia L^J_jb (L^J symmetric: L_ai = L_ia)."""
    L_ov = np.asarray(L_ov, dtype=np.float64)
    return np.einsum("Jia,Jjb->ijab", L_ov, L_ov)


def denominators(eps, o):
    eps = np.asarray(eps, dtype=np.float64)
    e_o, e_v = eps[:o], eps[o:]
    return e_o[:, None, None, None] + e_o[None, :, None, None] - e_v[None, None, :, None] - e_v[None, None, None, :]


def jacobi(L_vv, t1, t2, g, eps, n_iter):
    """n_iter Jacobi steps; returns the amplitudes and sum (t' - t)^2 per step."""
    t = np.asarray(t2, dtype=np.float64).copy()
    o = t.shape[0]
    D = denominators(eps, o)
    dn = []
    for _ in range(n_iter):
        tn = (g + residual_dense(L_vv, tau(t1, t))) / D
        dn.append(float(np.sum((tn - t) ** 2)))
        t = tn
    return t, np.array(dn)


def fixed_point(L_vv, t1, g, eps):
    """Direct solution of the fixed point, one (v^2 x v^2) system per (i, j)."""
    g = np.asarray(g, dtype=np.float64)
    o, _, v, _ = g.shape
    D = denominators(eps, o)
    G = g_vvvv(L_vv).transpose(0, 2, 1, 3).reshape(v * v, v * v)   # G[(a,b),(c,d)] = g_acbd
    t = np.empty_like(g)
    for i in range(o):
        for j in range(o):
            rhs = g[i, j].reshape(-1)
            if t1 is not None:
                rhs = rhs + G @ np.outer(t1[i], t1[j]).reshape(-1)
            t[i, j] = np.linalg.solve(np.diag(D[i, j].reshape(-1)) - G, rhs).reshape(v, v)
    return t

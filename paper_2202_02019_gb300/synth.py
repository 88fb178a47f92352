"""Seeded synthetic closed-shell systems for the CD-CCSD vvvv ladder.

This module is shared by the FP64 oracle tests and the CUDA path.  It holds
only input generation (random draws and the MP2 amplitude guess that shapes
t2); none of the ladder / density arithmetic lives here.

Recipe (one system, one seed; numpy PCG64 via ``default_rng``), in draw order:

1. occupied orbital energies  eps_i ~ U[-2, -0.3], i < o
2. virtual orbital energies   eps_a ~ U[0.1, 5],   a < v
3. for J = 0 .. nj-1: the upper triangle (p <= q, row-major, ``triu_indices``)
   of an (o+v) x (o+v) matrix drawn N(0, 1), mirrored to a symmetric matrix
   and scaled by sqrt(lambda_J), lambda_J = exp(-J / lam_scale)
   (the Cholesky vectors L^J_pq of the paper's Section II.A, occupied first)
4. t1 ~ N(0, 0.01) (0.01 is the standard deviation), shape [o, v]
5. t2 = MP2 guess  t_ij^ab = g_aibj / (eps_i + eps_j - eps_a - eps_b),
   g_aibj = sum_J L^J_ai L^J_bj, then symmetrised exactly under
   (i,a) <-> (j,b) so that t_ij^ab == t_ji^ba holds bit for bit.

The multipliers tbar1, tbar2 are t1, t2 of the same recipe run with
``seed + 1`` (its own eps' and L'), so tbar2 != t2.

Layouts (all C-contiguous float64):
  L_vv  [nj, v, v]     L^J_ac  at (J*v + a)*v + c
  t1    [o, v]         t_i^a
  t2    [o, o, v, v]   t_ij^ab at ((i*o + j)*v + a)*v + b
  eps   [o + v]        occupied first

``make_system_torch`` follows the same recipe with torch's device generator
(different random stream, same distributions and structure) for sizes where
host generation would dominate a run; its MP2 contraction runs in float32,
which only changes which synthetic t2 is drawn, not its structure.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["System", "CONFIGS", "make_system", "make_pair", "batch_sizes",
           "make_system_torch", "make_pair_torch"]


@dataclass
class System:
    o: int
    v: int
    nj: int
    L_vv: np.ndarray          # [nj, v, v]
    L_ov: np.ndarray          # [nj, o, v]   L^J_ia (occupied row, virtual column)
    eps: np.ndarray           # [o + v]
    t1: np.ndarray            # [o, v]
    t2: np.ndarray            # [o, o, v, v]


# Named workloads (o, v, nj, lam_scale).  lam_scale sets lambda_J = exp(-J/lam_scale).
CONFIGS = {
    "tiny": (4, 20, 60, 12.0),          # explicit-V^4 brute-force size
    "small": (24, 180, 900, 150.0),     # single-system FP64 baseline size
    "fd": (8, 48, 160, 160 / 6.0),      # finite-difference check size
    "grad": (30, 250, 1200, 200.0),     # autograd timing size
    "retinal": (78, 650, 4000, 700.0),  # retinal-scale single system
}


def _sym_pairs(t2: np.ndarray) -> np.ndarray:
    """Exact (i,a)<->(j,b) symmetrisation: t_ij^ab = t_ji^ba bit for bit."""
    return 0.5 * (t2 + t2.transpose(1, 0, 3, 2))


def make_system(o: int, v: int, nj: int, lam_scale: float, seed: int) -> System:
    if min(o, v, nj) < 1:
        raise ValueError("o, v, nj must be >= 1")
    rng = np.random.default_rng(seed)
    n = o + v
    eps_o = rng.uniform(-2.0, -0.3, o)
    eps_v = rng.uniform(0.1, 5.0, v)
    iu = np.triu_indices(n)
    L = np.empty((nj, n, n))
    for J in range(nj):
        m = np.zeros((n, n))
        m[iu] = rng.standard_normal(iu[0].size)
        m = m + np.triu(m, 1).T
        L[J] = m * math.sqrt(math.exp(-J / lam_scale))
    t1 = rng.normal(0.0, 0.01, (o, v))
    L_ov = np.ascontiguousarray(L[:, :o, o:])            # L^J_ia
    L_vv = np.ascontiguousarray(L[:, o:, o:])            # L^J_ac
    # g_aibj = sum_J L^J_ai L^J_bj (L symmetric: L^J_ai = L^J_ia)
    X = L_ov.reshape(nj, o * v)
    g = (X.T @ X).reshape(o, v, o, v)                    # [i, a, j, b]
    den = (eps_o[:, None, None, None] + eps_o[None, None, :, None]
           - eps_v[None, :, None, None] - eps_v[None, None, None, :])
    t2 = (g / den).transpose(0, 2, 1, 3)                 # [i, j, a, b]
    t2 = np.ascontiguousarray(_sym_pairs(t2))
    eps = np.concatenate([eps_o, eps_v])
    return System(o, v, nj, L_vv, L_ov, eps, t1, t2)


def make_pair(o: int, v: int, nj: int, lam_scale: float, seed: int = 2202):
    """(system, tbar1, tbar2): the system from ``seed``, multipliers from ``seed+1``."""
    s = make_system(o, v, nj, lam_scale, seed)
    m = make_system(o, v, nj, lam_scale, seed + 1)
    return s, m.t1, m.t2


def batch_sizes(n_sys: int = 24, seed: int = 2202):
    """Uneven batch: o ~ U{6..40}, v ~ U{50..300}, nj = 5 v (one seed)."""
    rng = np.random.default_rng(seed)
    o = rng.integers(6, 41, n_sys)
    v = rng.integers(50, 301, n_sys)
    return [(int(a), int(b), int(5 * b)) for a, b in zip(o, v)]


# ----------------------------------------------------------------------------
# Device-side generator (torch), same recipe, for the retinal-scale workload.
# ----------------------------------------------------------------------------
def make_system_torch(o: int, v: int, nj: int, lam_scale: float, seed: int,
                      device="cuda", chunk: int = 256):
    """Same recipe as ``make_system`` drawn with torch's generator on ``device``.

    Returns a dict of float64 device tensors: L_vv, eps, t1, t2.  Only the vv
    and ov blocks of each symmetric L^J are formed (the oo block is never
    needed), drawn as full N(0,1) blocks and symmetrised: L^J_ac = L^J_ca.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64
    eps_o = torch.rand(o, generator=g, device=device, dtype=f64) * 1.7 - 2.0
    eps_v = torch.rand(v, generator=g, device=device, dtype=f64) * 4.9 + 0.1
    L_vv = torch.empty(nj, v, v, device=device, dtype=f64)
    L_ov = torch.empty(nj, o, v, device=device, dtype=torch.float32)
    for j0 in range(0, nj, chunk):
        j1 = min(nj, j0 + chunk)
        sc = torch.exp(-torch.arange(j0, j1, device=device, dtype=f64) / lam_scale).sqrt()
        m = torch.randn(j1 - j0, v, v, generator=g, device=device, dtype=f64)
        m = torch.triu(m) + torch.triu(m, 1).transpose(1, 2)
        L_vv[j0:j1] = m * sc[:, None, None]
        w = torch.randn(j1 - j0, o, v, generator=g, device=device, dtype=f64)
        L_ov[j0:j1] = (w * sc[:, None, None]).float()
    t1 = torch.randn(o, v, generator=g, device=device, dtype=f64) * 0.01
    X = L_ov.reshape(nj, o * v)
    gm = (X.t() @ X).double().reshape(o, v, o, v)         # g_aibj at [i, a, j, b]
    del X, L_ov
    den = (eps_o[:, None, None, None] + eps_o[None, None, :, None]
           - eps_v[None, :, None, None] - eps_v[None, None, None, :])
    gm.div_(den)
    t2 = gm.permute(0, 2, 1, 3).contiguous()
    del gm, den
    t2 = 0.5 * (t2 + t2.permute(1, 0, 3, 2))
    t2 = t2.contiguous()
    eps = torch.cat([eps_o, eps_v])
    return {"o": o, "v": v, "nj": nj, "L_vv": L_vv, "eps": eps, "t1": t1, "t2": t2}


def make_pair_torch(o, v, nj, lam_scale, seed=2202, device="cuda"):
    s = make_system_torch(o, v, nj, lam_scale, seed, device)
    m = make_system_torch(o, v, nj, lam_scale, seed + 1, device)
    s["tbar1"] = m["t1"]
    s["tbar2"] = m["t2"]
    del m
    return s

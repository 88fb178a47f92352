"""How close the split-BF16 operand format itself comes to the oracle (CPU).

The mixed path stores every operand as three BF16 pieces and forms each
useful product from the six piece products of weight >= 2^-16.  This test
emulates exactly that with exact (FP64) sums through the residual's two
contractions -- the g-build and the ladder, with g re-split into pieces
between them as the GPU path does -- on the finite-difference case and a
larger one.  It shows what the format alone allows: Omega to ~1e-8 and the
Lagrangian E = sum tbar.Omega to well below 1e-9.  The GPU path's E errors
(3-6e-7 on these cases) are therefore not the format's: they come from the
tensor core's FP32 accumulation, which truncates (a toward-zero bias of about
2^-25 of the running sum per 16-term step).  The emulation is written from
the method's description, with its own BF16 rounding; it shares nothing with
the CUDA code.
"""
import numpy as np
import pytest

import oracle as O
from paper_2202_02019_gb300 import synth


def bf16_rn(x):
    # round to the nearest BF16 (8 significant bits), ties to even, via the FP32 bit pattern;
    # the inputs here are far from FP32 over/underflow, so FP32 conversion first is exact enough
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def split3(x):
    p0 = bf16_rn(x)
    r = x - p0
    p1 = bf16_rn(r)
    return p0, p1, bf16_rn(r - p1)


def mm6(A, B):
    """sum_k A[m, k] B[n, k] from the six piece products of weight >= 2^-16, summed exactly."""
    a, b = split3(A), split3(B)
    return sum(a[i] @ b[j].T for i, j in [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)])


def emulated_residual(L, tau):
    nj, v, _ = L.shape
    o = tau.shape[0]
    LT = L.reshape(nj, v * v).T                              # [(a,c)][J]
    g = mm6(LT, LT).reshape(v, v, v, v)                      # g_acbd at [a, c, b, d]
    Gab = g.transpose(0, 2, 1, 3).reshape(v * v, v * v)      # [(a,b)][(c,d)]
    return mm6(Gab, tau.reshape(o * o, v * v)).T.reshape(o, o, v, v)


@pytest.mark.parametrize("shape", [(8, 48, 160, 160 / 6.0), (3, 7, 5, 4.0), (12, 90, 400, 70.0)])
def test_split_bf16_format_alone_reaches_the_lagrangian_target(shape):
    o, v, nj, lam = shape
    s, tb1, tb2 = synth.make_pair(o, v, nj, lam, seed=2202)
    tt = O.tau(s.t1, s.t2)
    ref = O.residual_rows(s.L_vv, tt)
    E_ref = O.lagrangian(tb2, ref)
    om = emulated_residual(s.L_vv, tt)
    e_om = np.linalg.norm(om - ref) / np.linalg.norm(ref)
    e_E = abs(O.lagrangian(tb2, om) - E_ref) / abs(E_ref)
    print(f"{shape}: Omega {e_om:.2e}  E {e_E:.2e}")
    assert e_om < 2e-8
    assert e_E < 1e-9

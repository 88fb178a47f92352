"""GPU parity of the T1-transformed form (Sec. II.C) against the FP64 oracle.

The two small FP64 kernels (forward transform of the Cholesky vectors, back
transform of the density intermediate) are checked element-wise on shapes
that span several tiles and ragged tails in every dimension, and the whole
T1-form pass (transform, ladder with t2, density, back transform) is checked
against the oracle's full-matrix definition.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import t1 as T
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 1e-6, "fp16x2": 1e-6}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def full_L(o, v, nj, seed):
    # MO Cholesky vectors over all orbitals, not symmetric, t1 ~ N(0, 0.1)
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((nj, o + v, o + v))
    t1 = 0.1 * rng.standard_normal((o, v))
    return L, t1


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("o,v,nj", [(3, 7, 5), (5, 37, 70), (33, 70, 3), (1, 130, 2)])
def test_t1_transform_and_backtransform(o, v, nj):
    L, t1 = full_L(o, v, nj, seed=o * 1000 + v)
    ref = T.t1_transform_vv(L, t1)
    got = lad.cc_ladder_t1_transform(dev(L[:, o:, o:]), dev(L[:, :o, o:]), dev(t1))
    assert rel(got.cpu(), ref) < 1e-13
    W = np.zeros_like(L)
    W[:, o:, o:] = np.random.default_rng(v).standard_normal((nj, v, v))
    ref_w = T.w_backtransform_full(W, t1)[:, :o, o:]
    got_w = lad.cc_ladder_w_backtransform(dev(W[:, o:, o:]), dev(t1))
    assert rel(got_w.cpu(), ref_w) < 1e-13
    # twice in a row gives the same bits
    again = lad.cc_ladder_t1_transform(dev(L[:, o:, o:]), dev(L[:, :o, o:]), dev(t1))
    assert torch.equal(again, got)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_t1_form_pass_matches_oracle(prec):
    o, v, nj = 5, 37, 70
    s, tb1, tb2 = synth.make_pair(o, v, nj, 20.0, seed=2202)
    L = np.zeros((nj, o + v, o + v))
    L[:, o:, o:] = s.L_vv
    L[:, :o, o:] = s.L_ov
    L[:, o:, :o] = s.L_ov.transpose(0, 2, 1)
    t1 = s.t1
    Lt = T.t1_transform_vv(L, t1)
    om_ref = O.residual_dense(Lt, s.t2)
    D_ref = O.density_dense(Lt, tb2, s.t2)
    W = np.zeros_like(L)
    W[:, o:, o:] = D_ref
    Wov_ref = T.w_backtransform_full(W, t1)[:, :o, o:]

    Lt_d = lad.cc_ladder_t1_transform(dev(s.L_vv), dev(s.L_ov), dev(t1))
    sd = lad.System(L_vv=Lt_d, t2=dev(s.t2), t1=None, tbar2=dev(tb2))
    ws = lad.workspace([sd], prec)
    om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws)
    assert lad.cc_ladder_status(ws) == 0
    Wov = lad.cc_ladder_w_backtransform(D[0], dev(t1))
    assert rel(om[0].cpu(), om_ref) < TOL[prec]
    assert rel(D[0].cpu(), D_ref) < TOL[prec]
    assert rel(Wov.cpu(), Wov_ref) < TOL[prec]
    assert abs(float(E[0]) - O.lagrangian(tb2, om_ref)) < TOL[prec] * abs(O.lagrangian(tb2, om_ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_excited_state_density_matches_oracle(prec):
    # App. A: d^es_abcd = O^(2)(L2, U), U = T2 R0 + R2; two systems of different size in one call
    cases = [(5, 37, 70, 0.7), (3, 20, 30, -1.3)]
    systems, R2s, R0s, refs = [], [], [], []
    for k, (o, v, nj, r0) in enumerate(cases):
        s, l1, L2 = synth.make_pair(o, v, nj, 20.0, seed=2202 + k)
        rng = np.random.default_rng(40 + k)
        R2 = 0.05 * rng.standard_normal((o, o, v, v))
        R2 = 0.5 * (R2 + R2.transpose(1, 0, 3, 2))
        refs.append(O.density_dense(s.L_vv, L2, T.es_amplitudes(s.t2, R2, r0)))
        systems.append(lad.System(L_vv=dev(s.L_vv), t2=dev(s.t2), t1=dev(s.t1), tbar2=dev(L2)))
        R2s.append(dev(R2))
        R0s.append(r0)
    ws = lad.workspace(systems, prec, lad.CC_WS_DENSITY)
    D = lad.cc_ladder_density_es(systems, R2s, R0s, prec=prec, ws=ws)
    assert lad.cc_ladder_status(ws) == 0
    for k in range(len(cases)):
        assert rel(D[k].cpu(), refs[k]) < TOL[prec], (k, rel(D[k].cpu(), refs[k]))

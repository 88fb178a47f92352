"""GPU parity of the OV^3 contributions to the three-index intermediates
(ground-state d_abic, excited-state d_abci and d_abic) against the FP64 oracle
(explicit-density formulation)."""
import numpy as np
import pytest
import torch

from oracle import ov3 as V
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 1e-6, "fp16x2": 1e-6}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
@pytest.mark.parametrize("o,v,nj", [(3, 7, 5), (5, 37, 70), (8, 48, 160)])
def test_ov3_contributions_match_oracle(o, v, nj, prec):
    s, tb1, tb2 = synth.make_pair(o, v, nj, nj / 6.0, seed=2202)
    R0 = 0.9
    d = V.density_abic_gs(tb1, s.t2, R0)
    ref_vv, ref_ov = V.w_from_abic(d, s.L_vv, s.L_ov)
    W_vv, W_ov = lad.cc_ladder_ov3_gs(dev(s.L_vv), dev(s.L_ov), dev(s.t2), dev(tb1), R0, prec=prec)
    assert rel(W_vv.cpu(), ref_vv) < TOL[prec]
    assert rel(W_ov.cpu(), ref_ov) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("o,v,nj", [(3, 7, 5), (5, 37, 70), (8, 48, 160)])
def test_es_abci_contributions_match_oracle(o, v, nj, prec):
    s, _, L2 = synth.make_pair(o, v, nj, nj / 6.0, seed=2203)
    R1 = np.random.default_rng(o + v).standard_normal((o, v))
    d = V.density_abci_es(L2, R1)
    ref_vv, ref_vo = V.w_from_abci(d, s.L_vv, s.L_ov)
    W_vv, W_vo = lad.cc_ladder_ov3_es_abci(dev(s.L_vv), dev(s.L_ov), dev(L2), dev(R1), prec=prec)
    assert rel(W_vv.cpu(), ref_vv) < TOL[prec]
    assert rel(W_vo.cpu(), ref_vo) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
@pytest.mark.parametrize("o,v,nj", [(3, 7, 5), (5, 37, 70), (8, 48, 160)])
def test_es_abic_contributions_match_oracle(o, v, nj, prec):
    """Excited-state d_abic (App. A, eight terms): W from the explicit OV^3 density of the oracle."""
    s, tb1, L2 = synth.make_pair(o, v, nj, nj / 6.0, seed=2204)
    rng = np.random.default_rng(o * v)
    R1 = 0.1 * rng.standard_normal((o, v))
    R2 = 0.01 * rng.standard_normal((o, o, v, v))
    R2 = 0.5 * (R2 + R2.transpose(1, 0, 3, 2))
    R0 = 0.8
    d = V.density_abic_es(tb1, L2, s.t2, R0, R1, R2)
    ref_vv, ref_ov = V.w_from_abic(d, s.L_vv, s.L_ov)
    W_vv, W_ov = lad.cc_ladder_ov3_es_abic(dev(s.L_vv), dev(s.L_ov), dev(tb1), dev(L2), dev(s.t2), R0, dev(R1),
                                           dev(R2), prec=prec)
    torch.cuda.synchronize()
    print(f"{o}/{v}/{nj} {prec}: W_vv {rel(W_vv.cpu(), ref_vv):.2e}  W_ov {rel(W_ov.cpu(), ref_ov):.2e}")
    assert rel(W_vv.cpu(), ref_vv) < TOL[prec]
    assert rel(W_ov.cpu(), ref_ov) < TOL[prec]

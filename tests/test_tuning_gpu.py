"""Every pair-block edge and leading-product window the tuning knobs and the
autotuner can pick, checked against the FP64 oracle on a system wide enough
for several pair-block rows with ragged tails (v = 157: 5 rows of 32, 4 of
48, 3 of 64, 2 of 96, each with a short last row), and the autotuner's own
choice checked against the oracle, not just for finiteness."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import autotune
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

O_, V_, NJ_, LAM_ = 6, 157, 300, 50.0
TOL = {"fp64": 1e-11, "mixed": 1e-6, "fp16x2": 1e-6}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def case():
    s, tb1, tb2 = synth.make_pair(O_, V_, NJ_, LAM_, seed=2202)
    tt = O.tau(s.t1, s.t2)
    om = O.residual_rows(s.L_vv, tt)
    D = O.density_rows(s.L_vv, tb2, tt)
    d = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    sd = lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps))
    return sd, om, D, O.lagrangian(tb2, om)


def run_checked(sd, prec, om_ref, D_ref, E_ref):
    ws = lad.workspace([sd], prec)
    om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws)
    assert lad.cc_ladder_status(ws) == 0
    eo, ed = rel(om[0].cpu(), om_ref), rel(D[0].cpu(), D_ref)
    ee = abs(float(E[0]) - E_ref) / abs(E_ref)
    return eo, ed, ee


@pytest.mark.parametrize("win", [1, 2, 4])
@pytest.mark.parametrize("block", [32, 48, 64, 96])
@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_every_tuning_candidate_matches_oracle(case, prec, block, win):
    sd, om_ref, D_ref, E_ref = case
    try:
        assert lad.cc_ladder_set_tuning(block, win) is None
        eo, ed, ee = run_checked(sd, prec, om_ref, D_ref, E_ref)
    finally:
        lad.cc_ladder_set_tuning(0, 0)
    print(f"{prec} block {block} win {win}: Omega {eo:.2e} D {ed:.2e} E {ee:.2e}")
    assert eo < TOL[prec] and ed < TOL[prec] and ee < TOL[prec], (eo, ed, ee)


@pytest.mark.parametrize("block", [32, 96, 160])
def test_block_edges_on_the_fp64_path(case, block):
    sd, om_ref, D_ref, E_ref = case
    try:
        lad.cc_ladder_set_tuning(block, 0)
        eo, ed, ee = run_checked(sd, "fp64", om_ref, D_ref, E_ref)
    finally:
        lad.cc_ladder_set_tuning(0, 0)
    assert eo < 1e-11 and ed < 1e-11 and ee < 1e-11, (eo, ed, ee)


def test_autotuned_choice_matches_oracle(case, tmp_path):
    sd, om_ref, D_ref, E_ref = case
    try:
        r = autotune.tune([sd], prec="mixed", path=str(tmp_path / "tune.json"))
        assert r["source"] == "measured" and r["block"] > 0 and r["win"] >= 0
        assert r["kernel"] in (lad.CC_KERNEL_SINGLE, lad.CC_KERNEL_KBLOCK_WINDOWS)
        assert len([t for t in r["tried"] if t["ms"] is not None]) >= 2
        eo, ed, ee = run_checked(sd, "mixed", om_ref, D_ref, E_ref)   # runs with the tuned knobs
    finally:
        lad.cc_ladder_set_tuning(0, 0)
        lad.cc_ladder_set_contraction(0)
    assert eo < TOL["mixed"] and ed < TOL["mixed"] and ee < TOL["mixed"], (r, eo, ed, ee)

"""One system split over several GPUs, emulated on one: an LPT partition of the
pair blocks into shards, each run through cc_ladder_step_blocks as a rank
would.  The shards' Omega entries are disjoint, cover every entry and equal the
whole step's (bit for bit on the split paths; on the FP64 path up to the order
of its atomic split-K additions); their partial D and E sum to the whole step's
(up to the order of the additions) and to the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def case():
    s, tb1, tb2 = synth.make_pair(6, 61, 150, 25.0, seed=2202)
    tt = O.tau(s.t1, s.t2)
    om = O.residual_rows(s.L_vv, tt)
    D = O.density_rows(s.L_vv, tb2, tt)
    d = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    return lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps)), om, D, O.lagrangian(tb2, om)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_shards_reassemble_the_step(case, prec, world):
    sd, om_ref, D_ref, E_ref = case
    try:
        lad.cc_ladder_set_tuning(16, 0)          # 4 block rows, 10 pair blocks at v = 61
        n, edge = lad.cc_ladder_pair_blocks(sd)
        assert n == 10 and edge == 16
        ws = lad.workspace([sd], prec)
        om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws)
        om_s = torch.full_like(sd.t2, float("nan"))
        D_sum = torch.zeros_like(sd.L_vv)
        E_sum = 0.0
        owned = []
        for rank in range(world):
            mine = shard.rank_blocks(sd, rank, world)
            owned += mine
            _, Dp, Ep = lad.cc_ladder_step_blocks(sd, mine, prec=prec, ws=ws, omega=om_s)
            assert lad.cc_ladder_status(ws) == 0
            D_sum += Dp
            E_sum += float(Ep[0])
        torch.cuda.synchronize()
    finally:
        lad.cc_ladder_set_tuning(0, 0)
    assert sorted(owned) == list(range(n))
    assert not torch.isnan(om_s).any()                      # every entry written by some shard
    if prec == "fp64":   # split-K chunks meet in FP64 atomic adds: equal up to the order of the additions
        assert rel(om_s.cpu(), om[0].cpu()) < 1e-14
    else:                # no atomics on the split paths: the same bits as the whole step
        assert torch.equal(om_s, om[0])
    assert rel(D_sum.cpu(), D[0].cpu()) < 1e-13
    assert abs(E_sum - float(E[0])) < 1e-13 * abs(float(E[0]))
    tol = 1e-11 if prec == "fp64" else 1e-6
    assert rel(om_s.cpu(), om_ref) < tol and rel(D_sum.cpu(), D_ref) < tol

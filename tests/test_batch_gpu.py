"""Batched systems: one graph-captured call over systems of uneven size --
with the batched schedule (pair blocks of several systems in every grouped
contraction launch) and back to back -- gives the same bits as one call per
system on the split paths, and matches the oracle; the autotuner picks and
caches knobs whose results match the oracle."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import autotune
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(3, 7, 35), (6, 50, 250), (4, 23, 115), (8, 61, 305), (2, 12, 60), (5, 33, 165)]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def batch():
    d = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    host, dev = [], []
    for k, (o, v, nj) in enumerate(SIZES):
        s, tb1, tb2 = synth.make_pair(o, v, nj, 12.0, seed=2202 + 10 * k)
        host.append((s, tb2))
        dev.append(lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps)))
    return host, dev


@pytest.mark.parametrize("batched", [True, False], ids=["batched", "back_to_back"])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp16x2"])
def test_graph_captured_batch_equals_one_by_one(batch, prec, batched):
    host, systems = batch
    ws = lad.workspace(systems, prec, batched=batched)
    assert ws.numel() == lad.cc_ladder_workspace_size(systems, prec, batched=batched)
    if batched:
        assert ws.numel() > lad.cc_ladder_workspace_size(systems, prec)
    om = [torch.empty_like(s.t2) for s in systems]
    D = [torch.empty_like(s.L_vv) for s in systems]
    E = torch.empty(len(systems), dtype=torch.float64, device="cuda")
    lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)     # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)
    for x in om + D:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert lad.cc_ladder_status(ws) == 0
    tol = 1e-11 if prec == "fp64" else 1e-6
    for k, sd in enumerate(systems):
        om1, D1, E1 = lad.cc_ladder_step([sd], prec=prec)
        torch.cuda.synchronize()
        if prec != "fp64":    # no additive atomics on the split paths: replay is bit-for-bit
            assert torch.equal(om[k], om1[0]) and torch.equal(D[k], D1[0]) and float(E[k]) == float(E1[0])
        else:                 # FP64 split-K chunks meet in atomic adds: equal up to summation order
            assert rel(om[k].cpu(), om1[0].cpu()) < 1e-14 and rel(D[k].cpu(), D1[0].cpu()) < 1e-14
        s, tb2 = host[k]
        tt = O.tau(s.t1, s.t2)
        assert rel(om[k].cpu(), O.residual_rows(s.L_vv, tt)) < tol
        assert rel(D[k].cpu(), O.density_rows(s.L_vv, tb2, tt)) < tol


def test_autotuner_picks_and_caches(batch, tmp_path):
    host, systems = batch
    path = str(tmp_path / "tune.json")
    try:
        cands = ((48, 4, lad.CC_KERNEL_SINGLE), (32, 2, lad.CC_KERNEL_SINGLE), (48, 0, lad.CC_KERNEL_KBLOCK_WINDOWS))
        r = autotune.tune(systems[:3], prec="mixed", candidates=cands, path=path)
        assert r["source"] == "measured" and (r["block"], r["win"], r["kernel"]) in cands
        assert os.path.exists(path)
        r2 = autotune.tune(systems[:3], prec="mixed", path=path)
        assert r2["source"] == "cache" and (r2["block"], r2["win"], r2["kernel"]) == (r["block"], r["win"], r["kernel"])
        om, D, E = lad.cc_ladder_step(systems[:3], prec="mixed")      # runs with the tuned knobs
        torch.cuda.synchronize()
    finally:
        lad.cc_ladder_set_tuning(0, 0)
        lad.cc_ladder_set_contraction(0)
    for k in range(3):
        s, tb2 = host[k]
        tt = O.tau(s.t1, s.t2)
        om_ref = O.residual_rows(s.L_vv, tt)
        assert rel(om[k].cpu(), om_ref) < 1e-6
        assert rel(D[k].cpu(), O.density_rows(s.L_vv, tb2, tt)) < 1e-6
        E_ref = O.lagrangian(tb2, om_ref)
        assert abs(float(E[k]) - E_ref) < 1e-6 * abs(E_ref)


@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_batched_schedule_with_more_systems_than_slots(prec):
    """Eleven systems, eight scratch slots and a small block edge: slots change owner between waves many
    times while the two chains of a wave run on two streams; the outputs stay the bits of one call per
    system, and the oracle's."""
    d = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    sizes = [(3, 29, 40), (5, 44, 60), (2, 17, 30), (6, 51, 70), (4, 38, 50), (3, 25, 35), (7, 47, 65),
             (2, 33, 45), (5, 20, 28), (4, 41, 55), (6, 36, 48)]
    host, systems = [], []
    for k, (o, v, nj) in enumerate(sizes):
        s, tb1, tb2 = synth.make_pair(o, v, nj, 10.0, seed=4400 + k)
        host.append((s, tb2))
        systems.append(lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps)))
    try:
        lad.cc_ladder_set_tuning(12, 0)
        ws = lad.workspace(systems, prec, batched=True)
        om, D, E = lad.cc_ladder_step(systems, prec=prec, ws=ws)
        torch.cuda.synchronize()
        assert lad.cc_ladder_status(ws) == 0
        for k, sd in enumerate(systems):
            om1, D1, E1 = lad.cc_ladder_step([sd], prec=prec)
            torch.cuda.synchronize()
            assert torch.equal(om[k], om1[0]) and torch.equal(D[k], D1[0]) and float(E[k]) == float(E1[0]), k
    finally:
        lad.cc_ladder_set_tuning(0, 0)
    for k in range(len(systems)):
        s, tb2 = host[k]
        tt = O.tau(s.t1, s.t2)
        assert rel(om[k].cpu(), O.residual_rows(s.L_vv, tt)) < 1e-6
        assert rel(D[k].cpu(), O.density_rows(s.L_vv, tb2, tt)) < 1e-6

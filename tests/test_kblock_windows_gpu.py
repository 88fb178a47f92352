"""The one-window-per-k-block contraction kernels (all products of a 64-term
k-block in one accumulator, small products first, three window buffers; one
CTA per tile or CTA pairs) against the FP64 oracle: a tiny system, a system
with several ragged pair-block rows (v = 157) at several pair-block edges,
the pair form against the single-CTA form (bitwise), and a graph-captured
batch against one call per system (bitwise)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-6, "fp16x2": 1e-6}
K = lad.CC_KERNEL_KBLOCK_WINDOWS


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(o, v, nj, lam, seed):
    s, tb1, tb2 = synth.make_pair(o, v, nj, lam, seed=seed)
    tt = O.tau(s.t1, s.t2)
    om = O.residual_rows(s.L_vv, tt)
    D = O.density_rows(s.L_vv, tb2, tt)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sd = lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps))
    return sd, om, D, O.lagrangian(tb2, om)


def step(sd, prec, block=0, kernel=K):
    try:
        lad.cc_ladder_set_contraction(kernel)
        lad.cc_ladder_set_tuning(block, 0)
        ws = lad.workspace([sd], prec)
        om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws)
        torch.cuda.synchronize()
        assert lad.cc_ladder_status(ws) == 0
    finally:
        lad.cc_ladder_set_contraction(0)
        lad.cc_ladder_set_tuning(0, 0)
    return om[0].cpu(), D[0].cpu(), float(E[0])


@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_kblock_windows_tiny_system(prec):
    sd, om_ref, D_ref, E_ref = make(3, 7, 5, 2.0, seed=11)
    om, D, E = step(sd, prec)
    assert rel(om, om_ref) < TOL[prec] and rel(D, D_ref) < TOL[prec]
    assert abs(E - E_ref) / abs(E_ref) < TOL[prec]


@pytest.fixture(scope="module")
def ragged():
    return make(6, 157, 300, 50.0, seed=2202)


@pytest.mark.parametrize("block", [32, 48, 96])
@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_kblock_windows_match_oracle(ragged, prec, block):
    sd, om_ref, D_ref, E_ref = ragged
    om, D, E = step(sd, prec, block)
    eo, ed, ee = rel(om, om_ref), rel(D, D_ref), abs(E - E_ref) / abs(E_ref)
    print(f"k-block windows {prec} block {block}: Omega {eo:.2e} D {ed:.2e} E {ee:.2e}")
    assert eo < TOL[prec] and ed < TOL[prec] and ee < TOL[prec], (eo, ed, ee)
    om2, D2, E2 = step(sd, prec, block, lad.CC_KERNEL_PAIR_KBLOCK_WINDOWS)
    assert torch.equal(om, om2) and torch.equal(D, D2) and E == E2


@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_pair_kblock_windows_tiny_system(prec):
    sd, om_ref, D_ref, E_ref = make(3, 7, 5, 2.0, seed=12)
    om, D, E = step(sd, prec, 0, lad.CC_KERNEL_PAIR_KBLOCK_WINDOWS)
    assert rel(om, om_ref) < TOL[prec] and rel(D, D_ref) < TOL[prec]
    assert abs(E - E_ref) / abs(E_ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp16x2"])
def test_kblock_windows_batch_equals_one_by_one(prec):
    sizes = [(3, 7, 35), (6, 50, 250), (4, 23, 115), (8, 61, 305), (2, 12, 60)]
    systems = []
    for k, (o, v, nj) in enumerate(sizes):
        s, tb1, tb2 = synth.make_pair(o, v, nj, 12.0, seed=4202 + 10 * k)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        systems.append(lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps)))
    om = [torch.empty_like(s.t2) for s in systems]
    D = [torch.empty_like(s.L_vv) for s in systems]
    E = torch.empty(len(systems), dtype=torch.float64, device="cuda")
    try:
        lad.cc_ladder_set_contraction(K)
        ws = lad.workspace(systems, prec, batched=True)
        lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)
        for x in om + D:
            x.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert lad.cc_ladder_status(ws) == 0
    finally:
        lad.cc_ladder_set_contraction(0)
    for k, sd in enumerate(systems):
        o1, D1, E1 = step(sd, prec)
        assert torch.equal(om[k].cpu(), o1) and torch.equal(D[k].cpu(), D1)
        assert float(E[k]) == E1

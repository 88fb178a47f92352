"""GPU parity at the full retinal-scale workload (o=78, v=650, N_J=4000), in the
launch configuration the benchmark times: one cc_ladder_step on device-resident
inputs, checked on outputs the FP64 oracle computes one row at a time -- all
Omega_ij^ab and D^J_ac for one seeded virtual row a in every pair-block band
(rows 48k .. 48k+47, 14 bands, the last one ragged) and a seeded spread of
b / c columns -- and by the Euler identity sum_J,ac L^J_ac D^J_ac = E, which
holds at any size.  Each sampled row is checked on its own: its relative
Frobenius error and its largest element error against its largest element.

This is the longest GPU test (about two minutes on one GB300, most of it the
oracle's rows on the host cores); the file name sorts it after the other GPU
tests and before the no-allocation entry point's test.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-6, "fp16x2": 1e-6}
BLOCK = 48


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def band_rows(v, s, seed):
    rng = np.random.default_rng(seed)
    return [int(rng.integers(lo, min(lo + s, v))) for lo in range(0, v, s)]


def test_retinal_scale_sampled_parity():
    o, v, nj, lam = 78, 650, 4000, 700.0
    d = synth.make_pair_torch(o, v, nj, lam, seed=2202, device="cuda")
    sd = lad.System(L_vv=d["L_vv"], t2=d["t2"], t1=d["t1"], tbar2=d["tbar2"], eps=d["eps"])
    rows = band_rows(v, BLOCK, 2202)
    assert len(rows) == 14
    cols = sorted(np.random.default_rng(2203).choice(v, size=24, replace=False).tolist())
    h = {k: d[k].cpu().numpy() for k in ("L_vv", "t1", "t2", "tbar2")}
    tt = O.tau(h["t1"], h["t2"])
    om_ref = O.residual_rows(h["L_vv"], tt, rows, cols)          # [o, o, rows, cols]
    D_ref = O.density_rows(h["L_vv"], h["tbar2"], tt, rows, cols)  # [nj, rows, cols]
    del h, tt
    om = [torch.empty_like(sd.t2)]
    D = [torch.empty_like(sd.L_vv)]
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    for prec in ("mixed", "fp16x2"):
        ws = lad.workspace([sd], prec)
        lad.cc_ladder_step([sd], prec=prec, ws=ws, omega=om, D=D, E=E)
        assert lad.cc_ladder_status(ws) == 0
        del ws
        torch.cuda.empty_cache()
        got_om = om[0][:, :, rows, :][:, :, :, cols].cpu().numpy()
        got_D = D[0][:, rows, :][:, :, cols].cpu().numpy()
        assert rel(got_om, om_ref) < TOL[prec], (prec, rel(got_om, om_ref))
        assert rel(got_D, D_ref) < TOL[prec], (prec, rel(got_D, D_ref))
        for k, a in enumerate(rows):
            for name, g, r in (("Omega", got_om[:, :, k, :], om_ref[:, :, k, :]), ("D", got_D[:, k, :], D_ref[:, k, :])):
                fro = rel(g, r)
                mx = float(np.max(np.abs(g - r)) / np.max(np.abs(r)))
                assert fro < TOL[prec] and mx < TOL[prec], (prec, name, a, fro, mx)
        Ev = float(E[0])
        euler = float(torch.sum(sd.L_vv * D[0]))
        assert abs(euler - Ev) < TOL[prec] * abs(Ev), (prec, euler, Ev)

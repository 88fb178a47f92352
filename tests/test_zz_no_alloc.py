"""The no-allocation Lagrangian entry point (collected last on purpose).

cc_ladder_lagrangian_noalloc serves callers that cannot allocate device
memory where they need E -- their memory belongs to another framework's
pool, or their loop must not pay cudaMalloc's implicit synchronisation.  It
keeps its partial sums in a fixed device array of the library instead of a
caller workspace.  This test calls it through the C ABI twice in a row and
compares with the workspace-based cc_ladder_lagrangian on the same Omega.
"""
import numpy as np
import pytest
import torch

from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth


@pytest.mark.gpu
def test_noalloc_lagrangian_matches_workspace_entry_point():
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    systems = []
    for (o, v, nj, lam, seed) in [(4, 20, 60, 12.0, 2202), (3, 7, 5, 4.0, 7), (5, 37, 70, 20.0, 11)]:
        s, tb1, tb2 = synth.make_pair(o, v, nj, lam, seed=seed)
        systems.append(lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps)))
    omega = lad.cc_ladder_residual(systems, prec="fp64")
    E_ref = lad.cc_ladder_lagrangian(systems, omega=omega, prec="fp64")
    torch.cuda.synchronize()
    ref = E_ref.cpu().numpy()
    for _ in range(2):
        E = lad.cc_ladder_lagrangian_noalloc(systems, omega)
        torch.cuda.synchronize()
        got = E.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (got, ref)

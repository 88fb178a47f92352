"""The no-allocation Lagrangian entry point (collected last on purpose).

cc_ladder_lagrangian_noalloc serves callers that cannot allocate device
memory where they need E -- their memory belongs to another framework's
pool, or their loop must not pay cudaMalloc's implicit synchronisation.  It
keeps its partial sums in a fixed device array of the library instead of a
caller workspace.  This test calls it through the C ABI twice in a row with
a preallocated E and compares with the workspace-based cc_ladder_lagrangian
on the same Omega; around those two calls neither PyTorch's allocator nor
the device's free memory may change.  One call comes first, unmeasured: the
first call on a device resolves the array's device address, and under
CUDA's lazy module loading that is when the driver brings the library's
code and the array itself onto the GPU.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_02019_gb300 import ladder as lad
from paper_2202_02019_gb300 import synth


def _free_bytes():
    # cudaMemGetInfo through the runtime PyTorch already loaded
    free, _ = torch.cuda.mem_get_info()
    return free


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
    E = torch.full((len(systems),), float("nan"), dtype=torch.float64, device=dev)
    lib = lad.load()
    arr = lad._arr(systems)
    om = lad._outs(omega, systems, "t2", "Omega")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cc_ladder_lagrangian_noalloc(arr, len(systems), ctypes.c_void_p(E.data_ptr()), om, stream)
    assert rc == 0, lad.cc_ladder_strerror(rc)          # set-up call on this device
    E.fill_(float("nan"))
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), _free_bytes()
    results = []
    for _ in range(2):
        rc = lib.cc_ladder_lagrangian_noalloc(arr, len(systems), ctypes.c_void_p(E.data_ptr()), om, stream)
        assert rc == 0, lad.cc_ladder_strerror(rc)
        torch.cuda.synchronize()
        results.append(E.cpu().numpy().copy())
        E.fill_(float("nan"))   # the second call must write every entry again
        torch.cuda.synchronize()
    alloc1, free1 = torch.cuda.memory_allocated(), _free_bytes()
    for got in results:
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (got, ref)
    assert alloc1 == alloc0, (alloc0, alloc1)
    assert free1 == free0, (free0, free1)

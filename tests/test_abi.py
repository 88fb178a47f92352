"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/ccladder.h declares, sizes workspaces and rejects bad
arguments on the host."""
import ctypes
import os
import re

import pytest

from paper_2202_02019_gb300 import ladder as lad

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ccladder.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_ladder_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = lad.load()
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lad.EXPORTS)


def fake_sys(o, v, nj):
    # host-side sizing never dereferences these pointers
    return lad.cc_ladder_system(o, v, nj, 0x1000, 0x2000, 0x3000, 0x4000, 0x5000)


def test_workspace_size_host_only():
    lib = lad.load()
    for prec in (0, 1):
        arr = (lad.cc_ladder_system * 1)(fake_sys(4, 20, 60))
        r = lib.cc_ladder_workspace_size(arr, 1, prec, lad.CC_WS_RESIDUAL)
        d = lib.cc_ladder_workspace_size(arr, 1, prec, lad.CC_WS_DENSITY)
        s = lib.cc_ladder_workspace_size(arr, 1, prec, lad.CC_WS_STEP)
        assert r > 0 and d > 0 and s >= max(r, d)
    # retinal-scale workspace stays far below the 280 GB of one GPU
    arr = (lad.cc_ladder_system * 1)(fake_sys(78, 650, 4000))
    big = lib.cc_ladder_workspace_size(arr, 1, 1, lad.CC_WS_STEP)
    assert 10e9 < big < 100e9
    # a list is sized by its largest member
    arr2 = (lad.cc_ladder_system * 2)(fake_sys(4, 20, 60), fake_sys(6, 30, 90))
    one = (lad.cc_ladder_system * 1)(fake_sys(6, 30, 90))
    assert lib.cc_ladder_workspace_size(arr2, 2, 1, 7) == lib.cc_ladder_workspace_size(one, 1, 1, 7)


def test_host_argument_errors():
    lib = lad.load()
    arr = (lad.cc_ladder_system * 1)(fake_sys(0, 20, 60))
    assert lib.cc_ladder_workspace_size(arr, 1, 1, 7) == 0
    assert lib.cc_ladder_workspace_size(None, 1, 1, 7) == 0
    assert lib.cc_ladder_workspace_size((lad.cc_ladder_system * 1)(fake_sys(4, 20, 60)), 1, 5, 7) == 0
    out = (ctypes.c_void_p * 1)(0x6000)
    assert lib.cc_ladder_residual(arr, 1, out, 1, ctypes.c_void_p(0x10000), 1 << 20, None) == -1
    assert lib.cc_ladder_residual(None, 1, out, 1, ctypes.c_void_p(0x10000), 1 << 20, None) == -1
    good = (lad.cc_ladder_system * 1)(fake_sys(4, 20, 60))
    # misaligned workspace
    assert lib.cc_ladder_residual(good, 1, out, 1, ctypes.c_void_p(0x10008), 1 << 40, None) == -1
    # density without tbar2
    nob = (lad.cc_ladder_system * 1)(lad.cc_ladder_system(4, 20, 60, 0x1000, 0, 0x3000, 0, 0))
    assert lib.cc_ladder_density(nob, 1, out, 1, ctypes.c_void_p(0x10000), 1 << 40, None) == -1


def test_strerror():
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(lad.cc_ladder_strerror(code), str)
    assert "TIMEOUT" in lad.cc_ladder_strerror(-5)


def test_noalloc_size_limit_is_host_checked():
    lib = lad.load()
    n = 65
    arr = (lad.cc_ladder_system * n)(*[fake_sys(2, 3, 4) for _ in range(n)])
    om = (ctypes.c_void_p * n)(*([0x6000] * n))
    assert lib.cc_ladder_lagrangian_noalloc(arr, n, ctypes.c_void_p(0x7000), om, None) == -6
    assert "64 systems" in lad.cc_ladder_strerror(-6)


def test_t1_entry_points_host_checks():
    # argument errors are caught on the host before any device work
    lib = lad.load()
    P = ctypes.c_void_p
    good = [P(0x10000), P(0x20000), P(0x30000)]
    assert lib.cc_ladder_t1_transform(0, 5, 3, *good, P(0x40000), None) == -1
    assert lib.cc_ladder_t1_transform(2, 5, 3, None, good[1], good[2], P(0x40000), None) == -1
    assert lib.cc_ladder_t1_transform(2, 5, 3, *good, P(0x40004), None) == -1          # misaligned
    assert lib.cc_ladder_t1_transform(2, 5, 3, *good, P(0x10000 + 8), None) == -1      # output overlaps L_vv
    assert lib.cc_ladder_w_backtransform(2, 5, 0, good[0], good[1], P(0x40000), None) == -1
    assert lib.cc_ladder_w_backtransform(2, 5, 3, good[0], good[1], P(0x20000), None) == -1  # overlaps t1


def test_workspace_queries_and_argument_errors_of_the_extra_entry_points():
    # host-side checks only: sizes, NULLs and alignment are rejected before any device work
    lib = lad.load()
    P = ctypes.c_void_p
    assert lib.cc_ladder_mp2_driver_workspace_size(0, 5, 3, 1) == 0
    assert lib.cc_ladder_mp2_driver_workspace_size(2, 5, 3, 9) == 0
    assert lib.cc_ladder_mp2_driver_workspace_size(2, 5, 3, 0) > lib.cc_ladder_mp2_driver_workspace_size(2, 5, 3, 1) > 0
    assert lib.cc_ladder_ov3_workspace_size(2, 5, 3, 1) > 0 and lib.cc_ladder_ov3_workspace_size(2, 0, 3, 1) == 0
    ws = P(0x100000)
    assert lib.cc_ladder_mp2_driver(2, 5, 3, None, P(0x2000), 1, ws, 1 << 30, None) == -1
    assert lib.cc_ladder_mp2_driver(2, 5, 3, P(0x1000), P(0x2004), 1, ws, 1 << 30, None) == -1
    assert lib.cc_ladder_mp2_driver(2, 5, 3, P(0x1000), P(0x2000), 1, P(0x100008), 1 << 30, None) == -1
    assert lib.cc_ladder_ov3_gs(2, 5, 3, P(0x1000), P(0x2000), None, P(0x3000), ctypes.c_double(1.0),
                                P(0x4000), P(0x5000), 1, ws, 1 << 30, None) == -1
    assert lib.cc_ladder_ov3_es_abci(2, 5, 3, P(0x1000), P(0x2000), P(0x3000), P(0x3800), P(0x4000), None, 1,
                                     ws, 1 << 30, None) == -1
    arr = (lad.cc_ladder_system * 1)(fake_sys(2, 5, 3))
    assert lib.cc_ladder_iterate_workspace_size(arr, 1) > 0
    # eps is required by the iteration, and at least one step
    no_eps = (lad.cc_ladder_system * 1)(lad.cc_ladder_system(2, 5, 3, 0x1000, 0x2000, 0x3000, 0x4000, 0))
    assert lib.cc_ladder_iterate(no_eps, P(0x7000), 2, P(0x8000), P(0x9000), 1, ws, 1 << 30, None) == -1
    assert lib.cc_ladder_iterate(arr, P(0x7000), 0, P(0x8000), P(0x9000), 1, ws, 1 << 30, None) == -1
    assert lib.cc_ladder_density_es(arr, 1, None, (ctypes.c_double * 1)(1.0), (P * 1)(0x6000), 1, ws, 1 << 30,
                                    None) == -1


def test_binding_rejects_host_tensors_before_any_call():
    # a host pointer handed to the kernels would be read as device memory: the binding refuses it
    import torch
    s = lad.System(L_vv=torch.zeros(3, 4, 4, dtype=torch.float64), t2=torch.zeros(2, 2, 4, 4, dtype=torch.float64))
    with pytest.raises(ValueError):
        s.c_struct()
    with pytest.raises(ValueError):
        lad._ptrs([torch.zeros(4, dtype=torch.float64)])
    with pytest.raises(ValueError):
        lad._f64(torch.zeros(4, dtype=torch.float64), "x")
    with pytest.raises(ValueError):
        lad.cc_ladder_density_es([s], [], [1.0])


def test_binding_checks_lengths_shapes_and_E_on_the_host():
    # every check below fires before any device pointer is taken, so CPU tensors exercise them
    import torch
    f = lambda *sh: torch.zeros(*sh, dtype=torch.float64)
    s = lad.System(L_vv=f(3, 4, 4), t2=f(2, 2, 4, 4), t1=f(2, 4), tbar2=f(2, 2, 4, 4), eps=f(6))
    # one output per system, each shaped like the system's t2 (Omega) or L_vv (D)
    with pytest.raises(ValueError, match="one buffer per system"):
        lad._outs([f(2, 2, 4, 4), f(2, 2, 4, 4)], [s], "t2", "Omega")
    with pytest.raises(ValueError, match="one buffer per system"):
        lad._outs([], [s], "L_vv", "D")
    with pytest.raises(ValueError, match="shape"):
        lad._outs([f(2, 2, 4, 5)], [s], "t2", "Omega")
    with pytest.raises(ValueError, match="shape"):
        lad._outs([f(3, 4, 5)], [s], "L_vv", "D")
    # E: 1-D float64 with room for every system
    with pytest.raises(ValueError, match="at least 2"):
        lad._energy(f(1), 2)
    with pytest.raises(ValueError, match="at least 1"):
        lad._energy(f(1, 1), 1)
    with pytest.raises(ValueError, match="float64"):
        lad._energy(torch.zeros(2, dtype=torch.float32), 2)
    # inconsistent system shapes
    for bad in (dict(t1=f(2, 5)), dict(tbar2=f(2, 2, 4, 3)), dict(eps=f(5)), dict(L_vv=f(3, 4, 5))):
        kw = dict(L_vv=s.L_vv, t2=s.t2, t1=s.t1, tbar2=s.tbar2, eps=s.eps)
        kw.update(bad)
        with pytest.raises(ValueError, match="shape"):
            lad.System(**kw).c_struct()
    with pytest.raises(ValueError, match="at least one system"):
        lad._arr([])
    # a host workspace is refused before its address is taken
    with pytest.raises(ValueError, match="GPU memory"):
        lad._ws_args(torch.zeros(16, dtype=torch.uint8))
    # the no-allocation wrapper does not allocate E for the caller
    with pytest.raises(TypeError):
        lad.cc_ladder_lagrangian_noalloc([s], [f(2, 2, 4, 4)])


def test_batched_workspace_size_host_only():
    lib = lad.load()
    B = lad.CC_WS_BATCH
    one = (lad.cc_ladder_system * 1)(fake_sys(6, 30, 90))
    # a single system has nothing to interleave: same size either way
    assert lib.cc_ladder_workspace_size(one, 1, 1, 7 | B) == lib.cc_ladder_workspace_size(one, 1, 1, 7)
    sizes = [(4, 20, 60), (6, 30, 90), (5, 57, 120), (3, 11, 40)]
    arr = (lad.cc_ladder_system * 4)(*[fake_sys(*x) for x in sizes])
    for prec in (0, 1, 2):
        seq = lib.cc_ladder_workspace_size(arr, 4, prec, 7)
        bat = lib.cc_ladder_workspace_size(arr, 4, prec, 7 | B)
        # every system keeps its own prepared operands, and each slot fits the largest block
        singles = [lib.cc_ladder_workspace_size((lad.cc_ladder_system * 1)(fake_sys(*x)), 1, prec, 7) for x in sizes]
        assert seq == max(singles)
        assert bat > seq
        assert bat < sum(singles) + 4 * max(singles)
    # the batch bit alone (no call selected) is not a valid request
    assert lib.cc_ladder_workspace_size(arr, 4, 1, B) == 0
    assert lib.cc_ladder_workspace_size(arr, 4, 1, 7 | 16) == 0


def test_pair_block_enumeration_matches_the_shard_plan():
    # host-only query: the library's pair-block count and edge agree with shard.pair_blocks
    import ctypes as C
    from paper_2202_02019_gb300 import shard
    lib = lad.load()
    try:
        for edge in (0, 16, 48, 52):
            lib.cc_ladder_set_tuning(edge, 0)
            for v in (1, 7, 48, 49, 150, 650):
                arr = (lad.cc_ladder_system * 1)(fake_sys(3, v, 10))
                cnt, e = C.c_int32(), C.c_int32()
                assert lib.cc_ladder_pair_blocks(arr, C.byref(cnt), C.byref(e)) == 0
                assert len(shard.pair_blocks(v, e.value)) == cnt.value
                assert e.value == min(edge or 48, ((v + 3) // 4) * 4)
    finally:
        lib.cc_ladder_set_tuning(0, 0)
    # shard arguments are checked on the host: empty, out of range and repeated block lists
    P = C.c_void_p
    arr = (lad.cc_ladder_system * 1)(fake_sys(3, 20, 10))
    ws = P(0x100000)
    for bl in ([], [3], [0, 0], [-1]):
        arrb = (C.c_int32 * max(1, len(bl)))(*bl)
        assert lib.cc_ladder_step_blocks(arr, arrb, len(bl), P(0x8000), P(0x9000), P(0xA000), 1, ws, 1 << 40,
                                         None) == -1


def test_tuning_knobs_reject_unknown_values_on_the_host():
    lib = lad.load()
    for kind in (5, -1, 7):
        assert lib.cc_ladder_set_contraction(kind) == -1
    with pytest.raises(lad.LadderError):
        lad.cc_ladder_set_contraction(5)
    for kind in (0, lad.CC_KERNEL_SINGLE, lad.CC_KERNEL_PAIR, lad.CC_KERNEL_KBLOCK_WINDOWS, lad.CC_KERNEL_PAIR_KBLOCK_WINDOWS, 0):
        assert lib.cc_ladder_set_contraction(kind) == 0
    for win in (3, 5, 16, -1):
        assert lib.cc_ladder_set_tuning(0, win) == -1
    assert lib.cc_ladder_set_tuning(0, 0) == 0

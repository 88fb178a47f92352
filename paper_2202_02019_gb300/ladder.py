"""Thin ctypes binding of ``libccladder`` (see include/ccladder.h).

Argument marshalling only: every step of the ladder runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  Importing works
without a GPU; calling anything raises if the library or the device is
missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _build

CC_PREC = {"fp64": 0, "mixed": 1, "fp16x2": 2}
CC_WS_RESIDUAL, CC_WS_DENSITY, CC_WS_LAGRANGIAN, CC_WS_STEP = 1, 2, 4, 7

_lib = None


class LadderError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class cc_ladder_system(ctypes.Structure):
    _fields_ = [
        ("o", ctypes.c_int32), ("v", ctypes.c_int32), ("nj", ctypes.c_int32),
        ("L_vv", ctypes.c_void_p), ("t1", ctypes.c_void_p), ("t2", ctypes.c_void_p),
        ("tbar2", ctypes.c_void_p), ("eps", ctypes.c_void_p),
    ]


def load(build_if_missing: bool = True):
    """Load (building first if needed) the in-tree shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libccladder is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, S, I, VP = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    SYS = ctypes.POINTER(cc_ladder_system)
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.cc_ladder_workspace_size.argtypes = [SYS, I, I, I]
    lib.cc_ladder_workspace_size.restype = S
    for name in ("cc_ladder_residual", "cc_ladder_density", "cc_ladder_residual_adjoint"):
        getattr(lib, name).argtypes = [SYS, I, PP, I, VP, S, VP]
        getattr(lib, name).restype = I
    lib.cc_ladder_density_es.argtypes = [SYS, I, PP, ctypes.POINTER(ctypes.c_double), PP, I, VP, S, VP]
    lib.cc_ladder_density_es.restype = I
    lib.cc_ladder_lagrangian.argtypes = [SYS, I, P, PP, I, VP, S, VP]
    lib.cc_ladder_lagrangian.restype = I
    lib.cc_ladder_step.argtypes = [SYS, I, PP, PP, P, I, VP, S, VP]
    lib.cc_ladder_step.restype = I
    lib.cc_ladder_update.argtypes = [SYS, I, PP, PP, VP]
    lib.cc_ladder_update.restype = I
    lib.cc_ladder_status.argtypes = [VP, VP]
    lib.cc_ladder_status.restype = I
    lib.cc_ladder_debug_wait.argtypes = [P, ctypes.c_longlong, VP, VP]
    lib.cc_ladder_debug_wait.restype = I
    lib.cc_ladder_strerror.argtypes = [I]
    lib.cc_ladder_strerror.restype = ctypes.c_char_p
    lib.cc_ladder_launch_count.argtypes = []
    lib.cc_ladder_launch_count.restype = ctypes.c_longlong
    lib.cc_ladder_lagrangian_noalloc.argtypes = [SYS, I, P, PP, VP]
    lib.cc_ladder_lagrangian_noalloc.restype = I
    lib.cc_ladder_t1_transform.argtypes = [I, I, I, P, P, P, P, VP]
    lib.cc_ladder_t1_transform.restype = I
    lib.cc_ladder_w_backtransform.argtypes = [I, I, I, P, P, P, VP]
    lib.cc_ladder_w_backtransform.restype = I
    lib.cc_ladder_mp2_driver_workspace_size.argtypes = [I, I, I, I]
    lib.cc_ladder_mp2_driver_workspace_size.restype = S
    lib.cc_ladder_mp2_driver.argtypes = [I, I, I, P, P, I, VP, S, VP]
    lib.cc_ladder_mp2_driver.restype = I
    lib.cc_ladder_iterate_workspace_size.argtypes = [SYS, I]
    lib.cc_ladder_iterate_workspace_size.restype = S
    lib.cc_ladder_iterate.argtypes = [SYS, P, I, P, P, I, VP, S, VP]
    lib.cc_ladder_iterate.restype = I
    lib.cc_ladder_ov3_workspace_size.argtypes = [I, I, I, I]
    lib.cc_ladder_ov3_workspace_size.restype = S
    lib.cc_ladder_ov3_gs.argtypes = [I, I, I, P, P, P, P, ctypes.c_double, P, P, I, VP, S, VP]
    lib.cc_ladder_ov3_gs.restype = I
    lib.cc_ladder_ov3_es_abci.argtypes = [I, I, I, P, P, P, P, P, P, I, VP, S, VP]
    lib.cc_ladder_ov3_es_abci.restype = I
    lib.cc_ladder_set_tuning.argtypes = [I, I]
    lib.cc_ladder_set_tuning.restype = I
    lib.cc_ladder_profile.argtypes = [I]
    lib.cc_ladder_profile.restype = None
    lib.cc_ladder_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_double)]
    lib.cc_ladder_profile_read.restype = I
    _lib = lib
    return lib


EXPORTS = (
    "cc_ladder_workspace_size", "cc_ladder_residual", "cc_ladder_density",
    "cc_ladder_lagrangian", "cc_ladder_step", "cc_ladder_update", "cc_ladder_status",
    "cc_ladder_debug_wait", "cc_ladder_strerror", "cc_ladder_launch_count",
    "cc_ladder_profile", "cc_ladder_profile_read", "cc_ladder_lagrangian_noalloc",
    "cc_ladder_residual_adjoint", "cc_ladder_set_tuning", "cc_ladder_t1_transform",
    "cc_ladder_w_backtransform", "cc_ladder_density_es", "cc_ladder_mp2_driver_workspace_size",
    "cc_ladder_mp2_driver", "cc_ladder_iterate_workspace_size", "cc_ladder_iterate",
    "cc_ladder_ov3_workspace_size", "cc_ladder_ov3_gs", "cc_ladder_ov3_es_abci",
)


@dataclass
class System:
    """One closed-shell system; tensors are float64 and C-contiguous."""
    L_vv: torch.Tensor                 # [nj, v, v]
    t2: torch.Tensor                   # [o, o, v, v]
    t1: Optional[torch.Tensor] = None  # [o, v]
    tbar2: Optional[torch.Tensor] = None
    eps: Optional[torch.Tensor] = None

    @property
    def o(self):
        return int(self.t2.shape[0])

    @property
    def v(self):
        return int(self.t2.shape[2])

    @property
    def nj(self):
        return int(self.L_vv.shape[0])

    def c_struct(self) -> cc_ladder_system:
        def ptr(t):
            if t is None:
                return None
            if t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("ladder tensors must be contiguous float64")
            if not t.is_cuda:
                raise ValueError("ladder tensors must live on the GPU (the kernels read device memory)")
            return t.data_ptr()
        return cc_ladder_system(self.o, self.v, self.nj, ptr(self.L_vv), ptr(self.t1),
                                ptr(self.t2), ptr(self.tbar2), ptr(self.eps))


def _arr(systems: Sequence[System]):
    arr = (cc_ladder_system * len(systems))()
    for k, s in enumerate(systems):
        arr[k] = s.c_struct()
    return arr


def _ptrs(ts):
    for t in ts:
        if t.dtype != torch.float64 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("output and amplitude buffers must be contiguous float64 GPU tensors")
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int):
    if rc != 0:
        raise LadderError(rc, load().cc_ladder_strerror(rc).decode())


def _prec(p):
    return CC_PREC[p] if isinstance(p, str) else int(p)


def cc_ladder_workspace_size(systems: Sequence[System], prec="mixed", which=CC_WS_STEP) -> int:
    lib = load()
    return int(lib.cc_ladder_workspace_size(_arr(systems), len(systems), _prec(prec), which))


def workspace(systems: Sequence[System], prec="mixed", which=CC_WS_STEP, device=None) -> torch.Tensor:
    n = cc_ladder_workspace_size(systems, prec, which)
    if n == 0:
        raise LadderError(-1, "invalid systems for workspace sizing")
    dev = device or systems[0].L_vv.device
    return torch.empty(n, dtype=torch.uint8, device=dev)


def _ws(systems, prec, which, ws):
    if ws is None:
        ws = workspace(systems, prec, which)
    if not ws.is_cuda:
        raise ValueError("the workspace must be GPU memory")
    return ws


def cc_ladder_residual(systems, prec="mixed", ws=None, out=None, stream=None):
    lib = load()
    ws = _ws(systems, prec, CC_WS_RESIDUAL, ws)
    out = out or [torch.empty_like(s.t2) for s in systems]
    _check(lib.cc_ladder_residual(_arr(systems), len(systems), _ptrs(out), _prec(prec),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def cc_ladder_residual_adjoint(systems, prec="mixed", ws=None, out=None, stream=None):
    """dE/dtau_ij^cd = sum_ab tbar_ij^ab g_acbd (the adjoint ladder), one buffer per system."""
    lib = load()
    ws = _ws(systems, prec, CC_WS_RESIDUAL, ws)
    out = out or [torch.empty_like(s.t2) for s in systems]
    _check(lib.cc_ladder_residual_adjoint(_arr(systems), len(systems), _ptrs(out), _prec(prec),
                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def cc_ladder_density(systems, prec="mixed", ws=None, out=None, stream=None):
    lib = load()
    ws = _ws(systems, prec, CC_WS_DENSITY, ws)
    out = out or [torch.empty_like(s.L_vv) for s in systems]
    _check(lib.cc_ladder_density(_arr(systems), len(systems), _ptrs(out), _prec(prec),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def cc_ladder_density_es(systems, R2, R0, prec="mixed", ws=None, out=None, stream=None):
    """Excited-state density: D with U = R0 * t2 + R2 in place of tau (tbar2 = left doubles L2)."""
    if len(R2) != len(systems) or len(R0) != len(systems):
        raise ValueError("one R2 buffer and one R0 value per system")
    for s_, r in zip(systems, R2):
        if tuple(r.shape) != tuple(s_.t2.shape):
            raise ValueError("R2 must have the shape of t2")
    lib = load()
    ws = _ws(systems, prec, CC_WS_DENSITY, ws)
    out = out or [torch.empty_like(s.L_vv) for s in systems]
    r0 = (ctypes.c_double * len(systems))(*[float(x) for x in R0])
    for r in R2:
        _f64(r, "R2")
    _check(lib.cc_ladder_density_es(_arr(systems), len(systems), _ptrs(R2), r0, _ptrs(out), _prec(prec),
                                    ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def cc_ladder_lagrangian(systems, omega=None, prec="mixed", ws=None, E=None, stream=None):
    lib = load()
    ws = _ws(systems, prec, CC_WS_LAGRANGIAN, ws)
    if E is None:
        E = torch.empty(len(systems), dtype=torch.float64, device=systems[0].L_vv.device)
    om = _ptrs(omega) if omega is not None else None
    _check(lib.cc_ladder_lagrangian(_arr(systems), len(systems), ctypes.c_void_p(E.data_ptr()), om,
                                    _prec(prec), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                    _stream(stream)))
    return E


def cc_ladder_lagrangian_noalloc(systems, omega, E=None, stream=None):
    """E = sum tbar2 * Omega with no workspace and no device allocation (see the C header)."""
    lib = load()
    if E is None:
        E = torch.empty(len(systems), dtype=torch.float64, device=systems[0].L_vv.device)
    _check(lib.cc_ladder_lagrangian_noalloc(_arr(systems), len(systems), ctypes.c_void_p(E.data_ptr()),
                                            _ptrs(omega), _stream(stream)))
    return E


def cc_ladder_step(systems, prec="mixed", ws=None, omega=None, D=None, E=None, stream=None):
    lib = load()
    ws = _ws(systems, prec, CC_WS_STEP, ws)
    omega = omega or [torch.empty_like(s.t2) for s in systems]
    D = D or [torch.empty_like(s.L_vv) for s in systems]
    if E is None:
        E = torch.empty(len(systems), dtype=torch.float64, device=systems[0].L_vv.device)
    _check(lib.cc_ladder_step(_arr(systems), len(systems), _ptrs(omega), _ptrs(D),
                              ctypes.c_void_p(E.data_ptr()), _prec(prec),
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return omega, D, E


def cc_ladder_update(systems, omega, out=None, stream=None):
    lib = load()
    out = out or [torch.empty_like(s.t2) for s in systems]
    _check(lib.cc_ladder_update(_arr(systems), len(systems), _ptrs(omega), _ptrs(out), _stream(stream)))
    return out


def cc_ladder_status(ws, stream=None) -> int:
    return int(load().cc_ladder_status(ctypes.c_void_p(ws.data_ptr()), _stream(stream)))


def cc_ladder_debug_wait(flag: torch.Tensor, timeout_ns: int, ws, stream=None):
    _check(load().cc_ladder_debug_wait(ctypes.c_void_p(flag.data_ptr()), int(timeout_ns),
                                       ctypes.c_void_p(ws.data_ptr()), _stream(stream)))


def cc_ladder_launch_count() -> int:
    return int(load().cc_ladder_launch_count())


def cc_ladder_strerror(code: int) -> str:
    return load().cc_ladder_strerror(int(code)).decode()


def cc_ladder_profile(enable: bool):
    load().cc_ladder_profile(1 if enable else 0)


def cc_ladder_profile_read():
    """(contraction ms, contraction launches, padded contraction flops) since the last read."""
    ms, n, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(load().cc_ladder_profile_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
    return ms.value, n.value, fl.value


def _f64(t, name):
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on the GPU (the kernels read device memory)")
    return ctypes.c_void_p(t.data_ptr())


def cc_ladder_t1_transform(L_vv, L_ov, t1, out=None, stream=None):
    """vv block of the T1-transformed Cholesky vectors: L_vv - t1^T L_ov per J."""
    nj, v, _ = L_vv.shape
    o = t1.shape[0]
    out = torch.empty_like(L_vv) if out is None else out
    _check(load().cc_ladder_t1_transform(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(t1, "t1"),
                                         _f64(out, "out"), _stream(stream)))
    return out


def cc_ladder_w_backtransform(W_vv, t1, out=None, stream=None):
    """ov block of x^T W y for a vv-only W: -t1 W per J."""
    nj, v, _ = W_vv.shape
    o = t1.shape[0]
    out = torch.empty((nj, o, v), dtype=torch.float64, device=W_vv.device) if out is None else out
    _check(load().cc_ladder_w_backtransform(o, v, nj, _f64(W_vv, "W_vv"), _f64(t1, "t1"), _f64(out, "out"),
                                            _stream(stream)))
    return out


def cc_ladder_mp2_driver(L_ov, prec="mixed", ws=None, out=None, stream=None):
    """g[i, j, a, b] = sum_J L_ov[J, i, a] L_ov[J, j, b] (the MP2-like driver)."""
    lib = load()
    nj, o, v = L_ov.shape
    n = int(lib.cc_ladder_mp2_driver_workspace_size(o, v, nj, _prec(prec)))
    if n == 0:
        raise LadderError(-1, "invalid sizes for the driver workspace")
    ws = torch.empty(n, dtype=torch.uint8, device=L_ov.device) if ws is None else ws
    out = torch.empty((o, o, v, v), dtype=torch.float64, device=L_ov.device) if out is None else out
    _check(lib.cc_ladder_mp2_driver(o, v, nj, _f64(L_ov, "L_ov"), _f64(out, "out"), _prec(prec),
                                    ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def cc_ladder_iterate(system, g_drv, n_iter, prec="mixed", ws=None, out=None, dnorm2=None, stream=None):
    """n_iter Jacobi steps of the ladder + driver doubles equations; returns (t2, sum (t' - t)^2 per step)."""
    if tuple(g_drv.shape) != tuple(system.t2.shape):
        raise ValueError("the driver must have the shape of t2")
    lib = load()
    arr = _arr([system])
    if ws is None:
        n = int(lib.cc_ladder_iterate_workspace_size(arr, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid system for the iteration workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=system.L_vv.device)
    out = torch.empty_like(system.t2) if out is None else out
    dnorm2 = torch.empty(n_iter, dtype=torch.float64, device=system.L_vv.device) if dnorm2 is None else dnorm2
    _check(lib.cc_ladder_iterate(arr, _f64(g_drv, "g_drv"), int(n_iter), _f64(out, "out"), _f64(dnorm2, "dnorm2"),
                                 _prec(prec), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out, dnorm2


def cc_ladder_ov3_gs(L_vv, L_ov, t2, tbar1, R0=1.0, prec="mixed", ws=None, stream=None):
    """Ground-state OV^3 contributions (W_vv [nj, v, v], W_ov [nj, o, v])."""
    lib = load()
    nj, o, v = L_ov.shape
    if ws is None:
        n = int(lib.cc_ladder_ov3_workspace_size(o, v, nj, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid sizes for the OV^3 workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=L_vv.device)
    W_vv = torch.empty_like(L_vv)
    W_ov = torch.empty_like(L_ov)
    _check(lib.cc_ladder_ov3_gs(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(t2, "t2"),
                                _f64(tbar1, "tbar1"), float(R0), _f64(W_vv, "W_vv"), _f64(W_ov, "W_ov"),
                                _prec(prec), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return W_vv, W_ov


def cc_ladder_ov3_es_abci(L_vv, L_ov, L2, R1, prec="mixed", ws=None, stream=None):
    """Excited-state d_abci contributions (W_vv [nj, v, v], W_vo [nj, o, v] = W_ci)."""
    lib = load()
    nj, o, v = L_ov.shape
    if ws is None:
        n = int(lib.cc_ladder_ov3_workspace_size(o, v, nj, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid sizes for the OV^3 workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=L_vv.device)
    W_vv = torch.empty_like(L_vv)
    W_vo = torch.empty_like(L_ov)
    _check(lib.cc_ladder_ov3_es_abci(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(L2, "L2"),
                                     _f64(R1, "R1"), _f64(W_vv, "W_vv"), _f64(W_vo, "W_vo"), _prec(prec),
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return W_vv, W_vo


def cc_ladder_set_tuning(block_edge: int = 0, win_kblocks: int = 0):
    """Process-wide tuning knobs (0 = default); see the C header."""
    _check(load().cc_ladder_set_tuning(int(block_edge), int(win_kblocks)))

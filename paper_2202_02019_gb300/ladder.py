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
CC_WS_RESIDUAL, CC_WS_DENSITY, CC_WS_LAGRANGIAN, CC_WS_STEP, CC_WS_BATCH = 1, 2, 4, 7, 8

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
    lib.cc_ladder_ov3_es_abic_workspace_size.argtypes = [I, I, I, I]
    lib.cc_ladder_ov3_es_abic_workspace_size.restype = S
    lib.cc_ladder_ov3_es_abic.argtypes = [I, I, I, P, P, P, P, P, ctypes.c_double, P, P, P, P, I, VP, S, VP]
    lib.cc_ladder_ov3_es_abic.restype = I
    lib.cc_ladder_pair_blocks.argtypes = [SYS, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.cc_ladder_pair_blocks.restype = I
    lib.cc_ladder_step_blocks.argtypes = [SYS, ctypes.POINTER(ctypes.c_int32), I, P, P, P, I, VP, S, VP]
    lib.cc_ladder_step_blocks.restype = I
    lib.cc_ladder_scale_by.argtypes = [P, ctypes.c_int64, ctypes.c_double, P, VP]
    lib.cc_ladder_scale_by.restype = I
    lib.cc_ladder_set_tuning.argtypes = [I, I]
    lib.cc_ladder_set_tuning.restype = I
    lib.cc_ladder_set_contraction.argtypes = [I]
    lib.cc_ladder_set_contraction.restype = I
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
    "cc_ladder_residual_adjoint", "cc_ladder_set_tuning", "cc_ladder_set_contraction", "cc_ladder_t1_transform",
    "cc_ladder_w_backtransform", "cc_ladder_density_es", "cc_ladder_mp2_driver_workspace_size",
    "cc_ladder_mp2_driver", "cc_ladder_iterate_workspace_size", "cc_ladder_iterate",
    "cc_ladder_ov3_workspace_size", "cc_ladder_ov3_gs", "cc_ladder_ov3_es_abci",
    "cc_ladder_pair_blocks", "cc_ladder_step_blocks", "cc_ladder_scale_by",
    "cc_ladder_ov3_es_abic_workspace_size", "cc_ladder_ov3_es_abic",
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
        o, v, nj = self.o, self.v, self.nj
        _shape(self.L_vv, (nj, v, v), "L_vv")
        _shape(self.t2, (o, o, v, v), "t2")
        if self.t1 is not None:
            _shape(self.t1, (o, v), "t1")
        if self.tbar2 is not None:
            _shape(self.tbar2, (o, o, v, v), "tbar2")
        if self.eps is not None:
            _shape(self.eps, (o + v,), "eps")

        def ptr(t):
            if t is None:
                return None
            return _dev_ptr(t, "ladder tensors")
        return cc_ladder_system(o, v, nj, ptr(self.L_vv), ptr(self.t1),
                                ptr(self.t2), ptr(self.tbar2), ptr(self.eps))


def _shape(t, shape, name):
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _dev_ptr(t, name):
    """Device address of a contiguous float64 tensor on the current GPU (checks in that order,
    so that shape and dtype errors are reported without touching CUDA)."""
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous float64 tensors")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on the GPU (the kernels read device memory)")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must live on the current CUDA device "
                         f"(cuda:{torch.cuda.current_device()}), not {t.device}")
    return t.data_ptr()


def _arr(systems: Sequence[System]):
    if len(systems) < 1:
        raise ValueError("at least one system")
    arr = (cc_ladder_system * len(systems))()
    for k, s in enumerate(systems):
        arr[k] = s.c_struct()
    return arr


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[_dev_ptr(t, "output and amplitude buffers") for t in ts])


def _outs(ts, systems, like, name):
    """One buffer per system, each with the shape of that system's `like` tensor (t2 or L_vv)."""
    ts = list(ts)
    if len(ts) != len(systems):
        raise ValueError(f"{name}: one buffer per system ({len(ts)} given for {len(systems)} systems)")
    for t, s in zip(ts, systems):
        _shape(t, tuple(getattr(s, like).shape), name)
    return _ptrs(ts)


def _energy(E, n):
    if E.dim() != 1 or E.numel() < n:
        raise ValueError(f"E must be a 1-D tensor of at least {n} float64 values")
    return ctypes.c_void_p(_dev_ptr(E, "E"))


def _ws_args(ws):
    """(device address, size in bytes) of a workspace tensor on the current GPU."""
    if not ws.is_contiguous():
        raise ValueError("the workspace must be a contiguous tensor")
    if not ws.is_cuda:
        raise ValueError("the workspace must be GPU memory")
    if ws.device.index != torch.cuda.current_device():
        raise ValueError(f"the workspace must live on the current CUDA device, not {ws.device}")
    return ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int):
    if rc != 0:
        raise LadderError(rc, load().cc_ladder_strerror(rc).decode())


def _prec(p):
    return CC_PREC[p] if isinstance(p, str) else int(p)


def cc_ladder_workspace_size(systems: Sequence[System], prec="mixed", which=CC_WS_STEP, batched=False) -> int:
    """Workspace bytes; batched=True sizes the batched schedule of a list of systems."""
    lib = load()
    if batched:
        which |= CC_WS_BATCH
    return int(lib.cc_ladder_workspace_size(_arr(systems), len(systems), _prec(prec), which))


def workspace(systems: Sequence[System], prec="mixed", which=CC_WS_STEP, device=None, batched=False) -> torch.Tensor:
    n = cc_ladder_workspace_size(systems, prec, which, batched)
    if n == 0:
        raise LadderError(-1, "invalid systems for workspace sizing")
    dev = device or systems[0].L_vv.device
    return torch.empty(n, dtype=torch.uint8, device=dev)


def _ws(systems, prec, which, ws):
    if ws is None:
        ws = workspace(systems, prec, which)
    return ws


def cc_ladder_residual(systems, prec="mixed", ws=None, out=None, stream=None):
    lib = load()
    arr = _arr(systems)
    out = out or [torch.empty_like(s.t2) for s in systems]
    po = _outs(out, systems, "t2", "Omega")
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_RESIDUAL, ws))
    _check(lib.cc_ladder_residual(arr, len(systems), po, _prec(prec), wp, wn, _stream(stream)))
    return out


def cc_ladder_residual_adjoint(systems, prec="mixed", ws=None, out=None, stream=None):
    """dE/dtau_ij^cd = sum_ab tbar_ij^ab g_acbd (the adjoint ladder), one buffer per system."""
    lib = load()
    arr = _arr(systems)
    out = out or [torch.empty_like(s.t2) for s in systems]
    po = _outs(out, systems, "t2", "dE/dtau")
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_RESIDUAL, ws))
    _check(lib.cc_ladder_residual_adjoint(arr, len(systems), po, _prec(prec), wp, wn, _stream(stream)))
    return out


def cc_ladder_density(systems, prec="mixed", ws=None, out=None, stream=None):
    lib = load()
    arr = _arr(systems)
    out = out or [torch.empty_like(s.L_vv) for s in systems]
    po = _outs(out, systems, "L_vv", "D")
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_DENSITY, ws))
    _check(lib.cc_ladder_density(arr, len(systems), po, _prec(prec), wp, wn, _stream(stream)))
    return out


def cc_ladder_density_es(systems, R2, R0, prec="mixed", ws=None, out=None, stream=None):
    """Excited-state density: D with U = R0 * t2 + R2 in place of tau (tbar2 = left doubles L2)."""
    if len(R2) != len(systems) or len(R0) != len(systems):
        raise ValueError("one R2 buffer and one R0 value per system")
    lib = load()
    arr = _arr(systems)
    pr2 = _outs(R2, systems, "t2", "R2")
    out = out or [torch.empty_like(s.L_vv) for s in systems]
    po = _outs(out, systems, "L_vv", "D")
    r0 = (ctypes.c_double * len(systems))(*[float(x) for x in R0])
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_DENSITY, ws))
    _check(lib.cc_ladder_density_es(arr, len(systems), pr2, r0, po, _prec(prec), wp, wn, _stream(stream)))
    return out


def cc_ladder_lagrangian(systems, omega=None, prec="mixed", ws=None, E=None, stream=None):
    lib = load()
    arr = _arr(systems)
    om = _outs(omega, systems, "t2", "Omega") if omega is not None else None
    if E is None:
        E = torch.empty(len(systems), dtype=torch.float64, device=systems[0].L_vv.device)
    pe = _energy(E, len(systems))
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_LAGRANGIAN, ws))
    _check(lib.cc_ladder_lagrangian(arr, len(systems), pe, om, _prec(prec), wp, wn, _stream(stream)))
    return E


def cc_ladder_lagrangian_noalloc(systems, omega, E, stream=None):
    """E = sum tbar2 * Omega with no workspace and no device allocation (see the C header).
    E is the caller's device buffer of at least len(systems) float64 values: this wrapper
    allocates nothing either."""
    lib = load()
    arr = _arr(systems)
    om = _outs(omega, systems, "t2", "Omega")
    _check(lib.cc_ladder_lagrangian_noalloc(arr, len(systems), _energy(E, len(systems)), om, _stream(stream)))
    return E


def cc_ladder_step(systems, prec="mixed", ws=None, omega=None, D=None, E=None, stream=None):
    lib = load()
    arr = _arr(systems)
    omega = omega or [torch.empty_like(s.t2) for s in systems]
    D = D or [torch.empty_like(s.L_vv) for s in systems]
    if E is None:
        E = torch.empty(len(systems), dtype=torch.float64, device=systems[0].L_vv.device)
    po, pd, pe = _outs(omega, systems, "t2", "Omega"), _outs(D, systems, "L_vv", "D"), _energy(E, len(systems))
    wp, wn = _ws_args(_ws(systems, prec, CC_WS_STEP, ws))
    _check(lib.cc_ladder_step(arr, len(systems), po, pd, pe, _prec(prec), wp, wn, _stream(stream)))
    return omega, D, E


def cc_ladder_pair_blocks(system):
    """(number of pair blocks, block edge) of one system under the current tuning (host only)."""
    cnt, edge = ctypes.c_int32(), ctypes.c_int32()
    _check(load().cc_ladder_pair_blocks(_arr([system]), ctypes.byref(cnt), ctypes.byref(edge)))
    return cnt.value, edge.value


def cc_ladder_step_blocks(system, blocks, prec="mixed", ws=None, omega=None, D=None, E=None, stream=None):
    """One shard of a system's step: Omega for the pairs of the listed pair blocks (written into
    `omega`, other entries untouched), their partial D and partial E (see the C header)."""
    lib = load()
    blocks = [int(b) for b in blocks]
    if not blocks:
        raise ValueError("a shard needs at least one pair block")
    arr = _arr([system])
    omega = torch.empty_like(system.t2) if omega is None else omega
    D = torch.empty_like(system.L_vv) if D is None else D
    E = torch.empty(1, dtype=torch.float64, device=system.L_vv.device) if E is None else E
    po = _outs([omega], [system], "t2", "Omega")
    pd = _outs([D], [system], "L_vv", "D")
    pe = _energy(E, 1)
    wp, wn = _ws_args(_ws([system], prec, CC_WS_STEP, ws))
    bl = (ctypes.c_int32 * len(blocks))(*blocks)
    _check(lib.cc_ladder_step_blocks(arr, bl, len(blocks), ctypes.c_void_p(po[0]), ctypes.c_void_p(pd[0]), pe,
                                     _prec(prec), wp, wn, _stream(stream)))
    return omega, D, E


def cc_ladder_scale_by(x, factor, g=None, stream=None):
    """x *= factor * g (g: a float64 device scalar tensor, or None), in the library; returns x."""
    gp = None
    if g is not None:
        if g.numel() != 1:
            raise ValueError("g must hold one value")
        gp = ctypes.c_void_p(_dev_ptr(g.reshape(1), "g"))
    _check(load().cc_ladder_scale_by(ctypes.c_void_p(_dev_ptr(x, "x")), x.numel(), float(factor), gp,
                                     _stream(stream)))
    return x


def cc_ladder_update(systems, omega, out=None, stream=None):
    lib = load()
    arr = _arr(systems)
    pom = _outs(omega, systems, "t2", "Omega")
    out = out or [torch.empty_like(s.t2) for s in systems]
    po = _outs(out, systems, "t2", "t2_out")
    _check(lib.cc_ladder_update(arr, len(systems), pom, po, _stream(stream)))
    return out


def cc_ladder_status(ws, stream=None) -> int:
    return int(load().cc_ladder_status(_ws_args(ws)[0], _stream(stream)))


def cc_ladder_debug_wait(flag: torch.Tensor, timeout_ns: int, ws, stream=None):
    if flag.dtype != torch.int32 or not flag.is_cuda:
        raise ValueError("the flag must be an int32 GPU tensor")
    _check(load().cc_ladder_debug_wait(ctypes.c_void_p(flag.data_ptr()), int(timeout_ns),
                                       _ws_args(ws)[0], _stream(stream)))


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
    return ctypes.c_void_p(_dev_ptr(t, name))


def cc_ladder_t1_transform(L_vv, L_ov, t1, out=None, stream=None):
    """vv block of the T1-transformed Cholesky vectors: L_vv - t1^T L_ov per J."""
    nj, v, _ = L_vv.shape
    o = t1.shape[0]
    _shape(L_vv, (nj, v, v), "L_vv")
    _shape(L_ov, (nj, o, v), "L_ov")
    _shape(t1, (o, v), "t1")
    out = torch.empty_like(L_vv) if out is None else out
    _shape(out, (nj, v, v), "out")
    _check(load().cc_ladder_t1_transform(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(t1, "t1"),
                                         _f64(out, "out"), _stream(stream)))
    return out


def cc_ladder_w_backtransform(W_vv, t1, out=None, stream=None):
    """ov block of x^T W y for a vv-only W: -t1 W per J."""
    nj, v, _ = W_vv.shape
    o = t1.shape[0]
    _shape(W_vv, (nj, v, v), "W_vv")
    _shape(t1, (o, v), "t1")
    out = torch.empty((nj, o, v), dtype=torch.float64, device=W_vv.device) if out is None else out
    _shape(out, (nj, o, v), "out")
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
    _shape(out, (o, o, v, v), "out")
    _check(lib.cc_ladder_mp2_driver(o, v, nj, _f64(L_ov, "L_ov"), _f64(out, "out"), _prec(prec),
                                    *_ws_args(ws), _stream(stream)))
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
    _shape(out, tuple(system.t2.shape), "out")
    dnorm2 = torch.empty(n_iter, dtype=torch.float64, device=system.L_vv.device) if dnorm2 is None else dnorm2
    if dnorm2.dim() != 1 or dnorm2.numel() < n_iter:
        raise ValueError(f"dnorm2 must hold at least n_iter = {n_iter} values")
    _check(lib.cc_ladder_iterate(arr, _f64(g_drv, "g_drv"), int(n_iter), _f64(out, "out"), _f64(dnorm2, "dnorm2"),
                                 _prec(prec), *_ws_args(ws), _stream(stream)))
    return out, dnorm2


def cc_ladder_ov3_gs(L_vv, L_ov, t2, tbar1, R0=1.0, prec="mixed", ws=None, stream=None):
    """Ground-state OV^3 contributions (W_vv [nj, v, v], W_ov [nj, o, v])."""
    lib = load()
    nj, o, v = L_ov.shape
    _shape(L_vv, (nj, v, v), "L_vv")
    _shape(t2, (o, o, v, v), "t2")
    _shape(tbar1, (o, v), "tbar1")
    if ws is None:
        n = int(lib.cc_ladder_ov3_workspace_size(o, v, nj, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid sizes for the OV^3 workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=L_vv.device)
    W_vv = torch.empty_like(L_vv)
    W_ov = torch.empty_like(L_ov)
    _check(lib.cc_ladder_ov3_gs(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(t2, "t2"),
                                _f64(tbar1, "tbar1"), float(R0), _f64(W_vv, "W_vv"), _f64(W_ov, "W_ov"),
                                _prec(prec), *_ws_args(ws), _stream(stream)))
    return W_vv, W_ov


def cc_ladder_ov3_es_abci(L_vv, L_ov, L2, R1, prec="mixed", ws=None, stream=None):
    """Excited-state d_abci contributions (W_vv [nj, v, v], W_vo [nj, o, v] = W_ci)."""
    lib = load()
    nj, o, v = L_ov.shape
    _shape(L_vv, (nj, v, v), "L_vv")
    _shape(L2, (o, o, v, v), "L2")
    _shape(R1, (o, v), "R1")
    if ws is None:
        n = int(lib.cc_ladder_ov3_workspace_size(o, v, nj, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid sizes for the OV^3 workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=L_vv.device)
    W_vv = torch.empty_like(L_vv)
    W_vo = torch.empty_like(L_ov)
    _check(lib.cc_ladder_ov3_es_abci(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(L2, "L2"),
                                     _f64(R1, "R1"), _f64(W_vv, "W_vv"), _f64(W_vo, "W_vo"), _prec(prec),
                                     *_ws_args(ws), _stream(stream)))
    return W_vv, W_vo


def cc_ladder_ov3_es_abic(L_vv, L_ov, tbar1, L2, t2, R0, R1, R2, prec="mixed", ws=None, stream=None):
    """Excited-state d_abic contributions (W_vv [nj, v, v], W_ov [nj, o, v]); see the C header."""
    lib = load()
    nj, o, v = L_ov.shape
    _shape(L_vv, (nj, v, v), "L_vv")
    _shape(tbar1, (o, v), "tbar1")
    _shape(R1, (o, v), "R1")
    for t, n in ((L2, "L2"), (t2, "t2"), (R2, "R2")):
        _shape(t, (o, o, v, v), n)
    if ws is None:
        n = int(lib.cc_ladder_ov3_es_abic_workspace_size(o, v, nj, _prec(prec)))
        if n == 0:
            raise LadderError(-1, "invalid sizes for the OV^3 workspace")
        ws = torch.empty(n, dtype=torch.uint8, device=L_vv.device)
    W_vv = torch.empty_like(L_vv)
    W_ov = torch.empty_like(L_ov)
    _check(lib.cc_ladder_ov3_es_abic(o, v, nj, _f64(L_vv, "L_vv"), _f64(L_ov, "L_ov"), _f64(tbar1, "tbar1"),
                                     _f64(L2, "L2"), _f64(t2, "t2"), float(R0), _f64(R1, "R1"), _f64(R2, "R2"),
                                     _f64(W_vv, "W_vv"), _f64(W_ov, "W_ov"), _prec(prec), *_ws_args(ws),
                                     _stream(stream)))
    return W_vv, W_ov


def cc_ladder_set_tuning(block_edge: int = 0, win_kblocks: int = 0):
    """Process-wide tuning knobs (0 = default); see the C header."""
    _check(load().cc_ladder_set_tuning(int(block_edge), int(win_kblocks)))


CC_KERNEL_SINGLE, CC_KERNEL_PAIR, CC_KERNEL_KBLOCK_WINDOWS, CC_KERNEL_PAIR_KBLOCK_WINDOWS = 1, 2, 3, 4


def cc_ladder_set_contraction(kind: int = 0):
    """Contraction kernel of the split paths, process-wide: 0 default, CC_KERNEL_SINGLE
    (one CTA per 128 x 128 tile), CC_KERNEL_PAIR (two-CTA cluster per 256 x 128 tile) or
    CC_KERNEL_KBLOCK_WINDOWS (one window per 64-term k-block, three window buffers) or
    CC_KERNEL_PAIR_KBLOCK_WINDOWS (both)."""
    _check(load().cc_ladder_set_contraction(int(kind)))

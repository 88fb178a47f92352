"""Autotuner for the ladder library's tuning knobs.

The pair-block edge s (virtual rows per block) sets the size of every
tensor-core contraction of a block (M = s*v for the g-build and D, M = s^2
pairs for the ladder and Gamma) and the scratch footprint (~s^2 v^2); the
leading-product window sets how often the split paths restart their
truncating FP32 accumulator (accuracy vs drain work); the contraction kernel
is the windowed single-CTA kernel or the one-window-per-k-block kernel (a
64-term window whatever the window knob says).  For a list of systems the
tuner times each candidate (block, window, kernel) on the caller's own inputs
with CUDA events and keeps the fastest one whose window does not exceed
``max_win`` (the accuracy cap: windows above 4 k-blocks are not offered),
then caches the choice per (precision, shapes) in a JSON file.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional, Sequence, Tuple

import torch

from . import ladder as lad

_S, _K = lad.CC_KERNEL_SINGLE, lad.CC_KERNEL_KBLOCK_WINDOWS
DEFAULT_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (48, 4, _S), (32, 4, _S), (64, 4, _S), (48, 2, _S), (32, 2, _S), (48, 0, _K), (32, 0, _K), (64, 0, _K))


def _apply(b: int, w: int, k: int) -> None:
    lad.cc_ladder_set_tuning(b, w)
    lad.cc_ladder_set_contraction(k)


def cache_path() -> str:
    p = os.environ.get("CC_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "ccladder_tune.json")


def _key(systems: Sequence[lad.System], prec) -> str:
    shapes = ",".join(f"{s.o}x{s.v}x{s.nj}" for s in systems)
    return f"{prec}|{shapes}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(systems: Sequence[lad.System], prec="mixed", candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
         reps: int = 1, max_win: int = 4, use_cache: bool = True, path: Optional[str] = None):
    """Pick (block_edge, win_kblocks) for these systems, apply it, return
    {"block": b, "win": w, "ms": t, "source": "cache"|"measured", "tried": [...]}."""
    path = path or cache_path()
    key = _key(systems, prec)
    cache = _load(path) if use_cache else {}
    if key in cache:
        c = dict(cache[key])
        c.setdefault("kernel", 0)
        _apply(c["block"], c["win"], c["kernel"])
        return dict(c, source="cache")
    dev = systems[0].L_vv.device
    om = [torch.empty_like(s.t2) for s in systems]
    D = [torch.empty_like(s.L_vv) for s in systems]
    E = torch.empty(len(systems), dtype=torch.float64, device=dev)
    tried = []
    best = None
    for cand in candidates:
        b, w, k = (tuple(cand) + (0,))[:3]   # (block, window) pairs keep the default kernel
        if w > max_win:
            continue
        vmax = max(s.v for s in systems)
        if b > ((vmax + 3) // 4) * 4 and b != 32:
            continue  # blocks wider than the system add nothing
        _apply(b, w, k)
        need = lad.cc_ladder_workspace_size(systems, prec, lad.CC_WS_STEP)
        free, _ = torch.cuda.mem_get_info(dev)
        if need == 0 or need > 0.9 * free:
            tried.append({"block": b, "win": w, "kernel": k, "ms": None, "skipped": "workspace"})
            continue
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            lad.cc_ladder_step(systems, prec=prec, ws=ws, omega=om, D=D, E=E)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if lad.cc_ladder_status(ws) != 0:
            ms = float("inf")
        tried.append({"block": b, "win": w, "kernel": k, "ms": ms})
        if best is None or ms < best[0]:
            best = (ms, b, w, k)
        del ws
    if best is None:
        _apply(0, 0, 0)
        return {"block": 0, "win": 0, "kernel": 0, "ms": None, "source": "default", "tried": tried}
    ms, b, w, k = best
    _apply(b, w, k)
    res = {"block": b, "win": w, "kernel": k, "ms": ms, "tried": tried}
    if use_cache:
        cache = _load(path)
        cache[key] = {"block": b, "win": w, "kernel": k, "ms": ms}
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(res, source="measured")

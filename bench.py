"""Benchmark of the CD-CCSD vvvv ladder hot path (Omega + D^J + E) on GB300.

One step = one cc_ladder_step call: the ladder residual Omega, the
three-index density D^J and the Lagrangian E of one retinal-scale system
(o=78, v=650, N_J=4000) in the mixed (split-BF16 tensor-core) path, with
inputs already resident in HBM.  The metric is useful TFLOP/s, counted with
the packed (+-) algorithm's flop formula

    F = 2 P+ v^2 N_J + 4 (P+^2 Q+ + P-^2 Q-) + 2 v^4 N_J,
    P+- = v(v+-1)/2, Q+- = o(o+-1)/2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--split]
Under torchrun each rank runs its own system (weak scaling, no collective on
the data path); value = N * F / (max over ranks of the step time).  With
--split the ranks share one system: each runs its LPT share of the pair
blocks (cc_ladder_step_blocks), the partial D meet in one NCCL
reduce-scatter and E in one all-reduce; value = F / (max step time).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (o, v, nj, lam_scale)
    "retinal": (78, 650, 4000, 700.0),
    "small": (24, 180, 900, 150.0),
    "grad": (30, 250, 1200, 200.0),
}
METRIC = "ladder Omega + D^J useful TFLOP/s (mixed-precision path), o78/v650/NJ4000"
# products per useful product and the arithmetic each --prec runs in
PREC = {
    "mixed": (6, "bf16x3 split (FP32 accumulate, FP64 reductions)"),
    "fp16x2": (3, "fp16x2 scaled split (FP32 accumulate, FP64 reductions)"),
    "fp64": (1, "f64 (DMMA)"),
}


# DRAM bytes of the contraction kernel per step (sum of dram__bytes_read.sum + dram__bytes_write.sum over its
# launches of one step) from one-pass ncu captures of this kernel version; null for combinations not captured
TRAFFIC = {
    ("retinal", "mixed"): (2.718e13, "dram__bytes_read.sum + dram__bytes_write.sum over the 420 launches of one "
                                     "retinal-scale step, persistent grouped kernel (queue-pulled 128x128 tiles)"),
}


def counted_flops(o, v, nj):
    pvp, pvm = v * (v + 1) // 2, v * (v - 1) // 2
    qop, qom = o * (o + 1) // 2, o * (o - 1) // 2
    return 2.0 * pvp * v * v * nj + 4.0 * (pvp * pvp * qop + pvm * pvm * qom) + 2.0 * float(v) ** 4 * nj


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return {"bf16": float(d.get("bf16_tflops")), "bf16_sustained": float(d.get("bf16_tflops_sustained")),
                    "hbm": float(d.get("hbm_gbs")), "source": "measured"}
        except Exception:
            pass
    return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "fallback"}


def dgemm_peak(torch, n=8192, reps=5):
    """FP64 tensor-core peak of this GPU, measured here: cuBLAS DGEMM n^3 (torch.matmul, float64),
    best of `reps` after one warm-up, CUDA events.  TFLOP/s."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "power_w_median": statistics.median(pw) if pw else None,
                "samples": len(rows)}


def host_cores():
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count()
    return n


# ---------------------------------------------------------------------------
# oracle leg (CPU): bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(h, rows, cols):
    """Time the FP64 oracle on Omega[:, :, a, cols] and D[:, a, cols] for a in rows."""
    import oracle as O
    t0 = time.perf_counter()
    tt = O.tau(h["t1"], h["t2"])
    om = O.residual_rows(h["L_vv"], tt, rows, cols)
    D = O.density_rows(h["L_vv"], h["tbar2"], tt, rows, cols)
    return time.perf_counter() - t0, om, D


def sample_spec(v, block=48, n_cols=8, seed=2202):
    """One seeded virtual row per pair-block band (rows block*k .. block*k + block - 1) and a seeded
    spread of n_cols columns: every band of the pair-block sequence is sampled."""
    import numpy as np
    rng = np.random.default_rng(seed)
    rows = [int(rng.integers(lo, min(lo + block, v))) for lo in range(0, v, block)]
    cols = sorted(np.random.default_rng(seed + 1).choice(v, size=min(n_cols, v), replace=False).tolist())
    return rows, cols


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import torch
    from paper_2202_02019_gb300 import synth
    o, v, nj, lam = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    d = synth.make_pair_torch(o, v, nj, lam, seed=2202, device=dev)
    h = {k: d[k].cpu().numpy() for k in ("L_vv", "t1", "t2", "tbar2")}
    del d
    rows, cols = sample_spec(v)
    F = counted_flops(o, v, nj)
    frac = len(rows) * len(cols) / float(v * v)
    for _ in range(args.warmup):
        oracle_sample(h, rows[:1], cols[:8])
    times = []
    for _ in range(args.steps):
        t, _, _ = oracle_sample(h, rows, cols)
        times.append(t)
    t = statistics.mean(times)
    val = F * frac / t / 1e12
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} o={o} v={v} nj={nj}", "sample": f"rows {rows} x cols {len(cols)}"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"Omega[:,:,a,b] and D[:,a,c] for a in {rows}, {len(cols)} b/c columns "
                                   f"({frac:.2e} of the outputs), credited F*{frac:.2e}"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def rel(a, b):
    import numpy as np
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fp64_vs_mixed_small(lad, synth, torch):
    """Both paths on the small single-system config (o=24, v=180, N_J=900)."""
    import numpy as np
    import oracle as O
    o, v, nj, lam = WORKLOADS["small"]
    s, tb1, tb2 = synth.make_pair(o, v, nj, lam, seed=2202)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sd = lad.System(L_vv=t(s.L_vv), t2=t(s.t2), t1=t(s.t1), tbar2=t(tb2), eps=t(s.eps))
    res = {"workload": f"small o={o} v={v} nj={nj}"}
    rows, cols = [0, v // 2, v - 1], list(range(0, v, 6))
    tt = O.tau(s.t1, s.t2)
    om_ref = O.residual_rows(s.L_vv, tt, rows)
    D_ref = O.density_rows(s.L_vv, tb2, tt, rows)
    F = counted_flops(o, v, nj)
    outs = {}
    for prec in ("mixed", "fp16x2", "fp64"):
        ws = lad.workspace([sd], prec)
        om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        om, D, E = lad.cc_ladder_step([sd], prec=prec, ws=ws, omega=om, D=D, E=E)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        outs[prec] = (om[0], D[0], float(E[0]))
        res[prec] = {"ms": ms, "tflops": F / (ms * 1e-3) / 1e12,
                     "rel_err_omega_vs_oracle_rows": rel(om[0][:, :, rows, :].cpu(), om_ref),
                     "rel_err_D_vs_oracle_rows": rel(D[0][:, rows, :].cpu(), D_ref)}
        del ws
    om64, D64, E64 = outs["fp64"]
    omm, Dm, Em = outs["mixed"]
    res["mixed_vs_fp64"] = {"rel_err_omega": rel(omm.cpu(), om64.cpu()), "rel_err_D": rel(Dm.cpu(), D64.cpu()),
                            "rel_err_E": abs(Em - E64) / abs(E64)}
    res["speedup_mixed_over_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    o16 = outs["fp16x2"]
    res["fp16x2_vs_fp64"] = {"rel_err_omega": rel(o16[0].cpu(), om64.cpu()), "rel_err_D": rel(o16[1].cpu(), D64.cpu()),
                             "rel_err_E": abs(o16[2] - E64) / abs(E64)}
    return res


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2202_02019_gb300 import ladder as lad
    from paper_2202_02019_gb300 import shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lad.load()
    o, v, nj, lam = WORKLOADS[args.workload]
    F = counted_flops(o, v, nj)
    split = args.split and world > 1
    # weak scaling: every rank its own system; --split: one system, its pair blocks dealt over the ranks
    d = synth.make_pair_torch(o, v, nj, lam, seed=2202 + (0 if args.split else 17 * rank), device="cuda")
    sd = lad.System(L_vv=d["L_vv"], t2=d["t2"], t1=d["t1"], tbar2=d["tbar2"], eps=d["eps"])
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ws = lad.workspace([sd], args.prec)
    om = [torch.empty_like(sd.t2)]
    D = [torch.empty_like(sd.L_vv)]
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    mine = shard.rank_blocks(sd, rank, world) if split else None

    def step():
        if not split:
            lad.cc_ladder_step([sd], prec=args.prec, ws=ws, omega=om, D=D, E=E, stream=stream)
            return
        # this rank's pair blocks, then D summed by one reduce-scatter and E by one all-reduce
        lad.cc_ladder_step_blocks(sd, mine, prec=args.prec, ws=ws, omega=om[0], D=D[0], E=E, stream=stream)
        shard.reduce_scatter_D(D[0], world)
        dist.all_reduce(E, op=dist.ReduceOp.SUM)

    for _ in range(args.warmup):
        step()
    assert lad.cc_ladder_status(ws) == 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    lad.cc_ladder_profile(True)
    n0 = lad.cc_ladder_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = lad.cc_ladder_launch_count() - n0
    gemm_ms, gemm_n, gemm_fl = lad.cc_ladder_profile_read()
    lad.cc_ladder_profile(False)
    status = lad.cc_ladder_status(ws)
    ms = e0.elapsed_time(e1) / args.steps
    # weak: world systems of F each; split: one system of F over all ranks
    ms_max, value = shard.aggregate_step_time(ms, world, F / world if split else F)

    pk = peaks()
    gemm_ms_step = gemm_ms / args.steps
    achieved = F / (gemm_ms_step * 1e-3) / 1e12
    nprod = PREC[args.prec][0]
    if args.prec == "fp64":
        peak_useful = dgemm_peak(torch)
        basis = "cuBLAS DGEMM 8192^3 measured in this run (torch.matmul float64, best of 5)"
    else:
        # FP16 and BF16 share the dense tensor rate: the measured BF16 figure serves both
        peak_useful = pk["bf16_sustained"] / nprod
        basis = f"{pk['source']} sustained BF16 (= FP16 rate) / {nprod} products"
    traffic, traffic_src = TRAFFIC.get((args.workload, args.prec), (None, None))
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_useful, "unit": "TFLOP/s",
                "frac": achieved / peak_useful, "traffic": traffic,
                "traffic_basis": ("DRAM bytes per step (ncu, one pass): " + traffic_src) if traffic_src else None,
                "kernel": "cc_gemm_split3_tc" if args.prec != "fp64" else "cc_gemm_f64_dmma",
                "peak_basis": basis,
                "kernel_share_of_step": gemm_ms_step / ms,
                "kernel_launches_per_step": gemm_n / args.steps,
                "padded_flops_per_step": gemm_fl / args.steps}

    extra = {}
    cpu = None
    e2e = None
    if rank == 0 and world == 1 and not args.no_extras:
        # end to end through the C ABI with host buffers (pinned)
        host = {k: torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for k, x in
                (("L_vv", sd.L_vv), ("t1", sd.t1), ("t2", sd.t2), ("tbar2", sd.tbar2), ("eps", sd.eps))}
        for k in host:
            host[k].copy_(getattr(sd, k))
        h_om = torch.empty(sd.t2.shape, dtype=torch.float64, pin_memory=True)
        h_D = torch.empty(sd.L_vv.shape, dtype=torch.float64, pin_memory=True)
        h_E = torch.empty(1, dtype=torch.float64, pin_memory=True)
        # parity on a bounded sample against the oracle (uses the timed step's outputs)
        rows, cols = sample_spec(v)
        g_om = om[0][:, :, rows, :][:, :, :, cols].cpu().numpy()
        g_D = D[0][:, rows, :][:, :, cols].cpu().numpy()
        g_E = float(E[0])
        hn = {k: host[k].numpy() for k in ("L_vv", "t1", "t2", "tbar2")}
        t_or, o_om, o_D = oracle_sample(hn, rows, cols)
        frac = len(rows) * len(cols) / float(v * v)
        cpu = {"value": F * frac / t_or / 1e12, "unit": "TFLOP/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"Omega[:,:,a,b] and D[:,a,c] for a in {rows}, {len(cols)} b/c columns "
                         f"({frac:.2e} of the outputs, credited F*{frac:.2e}); {t_or:.1f} s"}
        extra["parity_sampled"] = {"rel_err_omega": rel(g_om, o_om), "rel_err_D": rel(g_D, o_D),
                                   "rows": rows, "n_cols": len(cols)}
        # Euler identity check on the full outputs: sum L.D = E
        eul = float(torch.sum(sd.L_vv * D[0]))
        extra["euler_identity_rel"] = abs(eul - g_E) / abs(g_E)
        del hn
        # e2e: H2D inputs, step, D2H outputs, all inside the timed region
        dev_in = {k: torch.empty_like(getattr(sd, k)) for k in host}
        sd2 = lad.System(**dev_in)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in host:
            dev_in[k].copy_(host[k], non_blocking=True)
        lad.cc_ladder_step([sd2], prec=args.prec, ws=ws, omega=om, D=D, E=E, stream=stream)
        h_om.copy_(om[0], non_blocking=True)
        h_D.copy_(D[0], non_blocking=True)
        h_E.copy_(E, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        h2d = sum(x.numel() * x.element_size() for x in host.values())
        d2h = h_om.numel() * 8 + h_D.numel() * 8 + 8
        e2e = {"value": F / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms": e2e_ms}
        del host, h_om, h_D, dev_in, sd2
        extra["E"] = g_E
        # the other split precision on the same system: one step, sampled parity
        alt = "fp16x2" if args.prec == "mixed" else ("mixed" if args.prec == "fp16x2" else None)
        if alt is not None:
            del ws
            torch.cuda.empty_cache()
            ws = lad.workspace([sd], alt)
            lad.cc_ladder_step([sd], prec=alt, ws=ws, omega=om, D=D, E=E, stream=stream)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            lad.cc_ladder_step([sd], prec=alt, ws=ws, omega=om, D=D, E=E, stream=stream)
            a1.record(stream)
            torch.cuda.synchronize()
            a_ms = a0.elapsed_time(a1)
            extra["other_precision"] = {
                "prec": alt, "dtype": PREC[alt][1], "ms_per_step": a_ms, "value": F / (a_ms * 1e-3) / 1e12,
                "unit": "TFLOP/s", "status": lad.cc_ladder_status(ws),
                "rel_err_omega_sampled": rel(om[0][:, :, rows, :][:, :, :, cols].cpu().numpy(), o_om),
                "rel_err_D_sampled": rel(D[0][:, rows, :][:, :, cols].cpu().numpy(), o_D),
                "E": float(E[0]), "rel_diff_E_vs_timed": abs(float(E[0]) - g_E) / abs(g_E)}
        if not args.no_small:
            del ws
            torch.cuda.empty_cache()
            extra["small_config_fp64_vs_mixed"] = fp64_vs_mixed_small(lad, synth, torch)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "strong" if split else "weak",
            "vs_baseline": None, "dtype": PREC[args.prec][1],
            "data": "synthetic (seeded device generator: MP2 amplitudes from random symmetric Cholesky vectors)",
            "config": {"workload": f"{args.workload} o={o} v={v} nj={nj}", "global_batch": world,
                       "kernel": args.kernel,
                       "parallelism": (f"one system, pair blocks dealt over {world} GPUs (LPT), D by reduce-scatter"
                                       if split else f"independent systems, one per GPU ({world})"),
                       "l2": "inputs larger than L2 (55 GB resident), no flush needed",
                       "counted_flops_per_system": F},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "device_status": status,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """24 independent systems of uneven size (o ~ U{6..40}, v ~ U{50..300}, N_J = 5v,
    lambda_J = exp(-J/12)) in one graph-captured call, against one call per system."""
    import torch
    from paper_2202_02019_gb300 import autotune
    from paper_2202_02019_gb300 import ladder as lad
    from paper_2202_02019_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lad.load()
    sizes = synth.batch_sizes(24, seed=2202)
    systems = []
    for k, (o, v, nj) in enumerate(sizes):
        d = synth.make_pair_torch(o, v, nj, 12.0, seed=2202 + 100 * k, device="cuda")
        systems.append(lad.System(L_vv=d["L_vv"], t2=d["t2"], t1=d["t1"], tbar2=d["tbar2"], eps=d["eps"]))
        del d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    F = sum(counted_flops(o, v, nj) for o, v, nj in sizes)
    tuned = (autotune.tune(systems, prec=args.prec, reps=1, use_cache=False) if args.autotune is not False
             else {"block": 0, "win": 0, "kernel": 0, "source": "default"})
    tuned.pop("tried", None)
    ws = lad.workspace(systems, args.prec, batched=True)
    om = [torch.empty_like(s.t2) for s in systems]
    D = [torch.empty_like(s.L_vv) for s in systems]
    E = torch.empty(len(systems), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def one_by_one():
        for k, sd in enumerate(systems):
            lad.cc_ladder_step([sd], prec=args.prec, ws=ws, omega=[om[k]], D=[D[k]], E=E[k:k + 1], stream=stream)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_seq = timed(one_by_one)
    ref = [x.clone() for x in om + D] + [E.clone()]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lad.cc_ladder_step(systems, prec=args.prec, ws=ws, omega=om, D=D, E=E)
    n0 = lad.cc_ladder_launch_count()
    with Clocks(0) as clk:
        ms_graph = timed(g.replay)
    same = all(torch.equal(a, b) for a, b in zip(ref, om + D + [E]))
    line = {
        "metric": "ladder Omega + D^J useful TFLOP/s, 24-system uneven batch (mixed path)",
        "value": F / (ms_graph * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 split (FP32 accumulate, FP64 reductions)",
        "data": "synthetic (seeded, device generator)",
        "config": {"workload": "batch24 o~U{6..40} v~U{50..300} nj=5v", "global_batch": 24, "kernel": args.kernel,
                   "sizes": sizes, "counted_flops": F, "tuning": tuned},
        "one_call_per_system_ms": ms_seq, "graph_over_one_by_one": ms_seq / ms_graph,
        "graph_equals_one_by_one": same, "clocks": clk.summary(),
        "device_status": lad.cc_ladder_status(ws),
    }
    print(json.dumps(line), flush=True)
    lad.cc_ladder_set_tuning(0, 0)
    return 0


def run_autograd(args):
    """Forward + backward of the differentiable ladder energy E(L, tau, tbar) at one workload
    (default the gradient case o=30, v=250, N_J=1200) in the mixed path.  Counted flops, the
    work the two passes do: the forward is one step (g-build + ladder for Omega and E, Gamma + D
    for D, which dE/dL = 2D reuses); the backward is dE/dtau (adjoint ladder: g-build + ladder),
    dE/dtbar = Omega being kept from the forward."""
    import torch
    from paper_2202_02019_gb300 import autograd as AG
    from paper_2202_02019_gb300 import ladder as lad
    from paper_2202_02019_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lad.load()
    o, v, nj, lam = WORKLOADS[args.workload]
    d = synth.make_pair_torch(o, v, nj, lam, seed=2202, device="cuda")
    tau = (d["t2"] + torch.einsum("ic,jd->ijcd", d["t1"], d["t1"])).contiguous()
    L = d["L_vv"].clone().requires_grad_(True)
    T = tau.clone().requires_grad_(True)
    B = d["tbar2"].clone().requires_grad_(True)
    pvp, pvm = v * (v + 1) // 2, v * (v - 1) // 2
    qop, qom = o * (o + 1) // 2, o * (o - 1) // 2
    f_res = 2.0 * pvp * v * v * nj + 4.0 * (pvp * pvp * qop + pvm * pvm * qom) / 2
    f_den = 4.0 * (pvp * pvp * qop + pvm * pvm * qom) / 2 + 2.0 * float(v) ** 4 * nj
    F = (f_res + f_den) + f_res

    def step():
        L.grad = T.grad = B.grad = None
        E = AG.ladder_energy(L, T, B, prec=args.prec)
        E.backward()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = lad.cc_ladder_launch_count()
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": "differentiable ladder energy: forward + backward useful TFLOP/s", "value": F / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": PREC[args.prec][1],
            "data": "synthetic (seeded device generator)",
            "config": {"workload": f"{args.workload} o={o} v={v} nj={nj}",
                       "counted_flops": {"forward": f_res + f_den, "backward": f_res}},
            "gpu_launches": (lad.cc_ladder_launch_count() - n0), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_fp64cmp(args):
    """The plain FP64 path at one workload: its useful TFLOP/s against the FP64 DGEMM peak
    measured here, and the split paths' errors against it over the full Omega, D and E."""
    import torch
    from paper_2202_02019_gb300 import ladder as lad
    from paper_2202_02019_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lad.load()
    o, v, nj, lam = WORKLOADS[args.workload]
    F = counted_flops(o, v, nj)
    d = synth.make_pair_torch(o, v, nj, lam, seed=2202, device="cuda")
    sd = lad.System(L_vv=d["L_vv"], t2=d["t2"], t1=d["t1"], tbar2=d["tbar2"], eps=d["eps"])
    peak = dgemm_peak(torch)
    res = {}

    def timed_step(prec, warm=True):
        ws = lad.workspace([sd], prec)
        om = [torch.empty_like(sd.t2)]
        D = [torch.empty_like(sd.L_vv)]
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        if warm:
            lad.cc_ladder_step([sd], prec=prec, ws=ws, omega=om, D=D, E=E)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lad.cc_ladder_step([sd], prec=prec, ws=ws, omega=om, D=D, E=E)
        e1.record()
        torch.cuda.synchronize()
        st = lad.cc_ladder_status(ws)
        del ws
        torch.cuda.empty_cache()
        return om[0], D[0], float(E[0]), e0.elapsed_time(e1), st

    def frob(a, b):
        # chunked over the leading index: no full-size temporary at the retinal size
        num = den = 0.0
        for k in range(a.shape[0]):
            num += float(torch.sum((a[k] - b[k]) ** 2))
            den += float(torch.sum(b[k] ** 2))
        return (num / den) ** 0.5

    # at the retinal size one FP64 step is about an hour of FP64 tensor work: time it cold, once
    with Clocks(0) as clk:
        om64, D64, E64, ms64, st64 = timed_step("fp64", warm=args.workload != "retinal")
    res["fp64"] = {"ms": ms64, "tflops": F / (ms64 * 1e-3) / 1e12, "status": st64}
    # each split path at its default leading-product window first, then the other distinct windows
    # (win_kblocks * 32 K terms, at least one 64-term K step, so 1 and 2 are the same window); the
    # truncation bias of the FP32 tensor-core accumulation grows with the window
    for prec, wins in (("mixed", (4, 2, 8)), ("fp16x2", (2, 4))):
        for i, win in enumerate(wins):
            lad.cc_ladder_set_tuning(0, win)
            try:
                om, D, E, ms, st = timed_step(prec)
            finally:
                lad.cc_ladder_set_tuning(0, 0)
            r = {"ms": ms, "tflops": F / (ms * 1e-3) / 1e12, "status": st, "speedup_over_fp64": ms64 / ms,
                 "rel_err_omega_vs_fp64": frob(om, om64), "rel_err_D_vs_fp64": frob(D, D64),
                 "rel_err_E_vs_fp64": abs(E - E64) / abs(E64)}
            del om, D
            if i == 0:
                res[prec] = dict(r, win_kblocks=win, by_window={})
            else:
                res[prec]["by_window"][str(win)] = r
    line = {"metric": "plain FP64 path useful TFLOP/s; split paths' errors against it (full tensors)",
            "value": res["fp64"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": PREC["fp64"][1], "data": "synthetic (seeded device generator)",
            "config": {"workload": f"{args.workload} o={o} v={v} nj={nj}", "counted_flops": F,
                       "fp64_warmup_steps": 0 if args.workload == "retinal" else 1},
            "roofline": {"bound": "tensor", "achieved": res["fp64"]["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": res["fp64"]["tflops"] / peak, "traffic": None, "kernel": "cc_gemm_f64_dmma (step)",
                         "peak_basis": "cuBLAS DGEMM 8192^3 measured in this run (torch.matmul float64, best of 5)"},
            "paths": res, "E_fp64": E64, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp16x2", "fp64"],
                    help="arithmetic of the timed path (mixed = 3-piece split-BF16)")
    ap.add_argument("--workload", default="retinal", choices=sorted(WORKLOADS) + ["batch24"])
    ap.add_argument("--autotune", action="store_true", default=None,
                    help="pick the tuning knobs (block edge, window, kernel) with the autotuner; the batch24 default")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", help="batch24: the default knobs")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, oracle sample and small-config legs")
    ap.add_argument("--no-small", action="store_true", help="skip the small-config FP64-vs-mixed leg")
    ap.add_argument("--mode", default="step", choices=["step", "autograd", "fp64cmp"],
                    help="step: the timed ladder step (default); autograd: forward + backward of E(L, tau, tbar); "
                         "fp64cmp: the FP64 path against the measured DGEMM peak, split paths' errors against it")
    ap.add_argument("--split", action="store_true",
                    help="under torchrun: one system sharded over the ranks by pair blocks (strong scaling) "
                         "instead of one system per rank (weak scaling)")
    ap.add_argument("--kernel", default="default", choices=["default", "single", "pair", "kblock", "pairkblock"],
                    help="split paths' contraction kernel: one CTA per 128x128 tile, a two-CTA cluster per "
                         "256x128 tile (tcgen05 cta_group::2), or one CTA per tile with one window per k-block")
    args = ap.parse_args()
    if args.kernel != "default" and args.impl != "reference":
        from paper_2202_02019_gb300 import ladder as lad
        lad.cc_ladder_set_contraction({"single": lad.CC_KERNEL_SINGLE, "pair": lad.CC_KERNEL_PAIR,
                                       "kblock": lad.CC_KERNEL_KBLOCK_WINDOWS,
                                       "pairkblock": lad.CC_KERNEL_PAIR_KBLOCK_WINDOWS}[args.kernel])
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch24":
        return run_batch(args)
    if args.mode == "autograd":
        return run_autograd(args)
    if args.mode == "fp64cmp":
        return run_fp64cmp(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

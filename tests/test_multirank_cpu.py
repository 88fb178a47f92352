"""Multi-rank paths on CPU (gloo, world size 2).

1. One system sharded by pair blocks: each rank computes Omega for the pairs
   of its blocks and a partial D for their rows (FP64 oracle per shard); a
   reduce-scatter sums D, an all-gather assembles Omega; the result equals
   the single-rank oracle.
2. The weak-scaling aggregation bench.py uses under torchrun: max step time
   over ranks, value = world * F / time.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2202_02019_gb300 import shard, synth

O_, V_, NJ_ = 3, 14, 20
S_ = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, tb1, tb2 = synth.make_pair(O_, V_, NJ_, 6.0, seed=5)
        tt = O.tau(s.t1, s.t2)
        G = O.gamma_dense(tb2, tt)                         # [a, b, c, d]
        blocks = shard.pair_blocks(V_, S_)
        mine = shard.lpt_partition(blocks, world, O_, V_, NJ_)[rank]
        om = np.zeros((O_, O_, V_, V_))
        D = np.zeros((NJ_, V_, V_))
        for k in mine:
            b = blocks[k]
            A = range(b.a0, b.a0 + b.na)
            B = range(b.b0, b.b0 + b.nb)
            for a in A:
                cols = [x for x in B if (not b.diag) or x >= a]
                if cols:
                    om[:, :, a, cols] = O.residual_rows(s.L_vv, tt, [a], cols)[:, :, 0, :]
                    for j, x in enumerate(cols):      # Omega_ij^ba = Omega_ji^ab
                        om[:, :, x, a] = om[:, :, a, x].T
            # partial D: ordered pairs (x in alpha, y in beta) and (x in beta, y in alpha)
            pairs = [(list(A), list(B))] + ([] if b.diag else [(list(B), list(A))])
            for X, Y in pairs:
                D[:, X, :] += np.einsum("xycd,Jyd->Jxc", G[np.ix_(X, Y)], s.L_vv[:, Y, :])
        # D: the reduce-scatter of shard.reduce_scatter_D (gloo: all-reduce and keep this
        # rank's slice); Omega: ranks own disjoint entries, so a sum gathers it
        outD = shard.reduce_scatter_D(torch.from_numpy(D.copy()), world)
        omt = torch.from_numpy(om.copy())
        dist.all_reduce(omt, op=dist.ReduceOp.SUM)
        q.put((rank, outD.numpy(), omt.numpy(), mine))
    finally:
        dist.destroy_process_group()


def test_pair_block_sharding_equals_single_rank():
    assert (NJ_ * V_ * V_) % 2 == 0
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    s, tb1, tb2 = synth.make_pair(O_, V_, NJ_, 6.0, seed=5)
    tt = O.tau(s.t1, s.t2)
    om_ref = O.residual_dense(s.L_vv, tt)
    D_ref = O.density_dense(s.L_vv, tb2, tt)
    D = np.concatenate([r[1] for r in res]).reshape(D_ref.shape)
    assert np.allclose(D, D_ref, rtol=1e-12, atol=1e-12 * np.abs(D_ref).max())
    for r in res:
        assert np.allclose(r[2], om_ref, rtol=1e-12, atol=1e-12 * np.abs(om_ref).max())
    owned = sorted(res[0][3] + res[1][3])
    assert owned == list(range(len(shard.pair_blocks(V_, S_))))


def test_lpt_partition_balances():
    blocks = shard.pair_blocks(650, 48)
    parts = shard.lpt_partition(blocks, 8, 78, 650, 4000)
    loads = [sum(shard.block_flops(78, 650, 4000, blocks[k]) for k in p) for p in parts]
    assert sorted(sum(parts, [])) == list(range(len(blocks)))
    assert max(loads) / min(loads) < 1.1


def _agg_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, val = shard.aggregate_step_time(100.0 + 50.0 * rank, world, 1e15)
        q.put((rank, ms, val))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_agg_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, val in res:
        assert ms == 150.0
        assert abs(val - 2 * 1e15 / 0.150 / 1e12) < 1e-9

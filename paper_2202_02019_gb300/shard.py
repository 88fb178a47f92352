"""Partition of one system's pair blocks over ranks (multi-GPU design).

The ladder path shards along the virtual-pair blocks the library already
iterates over: block (alpha <= beta) holds the pairs a <= b with a in block
alpha and b in block beta.  A rank that owns a block produces Omega for its
pairs outright (no reduction: rows ab are disjoint between blocks) and a
partial D for the rows x of both blocks; the partial D of all ranks is summed
by one reduce-scatter (FP64), and Omega, if wanted whole, by an all-gather.
Blocks are dealt largest-first to the least-loaded rank (LPT) by their
counted flops.  The same blocking and flop count are used here as in the
library (csrc/ccladder.cu, cc_ladder_pair_blocks) and in bench.py; a rank
runs its share with cc_ladder_step_blocks and the partial D meet in one
reduce-scatter.
"""
from __future__ import annotations

from typing import List, NamedTuple


class PairBlock(NamedTuple):
    a0: int
    na: int
    b0: int
    nb: int
    diag: bool

    @property
    def npairs(self) -> int:
        return self.na * (self.na + 1) // 2 if self.diag else self.na * self.nb


def pair_blocks(v: int, s: int = 48) -> List[PairBlock]:
    s = max(4, (s // 4) * 4)
    s = min(s, ((v + 3) // 4) * 4)
    nblk = (v + s - 1) // s
    out = []
    for al in range(nblk):
        for be in range(al, nblk):
            a0, b0 = al * s, be * s
            out.append(PairBlock(a0, min(s, v - a0), b0, min(s, v - b0), al == be))
    return out


def block_flops(o: int, v: int, nj: int, b: PairBlock) -> float:
    """Counted (packed) flops of one block: g-build + ladder + Gamma + D."""
    p = b.npairs
    qop, qom = o * (o + 1) // 2, o * (o - 1) // 2
    pvp, pvm = v * (v + 1) // 2, v * (v - 1) // 2
    g = 2.0 * p * v * v * nj
    lad = 2.0 * p * (pvp * qop + pvm * qom)
    gam = lad
    dens = 2.0 * nj * v * v * (2 * b.na * b.nb if not b.diag else b.na * b.na)
    return g + lad + gam + dens


def lpt_partition(blocks: List[PairBlock], n_ranks: int, o: int, v: int, nj: int) -> List[List[int]]:
    """Indices of the blocks each rank owns, largest block first to the lightest rank."""
    order = sorted(range(len(blocks)), key=lambda k: -block_flops(o, v, nj, blocks[k]))
    load = [0.0] * n_ranks
    parts: List[List[int]] = [[] for _ in range(n_ranks)]
    for k in order:
        r = min(range(n_ranks), key=lambda i: load[i])
        parts[r].append(k)
        load[r] += block_flops(o, v, nj, blocks[k])
    return [sorted(p) for p in parts]


def aggregate_step_time(ms_local: float, world: int, flops_per_rank: float):
    """Weak-scaling figure of a multi-rank run: max step time over ranks and
    value = world * flops / time (TFLOP/s).  Needs an initialised process group
    when world > 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64)
    if world > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = t.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t[0])
    return ms, world * flops_per_rank / (ms * 1e-3) / 1e12


def rank_blocks(system, rank: int, world: int) -> List[int]:
    """Pair blocks of `system` (a ladder.System) that rank `rank` of `world` owns, in the
    library's pair-block numbering (the blocking is checked against the library's own)."""
    from . import ladder as lad
    count, edge = lad.cc_ladder_pair_blocks(system)
    blocks = pair_blocks(system.v, edge)
    if len(blocks) != count:
        raise RuntimeError(f"pair-block count mismatch: {len(blocks)} here, {count} in the library")
    return lpt_partition(blocks, world, system.o, system.v, system.nj)[rank]


def reduce_scatter_D(D_part, world: int):
    """Sum the ranks' partial D (any float64 tensor, flattened) and return this rank's
    contiguous slice of the sum, the flat D padded to a multiple of world.  One
    reduce-scatter with NCCL; gloo has none, so there it is an all-reduce and a slice."""
    import torch
    import torch.distributed as dist
    flat = D_part.reshape(-1)
    n = flat.numel()
    chunk = (n + world - 1) // world
    if chunk * world != n:
        flat = torch.cat([flat, flat.new_zeros(chunk * world - n)])
    rank = dist.get_rank()
    if dist.get_backend() == "nccl":
        out = flat.new_empty(chunk)
        dist.reduce_scatter_tensor(out, flat, op=dist.ReduceOp.SUM)
        return out
    full = flat.clone()
    dist.all_reduce(full, op=dist.ReduceOp.SUM)
    return full[rank * chunk:(rank + 1) * chunk].clone()

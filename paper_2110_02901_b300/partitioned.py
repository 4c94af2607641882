"""Row-partitioned mini-batch value iteration over several ranks (one GPU each).

The states are split by rows: rank r owns the contiguous range [lo_r, hi_r) of ``row_range``.  Every
rank keeps a full replica of V and evaluates the same order sigma_{seed,k} of sweep k (Sec. III-A),
so every rank knows batch t = positions [t b, (t+1) b).  In each batch a rank backs up the batch's
states it owns from its replica -- every state of a batch reads the values from before the batch
(eq. (11)) -- the ranks exchange the batch's b new values with one all-reduce (each position has
exactly one owner and the others contribute 0, so the sum is the owner's value exactly), and every
replica writes them.  The replicas therefore stay identical, and so does the sweep change delta_k
that stops the solve (the paper's VI stop rule).  b >= n is one batch: the Bellman operator T
(eq. (7)), whose order does not matter.

The exchange per batch is b * 4 bytes on a device (float32) and one collective, so the form pays only
when a batch's stream of transition rows, spread over the ranks, takes longer than that collective:
large b.  ``partitioned_vi`` wires the GPU pieces: the order from rmb_permutation, the owned states'
backups from rmb_backup_states (one warp per state, float32 values as given, not centred), and the
exchange through torch.distributed (NCCL between GPUs).  ``partitioned_mbvi`` is the loop itself,
with those three pieces passed in, so it can run on other backends as well.
"""
from __future__ import annotations

from typing import Callable, Dict

import torch


def row_range(n: int, rank: int, world: int):
    """The states [lo, hi) that rank owns: contiguous rows, sizes differing by at most one."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def partitioned_mbvi(n: int, b: int, eps: float, max_sweeps: int, V: torch.Tensor,
                     order_of: Callable[[int], torch.Tensor],
                     backup: Callable[[torch.Tensor, torch.Tensor], torch.Tensor],
                     allreduce_sum: Callable[[torch.Tensor], None],
                     rank: int, world: int, start_sweep: int = 0) -> Dict:
    """MB-VI on this rank's replica V (updated in place) until a sweep's sup-norm change is <= eps or
    max_sweeps sweeps.  order_of(k): the n states of sweep k in processing order (a tensor on V's
    device); backup(V, states): new values of the given states from V; allreduce_sum(x): in-place sum
    over the ranks.  Returns dict(sweeps, deltas) (the same on every rank)."""
    lo, hi = row_range(n, rank, world)
    b = max(1, min(int(b), int(n)))
    deltas = []
    for j in range(int(max_sweeps)):
        k = int(start_sweep) + j
        order = torch.arange(n, dtype=torch.int32, device=V.device) if b >= n else order_of(k)
        V_prev = V.clone()
        for p0 in range(0, n, b):
            states = order[p0:p0 + b]
            mine = (states >= lo) & (states < hi)
            W = torch.zeros(states.numel(), dtype=V.dtype, device=V.device)
            idx = torch.nonzero(mine).flatten()
            if idx.numel():
                W[idx] = backup(V, states[idx].contiguous())
            allreduce_sum(W)
            V[states.long()] = W
        delta = float((V - V_prev).abs().max())
        deltas.append(delta)
        if delta <= eps:
            break
    return {"sweeps": len(deltas), "deltas": deltas}


def partitioned_vi(dm, opts, V: torch.Tensor, group=None, stream=None) -> Dict:
    """Row-partitioned MB-VI of a DeviceMDP over the ranks of torch.distributed (each rank holds the
    whole MDP and a replica V on its GPU; opts.batch, seed, eps, max_sweeps and start_sweep apply)."""
    import torch.distributed as dist

    from . import rmb_backup_states, rmb_permutation
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0

    def order_of(k):
        return rmb_permutation(dm.n, opts.seed, k, stream=stream)

    def backup(Vr, states):
        return rmb_backup_states(dm, Vr, states, stream=stream)

    def allreduce_sum(x):
        if world > 1:
            dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)

    b = dm.n if opts.batch == 0 else opts.batch
    return partitioned_mbvi(dm.n, b, opts.eps, opts.max_sweeps, V, order_of, backup, allreduce_sum, rank, world,
                            start_sweep=opts.start_sweep)

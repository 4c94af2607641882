"""The bench's multi-rank path (replicas, one per GPU) on the host: world_size 2 over gloo on CPU.
Checks the max-over-ranks timing and the whole-job sums that bench.py reports."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 + rank, w)        # per-rank time: the slowest rank counts
    tot = bench.sum_over_ranks(1000 * (rank + 1), w)  # per-rank work: the job's total
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, mx, tot))


@pytest.mark.parametrize("world", [2])
def test_replica_aggregation_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, tot in out:
        assert mx == 10.0 + (world - 1)
        assert tot == 1000 * world * (world + 1) / 2


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5 and bench.sum_over_ranks(7, 1) == 7

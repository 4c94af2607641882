"""Row-partitioned mini-batch value iteration (states split by rows over ranks, V replicated, the
batch's new values exchanged by one all-reduce per batch) on the host: world_size 2 and 3 over gloo
on CPU.  Each rank's backups come from the FP64 oracle, so the partitioned trajectory must equal the
oracle's own MB-VI (eq. (11), the order sigma_{seed,k} of Sec. III-A) bit for bit: same values, same
sweep changes, same stopping sweep."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2110_02901_b300.partitioned import partitioned_mbvi, row_range  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _make(kind):
    import mdpgen
    if kind == "csr":
        return mdpgen.csr_ragged(211, 3, 6, gamma=0.9, seed=5, inadmissible_frac=0.2)
    return mdpgen.dense_dirichlet(150, 4, alpha=0.5, gamma=0.95, seed=6)


def _oracle_pieces(mdp, seed):
    import oracle

    def order_of(k):
        return torch.from_numpy(oracle.perm(mdp.n, seed, k).astype(np.int64))

    def backup(V, states):
        Vn = V.numpy()
        return torch.tensor([min(oracle.q_factor(mdp, int(s), a, Vn) for a in range(mdp.m)) for s in states.tolist()],
                            dtype=torch.float64)

    return order_of, backup


def _worker(rank, world, port, kind, b, eps, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mdp = _make(kind)
    order_of, backup = _oracle_pieces(mdp, 17)
    V = torch.zeros(mdp.n, dtype=torch.float64)
    res = partitioned_mbvi(mdp.n, b, eps, 400, V, order_of, backup,
                           lambda x: dist.all_reduce(x, op=dist.ReduceOp.SUM), rank, world, start_sweep=3)
    dist.destroy_process_group()
    q.put((rank, V.numpy(), res["sweeps"], res["deltas"]))


def test_row_range_partitions_the_states():
    for n, world in ((1, 1), (7, 3), (211, 2), (1000, 7)):
        spans = [row_range(n, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
        sizes = [h - l for l, h in spans]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("kind,b,world", [("csr", 37, 2), ("dense", 16, 3), ("csr", 211, 2)])
def test_partitioned_trajectory_equals_the_oracle(kind, b, world):
    import oracle
    mdp = _make(kind)
    eps = 1e-9
    ref = oracle.mbvi(mdp, b, seed=17, eps=eps, max_sweeps=400, start_sweep=3)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, b, eps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, V, sweeps, deltas in out:
        assert sweeps == ref["sweeps"], (rank, sweeps, ref["sweeps"])
        assert np.array_equal(V, ref["V"]), rank                      # bit for bit
        assert np.array_equal(np.array(deltas), ref["deltas"]), rank


def test_single_rank_needs_no_collective():
    import oracle
    mdp = _make("csr")
    order_of, backup = _oracle_pieces(mdp, 4)
    V = torch.zeros(mdp.n, dtype=torch.float64)
    res = partitioned_mbvi(mdp.n, 50, 0.0, 6, V, order_of, backup, lambda x: None, 0, 1)
    ref = oracle.mbvi(mdp, 50, seed=4, eps=0.0, max_sweeps=6)
    assert res["sweeps"] == 6 and np.array_equal(V.numpy(), ref["V"])

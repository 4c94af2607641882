"""2D-maze stand-ins of Sec. IV-A (generator checks) and oracle pins on them.

The pins tie the oracle to facts that hold on a maze independently of it:
* slip = 0 (deterministic moves, unit cost, absorbing zero-cost goal): J*(s) = (1 - gamma^d) / (1 - gamma)
  with d the breadth-first distance of s to the goal (a geometric sum along a shortest path);
* slip > 0: that value is a lower bound of J* (every path to the goal takes at least d unit-cost steps);
* the batch-size comparison theorem of Sec. III-B (costs >= 0, J0 = 0, b' | b): after every sweep
  B_{b'}^k 0 >= B_b^k 0 elementwise, so the error to J* after k sweeps is no larger for b'.
"""
from collections import deque

import numpy as np
import pytest

import mdpgen
import oracle
from oracle import exact


def bfs_distance(mdp):
    grid, cells, goal = mdp.meta["grid"], mdp.meta["cells"], mdp.meta["goal"]
    N = grid.shape[0]
    dist = -np.ones(grid.shape, dtype=np.int64)
    r0, c0 = cells[goal]
    dist[r0, c0] = 0
    q = deque([(r0, c0)])
    while q:
        r, c = q.popleft()
        for dr, dc in mdpgen.MAZE_MOVES:
            rr, cc = r + dr, c + dc
            if 0 <= rr < N and 0 <= cc < N and grid[rr, cc] and dist[rr, cc] < 0:
                dist[rr, cc] = dist[r, c] + 1
                q.append((rr, cc))
    return dist[cells[:, 0], cells[:, 1]]


@pytest.mark.parametrize("make,n", [(mdpgen.maze80, 6166), (mdpgen.maze100, 9706)])
def test_paper_shapes_and_connectivity(make, n):
    mdp = make()
    assert (mdp.n, mdp.m, mdp.gamma) == (n, 4, 0.95)
    assert int(mdp.meta["grid"].sum()) == n
    d = bfs_distance(mdp)
    assert (d >= 0).all()                       # every open cell reaches the goal
    assert d[mdp.meta["goal"]] == 0


def test_rows_costs_and_goal():
    mdp = mdpgen.maze(24, 500, slip=0.3, seed=3)
    grid, cells, goal = mdp.meta["grid"], mdp.meta["cells"], mdp.meta["goal"]
    N = grid.shape[0]
    index = {tuple(x): i for i, x in enumerate(cells)}
    c = mdp.cost.reshape(mdp.n, 4)
    assert (c[goal] == 0).all() and (np.delete(c, goal, axis=0) == 1).all()
    for s in range(mdp.n):
        r, cc = cells[s]
        nb = [index.get((r + dr, cc + dc), s) for dr, dc in mdpgen.MAZE_MOVES]
        for a in range(4):
            lo, hi = mdp.row_ptr[s * 4 + a], mdp.row_ptr[s * 4 + a + 1]
            col, p = mdp.col[lo:hi], mdp.prob[lo:hi].astype(np.float64)
            assert abs(p.sum() - 1.0) < 1e-6
            if s == goal:
                assert list(col) == [s] and p[0] == 1.0
                continue
            assert list(col) == sorted(set([s] + nb))           # the cell and its open neighbours
            assert (p > 0).all()                                 # every admissible triple has mass
            assert np.isclose(p[list(col).index(nb[a])], 0.7, atol=1e-7)


def test_deterministic_maze_closed_form():
    mdp = mdpgen.maze(20, 360, gamma=0.95, slip=0.0, seed=4)
    d = bfs_distance(mdp)
    want = (1.0 - 0.95 ** d.astype(np.float64)) / (1.0 - 0.95)
    jstar, _, _ = exact.policy_iteration(mdp)
    assert np.max(np.abs(jstar - want)) < 1e-10
    for b in (1, 37, mdp.n):
        ref = oracle.mbvi(mdp, b, seed=2, eps=1e-12, max_sweeps=5000)
        assert np.max(np.abs(ref["V"] - want)) < 1e-9, b


def test_slip_lower_bound():
    mdp = mdpgen.maze(20, 360, gamma=0.95, slip=0.2, seed=4)
    d = bfs_distance(mdp)
    low = (1.0 - 0.95 ** d.astype(np.float64)) / (1.0 - 0.95)
    jstar, _, _ = exact.policy_iteration(mdp)
    assert (jstar >= low - 1e-12).all()
    assert (jstar > low + 1e-3).sum() > mdp.n // 2         # slipping costs something almost everywhere


def test_batch_size_comparison_on_a_divisor_chain():
    mdp = mdpgen.maze(24, 520, gamma=0.95, slip=0.2, seed=7)     # chain 1 | 10 | 130 | 520
    jstar, _, _ = exact.policy_iteration(mdp)
    errs = {}
    for b in (1, 10, 130, 520):
        ref = oracle.mbvi(mdp, b, seed=11, eps=0.0, max_sweeps=40, traj=True)
        errs[b] = np.abs(ref["traj"] - jstar).max(axis=1)
        if b > 1:
            prev = oracle.mbvi(mdp, {10: 1, 130: 10, 520: 130}[b], seed=11, eps=0.0, max_sweeps=40, traj=True)
            assert (prev["traj"] >= ref["traj"] - 1e-12).all(), b    # B_{b'}^k 0 >= B_b^k 0
    for lo, hi in ((1, 10), (10, 130), (130, 520)):
        assert (errs[lo] <= errs[hi] + 1e-12).all()
    assert errs[1][-1] < errs[520][-1]

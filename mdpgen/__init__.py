"""Seeded synthetic MDP generators shared by the tests, the benchmark and the oracle checks.

This module only draws problem data (transition rows, costs, start values, policies).  It holds
none of the mini-batch operator's arithmetic, so both the CUDA path and the FP64 oracle can take
their inputs from it without sharing any of the method.

Every array is drawn in FP64 from ``numpy.random.Generator(PCG64(seed))`` and rounded to FP32
(int32 for successor indices, int64 for CSR row pointers).  The FP32-rounded arrays *are* the
problem: the oracle promotes them exactly to FP64 and never renormalises them.

Layout (shared with the C-ABI): row ``r = s*m + a`` holds P(.|s,a).
  dense: ``P[n, m, n]`` float32, row-major, so the m rows of a state are contiguous;
  CSR:   ``row_ptr[n*m+1]`` int64, ``col[nnz]`` int32 (sorted within a row), ``prob[nnz]`` float32;
  both:  ``cost[n*m]`` float32, ``+inf`` marks an inadmissible action (the paper's U(i), Sec. II-A).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "MDP", "dense_dirichlet", "csr_uniform_k", "batched_uneven", "random_values",
    "random_policy", "config1", "config2", "config3", "config4", "config5", "csr_ragged",
    "maze_grid", "maze", "maze80", "maze100",
]


@dataclasses.dataclass
class MDP:
    """A finite discounted MDP (S, U, P, g, alpha) of Sec. II-A with n states and m actions."""
    n: int
    m: int
    gamma: float
    fmt: str                                   # "dense" | "csr"
    cost: np.ndarray                           # float32 [n*m]
    P: Optional[np.ndarray] = None             # float32 [n, m, n] (dense)
    row_ptr: Optional[np.ndarray] = None       # int64 [n*m+1] (csr)
    col: Optional[np.ndarray] = None           # int32 [nnz] (csr)
    prob: Optional[np.ndarray] = None          # float32 [nnz] (csr)
    logits: Optional[np.ndarray] = None        # float32 [nnz] when prob = softmax(logits)
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)   # generator extras (maze grid, goal state)

    @property
    def nnz(self) -> int:
        return int(self.n) * self.m * int(self.n) if self.fmt == "dense" else int(self.row_ptr[-1])

    def p_bytes(self) -> int:
        """Bytes of transition data (probabilities + indices) one full pass over all rows reads."""
        if self.fmt == "dense":
            return self.P.nbytes
        return self.prob.nbytes + self.col.nbytes

    def uniform_k(self) -> int:
        """Successors per row if every CSR row has the same length, else 0."""
        if self.fmt != "csr":
            return 0
        rows = self.n * self.m
        k = int(self.row_ptr[-1]) // rows if rows else 0
        if k * rows != int(self.row_ptr[-1]):
            return 0
        if not np.array_equal(self.row_ptr, np.arange(rows + 1, dtype=np.int64) * k):
            return 0
        return k


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _seq(seed) -> np.random.SeedSequence:
    return seed if isinstance(seed, np.random.SeedSequence) else np.random.SeedSequence(seed)


def _costs(rng, rows, dist):
    if dist == "uniform":
        return rng.random(rows).astype(np.float32)
    if dist == "normal":
        return rng.standard_normal(rows).astype(np.float32)
    raise ValueError(dist)


def dense_dirichlet(n: int, m: int, alpha: float = 1.0, gamma: float = 0.95, seed: int = 0,
                    cost_dist: str = "uniform", block_rows: int = 4096, name: str = "") -> MDP:
    """Dense rows P(.|s,a) ~ Dirichlet(alpha) over all n states (normalised Gamma(alpha) draws).

    Rows are drawn blockwise from independent child seeds so memory stays bounded at large n.
    """
    rows = n * m
    ss = _seq(seed)
    c_seq, p_seq = ss.spawn(2)
    cost = _costs(_rng(c_seq), rows, cost_dist)
    P = np.empty((rows, n), dtype=np.float32)
    nblk = (rows + block_rows - 1) // block_rows
    for bi, child in enumerate(p_seq.spawn(nblk)):
        r0, r1 = bi * block_rows, min(rows, (bi + 1) * block_rows)
        g = _rng(child)
        if alpha == 1.0:
            x = g.standard_exponential((r1 - r0, n))
        else:
            x = g.standard_gamma(alpha, (r1 - r0, n))
        s = x.sum(axis=1, keepdims=True)
        # a Gamma(alpha<1) row can underflow to all-zeros only for absurdly small n*alpha; guard anyway
        bad = (s[:, 0] <= 0)
        if bad.any():
            x[bad, 0] = 1.0
            s = x.sum(axis=1, keepdims=True)
        P[r0:r1] = (x / s).astype(np.float32)
    return MDP(n=n, m=m, gamma=gamma, fmt="dense", cost=cost, P=P.reshape(n, m, n), name=name)


def _distinct_sorted(g: np.random.Generator, rows: int, n: int, k: int) -> np.ndarray:
    """k distinct successors per row, uniform without replacement, sorted ascending."""
    if k > n:
        raise ValueError("k > n")
    if k * 4 >= n:
        # dense regime: a per-row permutation prefix
        out = np.empty((rows, k), dtype=np.int32)
        for r in range(rows):
            out[r] = np.sort(g.permutation(n)[:k])
        return out
    idx = g.integers(0, n, size=(rows, k), dtype=np.int32)
    idx.sort(axis=1)
    while True:
        dup = (np.diff(idx, axis=1) == 0).any(axis=1)
        nd = int(dup.sum())
        if nd == 0:
            return idx
        fix = g.integers(0, n, size=(nd, k), dtype=np.int32)
        fix.sort(axis=1)
        idx[dup] = fix


def csr_uniform_k(n: int, m: int, k: int, gamma: float = 0.99, seed: int = 0,
                  prob_kind: str = "dirichlet1", cost_dist: str = "uniform",
                  block_rows: int = 1 << 20, name: str = "") -> MDP:
    """CSR MDP: every (s,a) row has k distinct successors drawn uniformly without replacement.

    prob_kind "dirichlet1": probabilities ~ Dirichlet(1) (normalised Exp(1));
    prob_kind "softmax":    probabilities = softmax of N(0,1) logits (logits are returned too).
    """
    rows = n * m
    nnz = rows * k
    ss = _seq(seed)
    c_seq, p_seq = ss.spawn(2)
    cost = _costs(_rng(c_seq), rows, cost_dist)
    col = np.empty(nnz, dtype=np.int32)
    prob = np.empty(nnz, dtype=np.float32)
    logits = np.empty(nnz, dtype=np.float32) if prob_kind == "softmax" else None
    nblk = (rows + block_rows - 1) // block_rows
    for bi, child in enumerate(p_seq.spawn(nblk)):
        r0, r1 = bi * block_rows, min(rows, (bi + 1) * block_rows)
        g = _rng(child)
        idx = _distinct_sorted(g, r1 - r0, n, k)
        col[r0 * k:r1 * k] = idx.reshape(-1)
        if prob_kind == "dirichlet1":
            x = g.standard_exponential((r1 - r0, k))
            p = x / x.sum(axis=1, keepdims=True)
        elif prob_kind == "softmax":
            z = g.standard_normal((r1 - r0, k))
            logits[r0 * k:r1 * k] = z.astype(np.float32).reshape(-1)
            z32 = z.astype(np.float32).astype(np.float64)   # the logits the problem actually holds
            e = np.exp(z32 - z32.max(axis=1, keepdims=True))
            p = e / e.sum(axis=1, keepdims=True)
        else:
            raise ValueError(prob_kind)
        prob[r0 * k:r1 * k] = p.astype(np.float32).reshape(-1)
    row_ptr = np.arange(rows + 1, dtype=np.int64) * k
    return MDP(n=n, m=m, gamma=gamma, fmt="csr", cost=cost, row_ptr=row_ptr, col=col,
               prob=prob, logits=logits, name=name)


def csr_ragged(n: int, m: int, kmax: int, gamma: float = 0.9, seed: int = 0,
               inadmissible_frac: float = 0.0, name: str = "") -> MDP:
    """CSR MDP with row lengths uniform in {1..kmax} (ragged rows exercise the generic row path).

    A fraction of (s,a) pairs gets cost +inf (inadmissible); action 0 always stays admissible so
    every U(i) is nonempty (Sec. II-A).
    """
    g = _rng(seed)
    rows = n * m
    lens = g.integers(1, kmax + 1, size=rows).astype(np.int64)
    lens = np.minimum(lens, n)
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    prob = np.empty(int(row_ptr[-1]), dtype=np.float32)
    for r in range(rows):
        L = int(lens[r])
        c = np.sort(g.choice(n, size=L, replace=False)).astype(np.int32)
        x = g.standard_exponential(L)
        col[row_ptr[r]:row_ptr[r + 1]] = c
        prob[row_ptr[r]:row_ptr[r + 1]] = (x / x.sum()).astype(np.float32)
    cost = g.random(rows).astype(np.float32)
    if inadmissible_frac > 0:
        mask = g.random(rows) < inadmissible_frac
        mask[0::m] = False
        cost[mask] = np.inf
    return MDP(n=n, m=m, gamma=gamma, fmt="csr", cost=cost, row_ptr=row_ptr, col=col,
               prob=prob, name=name)


def random_values(n: int, seed: int = 0, scale: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """A seeded FP32 value vector (start values / test functions J)."""
    return (offset + scale * _rng(seed).standard_normal(n)).astype(np.float32)


def random_policy(n: int, m: int, seed: int = 0) -> np.ndarray:
    return _rng(seed).integers(0, m, size=n, dtype=np.int32)


# ---------------------------------------------------------------------------------------------
# The five benchmark workloads (synthetic stand-ins; MDP seeds 0..4, permutation seed 12345).
# Each takes optional size overrides so tests can build the same shapes at small sizes.
# ---------------------------------------------------------------------------------------------
PERM_SEED = 12345


def config1(n: int = 500, m: int = 4, seed: int = 0) -> MDP:
    """Dense n=500, m=4, Dirichlet(1) rows over all states, c ~ U[0,1], gamma=0.95 (b=50)."""
    return dense_dirichlet(n, m, alpha=1.0, gamma=0.95, seed=seed, name=f"dense-dirichlet1-n{n}-m{m}")


def config2(n: int = 1 << 20, m: int = 8, k: int = 32, seed: int = 1) -> MDP:
    """CSR n=2^20, m=8, k=32 distinct uniform successors, Dirichlet(1), c ~ U[0,1], gamma=0.99."""
    return csr_uniform_k(n, m, k, gamma=0.99, seed=seed, name=f"csr-k{k}-n{n}-m{m}")


def config3(count: int = 256, nmin: int = 256, nmax: int = 65536, k: int = 16, seed: int = 2) -> List[MDP]:
    """256 CSR MDPs: n log-uniform in [256, 65536], m ~ U{2..16}, k=16, gamma ~ U[0.9, 0.99]."""
    return batched_uneven(count, nmin, nmax, k, seed)


def batched_uneven(count: int, nmin: int, nmax: int, k: int, seed: int) -> List[MDP]:
    g = _rng(seed)
    ns = np.floor(np.exp(g.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)
    ms = g.integers(2, 17, size=count)
    gammas = g.uniform(0.9, 0.99, size=count)
    seeds = np.random.SeedSequence(seed).spawn(count)
    out = []
    for i in range(count):
        n_i = int(max(ns[i], k))
        out.append(csr_uniform_k(n_i, int(ms[i]), k, gamma=float(gammas[i]), seed=seeds[i],
                                 name=f"batched-{i}"))
    return out


def config4(n: int = 16384, m: int = 16, seed: int = 3) -> MDP:
    """Dense n=16384, m=16, Dirichlet(0.1) rows (peaked), c ~ N(0,1), gamma=0.999."""
    return dense_dirichlet(n, m, alpha=0.1, gamma=0.999, seed=seed, cost_dist="normal",
                           name=f"dense-dirichlet0.1-n{n}-m{m}")


def config5(n: int = 65536, m: int = 8, k: int = 16, seed: int = 4) -> MDP:
    """CSR n=65536, m=8, k=16, P = softmax(N(0,1) logits), c ~ U[0,1], gamma=0.95."""
    return csr_uniform_k(n, m, k, gamma=0.95, seed=seed, prob_kind="softmax",
                         name=f"csr-softmax-k{k}-n{n}-m{m}")


def dense_dirichlet_device(n: int, m: int, alpha: float, gamma: float, seed: int, cost_dist: str = "normal",
                           device="cuda", block_rows: int = 2048, name: str = ""):
    """Large dense Dirichlet(alpha) rows drawn directly in device memory with torch's seeded CUDA
    generator (float64 Gamma draws, normalised, rounded to float32).  Same distribution as
    `dense_dirichlet`, different random stream; for sizes whose host generation would take minutes.
    Returns (P [n, m, n] float32 tensor, cost [n*m] float32 tensor)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rows = n * m
    P = torch.empty((rows, n), dtype=torch.float32, device=device)
    conc = torch.full((block_rows, n), float(alpha), dtype=torch.float64, device=device)
    for r0 in range(0, rows, block_rows):
        r1 = min(rows, r0 + block_rows)
        x = torch._standard_gamma(conc[: r1 - r0], generator=g)
        s = x.sum(dim=1, keepdim=True)
        x[:, 0] += (s[:, 0] <= 0).to(x.dtype)          # an all-underflow row becomes a point mass
        P[r0:r1] = (x / x.sum(dim=1, keepdim=True)).to(torch.float32)
    if cost_dist == "normal":
        cost = torch.randn(rows, generator=g, dtype=torch.float64, device=device).to(torch.float32)
    else:
        cost = torch.rand(rows, generator=g, dtype=torch.float64, device=device).to(torch.float32)
    return P.reshape(n, m, n), cost


# ---------------------------------------------------------------------------------------------
# 2D-maze stand-ins (Sec. IV-A: an N x N maze with obstacles, 4 actions, every admissible
# state-action-next-state triple has nonzero probability, unit cost except at the terminal state;
# N = 80 and N = 100 leave 6166 and 9706 open cells).  The authors' maps are not available: the
# walls here are seeded random segments, placed only where every open cell stays reachable.
# ---------------------------------------------------------------------------------------------
MAZE_MOVES = ((-1, 0), (0, 1), (1, 0), (0, -1))      # actions 0..3: up, right, down, left


def maze_grid(N: int, n_open: int, seed: int = 0) -> np.ndarray:
    """Boolean N x N grid (True = open) with exactly ``n_open`` open cells, all 4-connected.

    Walls grow as straight segments of max(2, N//8)..max(2, N//2) cells from random cells in random
    directions; a cell whose removal would split the open cells is skipped (the segment stops).
    """
    from scipy import ndimage

    if not 1 <= n_open <= N * N:
        raise ValueError("n_open must be in [1, N*N]")
    g = _rng(seed)
    grid = np.ones((N, N), dtype=bool)
    walls = N * N - n_open
    placed = 0
    tries = 0
    while placed < walls:
        tries += 1
        if tries > 100 * N * N:
            raise RuntimeError("could not place the walls")
        r, c = (int(x) for x in g.integers(0, N, size=2))
        dr, dc = MAZE_MOVES[int(g.integers(0, 4))]
        for _ in range(int(g.integers(max(2, N // 8), max(2, N // 2) + 1))):
            if placed >= walls or not (0 <= r < N and 0 <= c < N) or not grid[r, c]:
                break
            grid[r, c] = False
            if ndimage.label(grid)[1] != 1:
                grid[r, c] = True
                break
            placed += 1
            r, c = r + dr, c + dc
    return grid


def maze(N: int, n_open: int, gamma: float = 0.95, slip: float = 0.2, seed: int = 0, name: str = "") -> MDP:
    """CSR MDP of an N x N maze with ``n_open`` open cells (states, row-major order).

    The goal (terminal) is the open cell nearest the corner (N-1, N-1): absorbing, cost 0.  Every
    other (state, action) pair costs 1.  Action a aims at the neighbour in direction a (or at the
    cell itself when a wall or the border is there); the successors are the cell and its open
    4-neighbours, the aimed one with probability 1 - slip and the others sharing slip evenly.
    slip = 0 keeps only the aimed successor (a deterministic maze).
    ``meta``: grid, goal (state index), cells (row, col of every state).
    """
    if not 0.0 <= slip < 1.0:
        raise ValueError("slip must be in [0, 1)")
    grid = maze_grid(N, n_open, seed)
    cells = np.argwhere(grid)                       # row-major: state s is cells[s]
    index = -np.ones((N, N), dtype=np.int64)
    index[grid] = np.arange(len(cells))
    corner = np.abs(cells - (N - 1)).sum(axis=1)
    goal = int(np.argmin(corner))
    m = 4
    rows = len(cells) * m
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    cols: List[np.ndarray] = []
    probs: List[np.ndarray] = []
    cost = np.ones(rows, dtype=np.float32)
    for s, (r, c) in enumerate(cells):
        nb = []
        for dr, dc in MAZE_MOVES:
            rr, cc = r + dr, c + dc
            ok = 0 <= rr < N and 0 <= cc < N and grid[rr, cc]
            nb.append(int(index[rr, cc]) if ok else s)
        support = np.array(sorted(set([s] + nb)), dtype=np.int32)
        for a in range(m):
            if s == goal:
                col_a, p_a = np.array([s], np.int32), np.array([1.0])
                cost[s * m + a] = 0.0
            elif slip == 0.0 or len(support) == 1:
                col_a, p_a = np.array([nb[a]], np.int32), np.array([1.0])
            else:
                p_a = np.where(support == nb[a], 1.0 - slip, slip / (len(support) - 1))
                col_a = support
            cols.append(col_a)
            probs.append(p_a)
            row_ptr[s * m + a + 1] = row_ptr[s * m + a] + len(col_a)
    col = np.concatenate(cols).astype(np.int32)
    prob = np.concatenate(probs).astype(np.float32)
    return MDP(n=len(cells), m=m, gamma=gamma, fmt="csr", cost=cost, row_ptr=row_ptr, col=col, prob=prob,
               name=name or f"maze{N}", meta={"grid": grid, "goal": goal, "cells": cells})


def maze80(seed: int = 5, slip: float = 0.2) -> MDP:
    """The N = 80 maze shape of Sec. IV-A: 6166 states, 4 actions, gamma 0.95."""
    return maze(80, 6166, gamma=0.95, slip=slip, seed=seed, name="maze80")


def maze100(seed: int = 6, slip: float = 0.2) -> MDP:
    """The N = 100 maze shape of Sec. IV-A: 9706 states, 4 actions, gamma 0.95."""
    return maze(100, 9706, gamma=0.95, slip=slip, seed=seed, name="maze100")

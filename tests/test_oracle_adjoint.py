"""Pins for the oracle's fixed-point gradient: central finite differences (FP64, h = 1e-4) of the
exact optimal value (policy iteration with direct solves) with respect to costs and transition
logits, on coordinates away from action ties."""
import dataclasses

import numpy as np
import pytest

import mdpgen
from oracle import exact


def _loss(mdp, w):
    J, _, _ = exact.policy_iteration(mdp)
    return float(w @ J)


def _with_logits(mdp, z):
    m2 = dataclasses.replace(mdp)
    m2.prob = exact.softmax_rows(z, mdp.row_ptr)          # FP64 probabilities
    return m2


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    base = mdpgen.csr_uniform_k(40, 3, 5, gamma=0.9, seed=seed, prob_kind="softmax")
    z0 = base.logits.astype(np.float64)
    mdp = _with_logits(base, z0)
    w = np.random.default_rng(seed).standard_normal(mdp.n)
    lam, gc, gz, jstar, pistar = exact.fixed_point_gradient(mdp, w)
    _, _, gap, _ = exact.bellman_pass(mdp, jstar)
    h = 1e-4
    rng = np.random.default_rng(100 + seed)
    checked = 0
    # costs: greedy actions (nonzero gradient) and others (exactly zero)
    for r in list(np.arange(mdp.n) * mdp.m + pistar)[:12] + list(rng.integers(0, mdp.n * mdp.m, 8)):
        s = r // mdp.m
        if gap[s] < 1e-2:
            continue
        mp, mm = dataclasses.replace(mdp), dataclasses.replace(mdp)
        mp.cost = mdp.cost.astype(np.float64).copy(); mp.cost[r] += h
        mm.cost = mdp.cost.astype(np.float64).copy(); mm.cost[r] -= h
        fd = (_loss(mp, w) - _loss(mm, w)) / (2 * h)
        assert abs(fd - gc[r]) <= 1e-6 * max(1.0, abs(gc[r])), (r, fd, gc[r])
        checked += 1
    # logits of greedy rows
    for s in rng.permutation(mdp.n)[:10]:
        if gap[s] < 1e-2:
            continue
        r = s * mdp.m + pistar[s]
        e = int(mdp.row_ptr[r]) + int(rng.integers(0, 5))
        zp, zm = z0.copy(), z0.copy()
        zp[e] += h
        zm[e] -= h
        fd = (_loss(_with_logits(base, zp), w) - _loss(_with_logits(base, zm), w)) / (2 * h)
        assert abs(fd - gz[e]) <= 1e-6 * max(1.0, abs(gz[e])), (e, fd, gz[e])
        checked += 1
    assert checked >= 15


def test_lambda_is_the_discounted_occupancy_of_w():
    """lambda = sum_t alpha^t (P_mu^T)^t w (Neumann series of the adjoint system)."""
    mdp = mdpgen.csr_uniform_k(200, 4, 6, gamma=0.8, seed=5)
    w = np.random.default_rng(1).standard_normal(mdp.n)
    lam, gc, _, _, pistar = exact.fixed_point_gradient(mdp, w)
    Pm, _ = exact.policy_matrix(mdp, pistar)
    acc, term = np.zeros(mdp.n), w.copy()
    for _ in range(400):
        acc += term
        term = mdp.gamma * (Pm.T @ term)
    assert np.max(np.abs(acc - lam)) < 1e-10
    assert np.count_nonzero(gc) == np.count_nonzero(lam)

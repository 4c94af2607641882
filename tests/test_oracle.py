"""Pins for the FP64 oracle: each checks it against something other than itself.

* Philox4x32-10 against published known-answer vectors (tests/golden/philox4x32_10_kat.txt);
* the permutation: bijection, independence from b, uniform position of a state;
* a hand-derived closed form (tests/golden/two_state_closed_form.txt);
* brute force over every deterministic policy with direct solves (eq. (2), eq. (4));
* the set-based definition of M_b(i) and B_b (eqs. (10)-(12)) evaluated literally;
* the b=n (Bellman, eq. (7)) and b=1 (Gauss-Seidel, Sec. II-D) reductions (Sec. III-A);
* monotonicity, shift invariance, alpha-contraction, fixed point (Sec. III-B.1);
* the batch-size comparison theorem and corollary (Sec. III-B.2) on divisor chains;
* MB-MPI (Alg. 1) against exact policy iteration; the stopping error bound.
"""
import os

import numpy as np
import pytest

import mdpgen
import oracle
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(v[:4], v[4:6])
        assert list(int(x) for x in out) == v[6:]
        n += 1
    assert n == 3


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 17, 500, 1000, 4097, 65536, 99991])
def test_perm_is_bijection(n):
    for sweep in (0, 1, 12345678901):
        p = oracle.perm(n, 12345, sweep)
        assert np.array_equal(np.sort(p), np.arange(n))


def test_perm_large_bijection_and_sweeps_differ():
    n = 1 << 20
    a = oracle.perm(n, 12345, 0)
    b = oracle.perm(n, 12345, 1)
    assert np.array_equal(np.sort(a), np.arange(n))
    assert not np.array_equal(a, b)
    # a random bijection has about one fixed point
    assert np.sum(a == np.arange(n)) < 20


def test_perm_matches_single_evaluation_and_seed_matters():
    n = 777
    p = oracle.perm(n, 99, 5)
    for pos in (0, 1, 100, 776):
        assert oracle.perm_at(n, 99, 5, pos) == p[pos]
    assert not np.array_equal(p, oracle.perm(n, 100, 5))


def test_perm_uniform_position():
    """Chi-square: the position of a fixed state over many seeds is uniform on [0, n)."""
    n, trials = 10, 20000
    counts = np.zeros(n)
    for seed in range(trials):
        p = oracle.perm(n, seed, 3)
        counts[int(np.nonzero(p == 3)[0][0])] += 1
    e = trials / n
    chi2 = float(((counts - e) ** 2 / e).sum())
    assert chi2 < 27.88  # 99.9% quantile of chi-square with 9 dof


def test_perm_half_bits():
    assert oracle.perm_half_bits(1) == 1
    assert oracle.perm_half_bits(2) == 1
    assert oracle.perm_half_bits(4) == 1
    assert oracle.perm_half_bits(5) == 2
    assert oracle.perm_half_bits(500) == 5
    assert oracle.perm_half_bits(1 << 20) == 10
    assert oracle.perm_half_bits((1 << 20) + 1) == 11


# ------------------------------------------------------------------------------------------------
def _golden_two_state():
    rows, meta = {}, {}
    for line in open(os.path.join(GOLDEN, "two_state_closed_form.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        if t[0] == "row":
            rows[(int(t[1]), int(t[2]))] = (float(t[3]), [float(x) for x in t[4:]])
        else:
            meta[t[0]] = t[1:]
    n, m = 2, 2
    P = np.zeros((n, m, n), np.float32)
    c = np.zeros(n * m, np.float32)
    for (s, a), (cost, p) in rows.items():
        P[s, a] = p
        c[s * m + a] = cost
    mdp = mdpgen.MDP(n=n, m=m, gamma=float(meta["gamma"][0]), fmt="dense", cost=c, P=P)
    return mdp, meta


def test_golden_two_state_closed_form():
    mdp, meta = _golden_two_state()
    jstar = np.array([float(x) for x in meta["jstar"]])
    pistar = np.array([int(x) for x in meta["pistar"]])
    pol = np.array([int(x) for x in meta["policy"][:2]])
    val = np.array([float(x) for x in meta["policy"][3:5]])
    for b in (1, 2):
        r = oracle.mbvi(mdp, b, seed=7, eps=1e-14, max_sweeps=2000)
        assert np.allclose(r["V"], jstar, rtol=0, atol=1e-12)
        _, pi, _, _ = oracle.greedy(mdp, r["V"])
        assert np.array_equal(pi, pistar)
        ev = oracle.eval_policy(mdp, pol, b, seed=3, eps=1e-14, max_sweeps=5000)
        assert np.allclose(ev["V"], val, rtol=0, atol=1e-10)
    assert np.allclose(exact.policy_value(mdp, pol), val, atol=1e-12)
    assert np.allclose(exact.brute_force(mdp), jstar, atol=1e-12)


# ------------------------------------------------------------------------------------------------
def _tiny_mdps():
    out = []
    for seed in range(3):
        out.append(mdpgen.dense_dirichlet(6, 3, alpha=1.0, gamma=0.9, seed=seed))
        out.append(mdpgen.csr_uniform_k(6, 3, 3, gamma=0.85, seed=10 + seed))
    out.append(mdpgen.csr_ragged(5, 3, 4, gamma=0.8, seed=4, inadmissible_frac=0.3))
    out.append(mdpgen.dense_dirichlet(5, 2, alpha=0.1, gamma=0.95, seed=9, cost_dist="normal"))
    return out


@pytest.mark.parametrize("idx", range(8))
def test_mbvi_matches_brute_force(idx):
    mdp = _tiny_mdps()[idx]
    jstar = exact.brute_force(mdp)
    # every optimal policy is greedy w.r.t. J*; brute force identifies J* uniquely
    for b in sorted({1, 2, 3, mdp.n}):
        for seed in (0, 1, 2):
            r = oracle.mbvi(mdp, b, seed=seed, eps=1e-13, max_sweeps=20000)
            assert np.max(np.abs(r["V"] - jstar)) < 1e-10, (b, seed)
            TV, pi, gap, res = oracle.greedy(mdp, r["V"])
            Jpi = exact.policy_value(mdp, pi)
            sel = gap > 1e-9
            assert np.max(np.abs(Jpi - jstar)[sel] if sel.any() else 0) < 1e-8


@pytest.mark.parametrize("idx", range(8))
def test_policy_evaluation_closed_form(idx):
    mdp = _tiny_mdps()[idx]
    c = mdp.cost.reshape(mdp.n, mdp.m)
    rng = np.random.default_rng(idx)
    pi = np.array([rng.choice(np.nonzero(np.isfinite(c[s]))[0]) for s in range(mdp.n)], np.int32)
    J = exact.policy_value(mdp, pi)
    for b in (1, 2, mdp.n):
        r = oracle.eval_policy(mdp, pi, b, seed=5, eps=1e-13, max_sweeps=50000)
        assert np.max(np.abs(r["V"] - J)) < 1e-10


def test_policy_evaluation_closed_form_medium():
    mdp = mdpgen.csr_uniform_k(3000, 4, 8, gamma=0.95, seed=3)
    pi = mdpgen.random_policy(mdp.n, mdp.m, seed=1)
    J = exact.policy_value(mdp, pi)
    r = oracle.eval_policy(mdp, pi, 256, seed=12345, eps=1e-12, max_sweeps=5000)
    assert np.max(np.abs(r["V"] - J)) < 1e-9


# ------------------------------------------------------------------------------------------------
def _definition_B(mdp, J, b, order, pi=None):
    """B_b J evaluated literally from eqs. (10)-(12): state at 1-based position i of the processing
    order reads BJ on M_b(i) = {first b*floor((i-1)/b) states of the order} and J elsewhere."""
    n, m = mdp.n, mdp.m
    BJ = {}
    for i in range(1, n + 1):
        s = int(order[i - 1])
        M = set(int(x) for x in order[: b * ((i - 1) // b)])
        acts = [int(pi[s])] if pi is not None else range(m)
        vals = []
        for a in acts:
            r = s * m + a
            g = float(mdp.cost[r])
            if np.isinf(g):
                vals.append(np.inf)
                continue
            if mdp.fmt == "dense":
                succ = [(j, float(mdp.P[s, a, j])) for j in range(n)]
            else:
                succ = [(int(mdp.col[e]), float(mdp.prob[e])) for e in range(mdp.row_ptr[r], mdp.row_ptr[r + 1])]
            tot = g
            for j, p in succ:
                tot += mdp.gamma * p * (BJ[j] if j in M else float(J[j]))
            vals.append(tot)
        BJ[s] = min(vals)
    return np.array([BJ[s] for s in range(n)])


@pytest.mark.parametrize("idx", range(8))
def test_mb_apply_matches_set_definition(idx):
    mdp = _tiny_mdps()[idx]
    J = mdpgen.random_values(mdp.n, seed=idx).astype(np.float64)
    pi = mdpgen.random_policy(mdp.n, mdp.m, seed=idx)
    c = mdp.cost.reshape(mdp.n, mdp.m)
    pi = np.where(np.isfinite(c[np.arange(mdp.n), pi]), pi, 0).astype(np.int32)
    for b in range(1, mdp.n + 1):
        for sweep in (0, 3):
            order = oracle.perm(mdp.n, 12345, sweep)
            got, _ = oracle.mb_apply(mdp, J, b, 12345, sweep)
            assert np.allclose(got, _definition_B(mdp, J, b, order), rtol=0, atol=1e-12)
            got, _ = oracle.mb_apply(mdp, J, b, 12345, sweep, pi=pi)
            assert np.allclose(got, _definition_B(mdp, J, b, order, pi), rtol=0, atol=1e-12)


def test_mb_apply_matches_set_definition_larger_ragged_tail():
    mdp = mdpgen.csr_uniform_k(37, 3, 5, gamma=0.9, seed=2)
    J = mdpgen.random_values(37, seed=1).astype(np.float64)
    for b in (4, 5, 10, 36):
        order = oracle.perm(37, 1, 9)
        got, _ = oracle.mb_apply(mdp, J, b, 1, 9)
        assert np.allclose(got, _definition_B(mdp, J, b, order), rtol=0, atol=1e-12)


def test_reductions_b_equals_n_and_b_equals_1():
    for mdp in (mdpgen.csr_uniform_k(300, 4, 8, gamma=0.9, seed=5), mdpgen.dense_dirichlet(120, 3, seed=6)):
        J = mdpgen.random_values(mdp.n, seed=3).astype(np.float64)
        got, _ = oracle.mb_apply(mdp, J, mdp.n, 77, 4)
        assert np.array_equal(got, oracle.bellman_T(mdp, J))
        assert np.allclose(got, exact.bellman_pass(mdp, J)[0], rtol=0, atol=1e-12)
        got, _ = oracle.mb_apply(mdp, J, 1, 77, 4)
        assert np.array_equal(got, oracle.gauss_seidel_F(mdp, oracle.perm(mdp.n, 77, 4), J))


def test_delta_is_sup_norm_change():
    mdp = mdpgen.csr_uniform_k(500, 4, 8, gamma=0.9, seed=8)
    r = oracle.mbvi(mdp, 64, seed=3, eps=0, max_sweeps=6, traj=True)
    prev = np.zeros(mdp.n)
    for k in range(6):
        assert r["deltas"][k] == np.max(np.abs(r["traj"][k] - prev))
        prev = r["traj"][k]


# ------------------------------------------------------------------------------------------------
def _apply_k(mdp, J, b, k, seed=12345, pi=None):
    V = np.array(J, dtype=np.float64)
    for sweep in range(k):
        V, _ = oracle.mb_apply(mdp, V, b, seed, sweep, pi=pi)
    return V


def test_shift_lemma_equality_fails_for_small_batches():
    """For b < n the exact shift identity B(J + r e) = BJ + alpha r e is false (Sec. III-B.1
    states it for every b); the states of earlier batches carry the shift alpha*r, not r."""
    mdp = mdpgen.csr_uniform_k(200, 4, 6, gamma=0.9, seed=1)
    J = mdpgen.random_values(200, seed=2).astype(np.float64)
    BJ, _ = oracle.mb_apply(mdp, J, 7, 12345, 0)
    Bs, _ = oracle.mb_apply(mdp, J + 1.0, 7, 12345, 0)
    assert np.max(np.abs(Bs - BJ - mdp.gamma)) > 1e-3
    # the first batch reads no updated state, so there the identity holds exactly
    first = oracle.perm(200, 12345, 0)[:7]
    assert np.max(np.abs((Bs - BJ - mdp.gamma)[first])) < 1e-7   # FP32 rows sum to 1 +- 4e-8


@pytest.mark.parametrize("fmt", ["csr", "dense"])
def test_monotonicity_shift_contraction(fmt):
    # FP32 rows sum to 1 within ~4e-8, so shift / contraction bounds carry a 1e-7 slack
    mdp = (mdpgen.csr_uniform_k(200, 4, 6, gamma=0.9, seed=1) if fmt == "csr"
           else mdpgen.dense_dirichlet(80, 3, gamma=0.9, seed=2))
    a = mdp.gamma
    rng = np.random.default_rng(0)
    pi = mdpgen.random_policy(mdp.n, mdp.m, seed=4)
    for b in (1, 7, 32, mdp.n):
        for trial in range(3):
            J = rng.standard_normal(mdp.n)
            Jp = J + np.abs(rng.standard_normal(mdp.n))          # J <= J'
            for k in (1, 3):
                for p in (None, pi):
                    BJ, BJp = _apply_k(mdp, J, b, k, pi=p), _apply_k(mdp, Jp, b, k, pi=p)
                    assert np.all(BJ <= BJp + 1e-12)                                   # monotonicity
                    r = abs(float(rng.standard_normal()))
                    Bs = _apply_k(mdp, J + r, b, k, pi=p)
                    if b == mdp.n:                                                     # shift, b = n
                        assert np.max(np.abs(Bs - (BJ + a ** k * r))) < 1e-7
                    # b < n: the shift lemma's equality does not hold (its induction step shifts
                    # the already-updated states by r instead of alpha*r); the sandwich does
                    assert np.all(Bs >= BJ - 1e-12) and np.all(Bs <= BJ + a ** k * r + 1e-7)
                    Bn = _apply_k(mdp, J - r, b, k, pi=p)
                    assert np.all(Bn <= BJ + 1e-12) and np.all(Bn >= BJ - a ** k * r - 1e-7)
                    Jq = rng.standard_normal(mdp.n)
                    lhs = np.max(np.abs(BJ - _apply_k(mdp, Jq, b, k, pi=p)))
                    assert lhs <= a ** k * np.max(np.abs(J - Jq)) + 1e-7               # contraction


def test_fixed_point_and_error_bound():
    mdp = mdpgen.csr_uniform_k(400, 5, 8, gamma=0.95, seed=11)
    jstar, pistar, cert = exact.policy_iteration(mdp)
    assert cert < 1e-12
    for b in (1, 16, 400):
        for sweep in (0, 5):
            BJ, _ = oracle.mb_apply(mdp, jstar, b, 3, sweep)
            assert np.max(np.abs(BJ - jstar)) < 1e-11
            Bm, _ = oracle.mb_apply(mdp, exact.policy_value(mdp, pistar), b, 3, sweep, pi=pistar)
            assert np.max(np.abs(Bm - jstar)) < 1e-11
        # the FP32 rows sum to 1 only within ~4e-8: the sweep contracts by gamma * max row sum
        g = mdp.gamma * float(np.add.reduceat(mdp.prob.astype(np.float64), mdp.row_ptr[:-1]).max())
        for eps in (1e-3, 1e-6):
            r = oracle.mbvi(mdp, b, seed=9, eps=eps, max_sweeps=10000)
            d = r["deltas"][-1]
            assert d <= eps
            assert np.max(np.abs(r["V"] - jstar)) <= g / (1 - g) * d + 1e-12


def test_comparison_theorem_divisor_chain():
    """J=0 with costs >= 0 gives J <= TJ <= J*; then B_b^k J <= B_b'^k J <= J* for b' | b, and
    T^k J <= B_b^k J <= F^k J (Sec. III-B.2), sweep by sweep with a shared permutation sequence."""
    mdp = mdpgen.csr_uniform_k(256, 4, 6, gamma=0.95, seed=21)
    jstar, _, _ = exact.policy_iteration(mdp)
    J = np.zeros(mdp.n)
    chain = [256, 64, 16, 4, 1]
    V = {b: J.copy() for b in chain}
    for sweep in range(25):
        for b in chain:
            V[b], _ = oracle.mb_apply(mdp, V[b], b, 4242, sweep)
        for big, small in zip(chain[:-1], chain[1:]):
            assert np.all(V[big] <= V[small] + 1e-12), (sweep, big, small)
        assert np.all(V[1] <= jstar + 1e-12)
    # the inequality is strict somewhere: smaller batches converge faster here
    assert np.max(V[1] - V[256]) > 1e-3


def test_mpi_matches_policy_iteration():
    for mdp in (mdpgen.csr_uniform_k(300, 4, 8, gamma=0.95, seed=13), mdpgen.dense_dirichlet(60, 3, gamma=0.9, seed=1)):
        jstar, pistar, _ = exact.policy_iteration(mdp)
        for b in (1, 17, mdp.n):
            r = oracle.mpi(mdp, b, K=10, seed=5, eps=1e-10, max_iters=10000)
            assert r["resid"][-1] <= 1e-10
            assert np.max(np.abs(r["V"] - jstar)) < 1e-8
            _, _, gap, _ = exact.bellman_pass(mdp, jstar)
            sel = gap > 1e-6
            assert np.array_equal(r["pi"][sel], pistar[sel])
            assert r["sweeps"] == 10 * (r["iters"] - 1)


def test_inadmissible_actions_are_never_chosen():
    mdp = mdpgen.csr_ragged(40, 4, 5, gamma=0.9, seed=3, inadmissible_frac=0.5)
    r = oracle.mbvi(mdp, 8, seed=1, eps=1e-12, max_sweeps=10000)
    _, pi, _, _ = oracle.greedy(mdp, r["V"])
    assert np.all(np.isfinite(mdp.cost[np.arange(mdp.n) * mdp.m + pi]))
    jstar, _, _ = exact.policy_iteration(mdp)
    assert np.max(np.abs(r["V"] - jstar)) < 1e-9


def test_mpi_first_outer_iteration_closed_form():
    """Alg. 1 from J = 0: the improvement step picks mu0 = argmin_u g(i,u) (J = 0), then K sweeps
    of B_{mu0,n} = T_mu0 give sum_{t<K} alpha^t P_mu0^t g_mu0 (eq. (6) iterated)."""
    mdp = mdpgen.csr_uniform_k(150, 4, 6, gamma=0.9, seed=31)
    c = mdp.cost.reshape(mdp.n, mdp.m).astype(np.float64)
    mu0 = np.argmin(c, axis=1).astype(np.int32)
    Pm, g = exact.policy_matrix(mdp, mu0)
    K = 7
    want, term = np.zeros(mdp.n), g.copy()
    for t in range(K):
        want += term
        term = mdp.gamma * (Pm @ term)
    r = oracle.mpi(mdp, mdp.n, K=K, seed=1, eps=0.0, max_iters=2)
    assert r["iters"] == 2 and r["sweeps"] == K
    assert np.max(np.abs(r["V"] - want)) < 1e-12
    # with b < n the first sweep of B_{mu0,b} still starts from J = 0: the first batch equals g_mu0
    r1 = oracle.mpi(mdp, 10, K=1, seed=1, eps=0.0, max_iters=2)
    first = oracle.perm(mdp.n, 1, 0)[:10]
    assert np.max(np.abs(r1["V"][first] - g[first])) < 1e-15


def test_greedy_ties_resolve_to_lowest_action():
    """Exact ties (duplicated actions) resolve to the lowest action index, with Q-gap 0."""
    base = mdpgen.dense_dirichlet(30, 3, seed=5)
    P = base.P.copy()
    c = base.cost.reshape(30, 3).copy()
    P[:, 2] = P[:, 1]
    c[:, 2] = c[:, 1]          # action 2 duplicates action 1
    P[:, 0] = P[:, 1]
    c[:, 0] = c[:, 1] + 1.0    # action 0 is strictly worse
    mdp = mdpgen.MDP(n=30, m=3, gamma=0.9, fmt="dense", cost=c.reshape(-1), P=P)
    V = mdpgen.random_values(30, seed=1).astype(np.float64)
    TV, pi, gap, _ = oracle.greedy(mdp, V)
    assert np.all(pi == 1) and np.all(gap == 0)
    r = oracle.mpi(mdp, 7, K=3, seed=2, eps=1e-10, max_iters=1000)
    assert np.all(r["pi"] == 1)


# ----------------------------------------------------------------------------------------------
# Batch selection with replacement (the extension of Sec. V): uniform draws and draws by integer
# weights, pinned against the draw rule written out with Python integers, against each other, by
# frequency, against the batch-by-batch definition, and against J* through the stop rule.
# ----------------------------------------------------------------------------------------------
def _draws_by_definition(n, seed, sweep, select, weights=None):
    """u = x0 * 2^32 + x1 of Philox4x32-10(ctr = {p, 2^31, k_lo, k_hi}, key = {seed_lo, seed_hi});
    uniform: floor(u n / 2^64); weighted: r = floor(u W / 2^64), the first s whose cumulative
    weight exceeds r."""
    import bisect
    import itertools
    key = [seed & 0xFFFFFFFF, seed >> 32]
    cum = list(itertools.accumulate(int(w) for w in weights)) if select == 2 else None
    out = []
    for p in range(n):
        x = oracle.philox4x32_10([p, 1 << 31, sweep & 0xFFFFFFFF, sweep >> 32], key)
        u = (int(x[0]) << 32) | int(x[1])
        if select == 1:
            out.append((u * n) >> 64)
        else:
            out.append(bisect.bisect_right(cum, (u * cum[-1]) >> 64))
    return np.array(out, dtype=np.int64)


def test_draws_follow_their_definition():
    g = np.random.default_rng(5)
    for n, seed, sweep in ((1, 3, 0), (7, 12345, 2), (300, 2**40 + 7, 2**33 + 1)):
        assert np.array_equal(oracle.sweep_order(n, seed, sweep, 1), _draws_by_definition(n, seed, sweep, 1))
        w = g.integers(0, 50, size=n).astype(np.uint32)
        w[0] = max(int(w[0]), 1)
        got = oracle.sweep_order(n, seed, sweep, 2, w)
        assert np.array_equal(got, _draws_by_definition(n, seed, sweep, 2, w))
        assert (w[got] > 0).all()


def test_constant_weights_reproduce_uniform_draws():
    # floor(floor(u n c / 2^64) / c) = floor(u n / 2^64): any constant weight gives the uniform draws
    for n in (1, 7, 1000):
        for c in (1, 3, (2**32 - 1) // n):
            w = np.full(n, c, dtype=np.uint32)
            for sweep in (0, 5):
                assert np.array_equal(oracle.sweep_order(n, 99, sweep, 2, w), oracle.sweep_order(n, 99, sweep, 1))


def test_weighted_draw_frequencies():
    w = np.arange(8, dtype=np.uint32) * 3                  # state 0 has weight 0
    counts = np.zeros(8)
    for sweep in range(500):
        counts += np.bincount(oracle.sweep_order(8, 4242, sweep, 2, w), minlength=8)
    assert counts[0] == 0
    expect = counts.sum() * w[1:] / w.sum()
    chi2 = float(((counts[1:] - expect) ** 2 / expect).sum())
    assert chi2 < 22.46                                      # 6 dof, p = 0.001
    u = np.zeros(8)
    for sweep in range(500):
        u += np.bincount(oracle.sweep_order(8, 4242, sweep, 1), minlength=8)
    assert float(((u - 500) ** 2 / 500).sum()) < 24.32       # 7 dof, p = 0.001


def _definition_draws(mdp, J, b, order):
    """One sweep over an order with repeats: batch by batch, every state of the batch takes
    min_a [g + gamma sum_j p_j V(j)] at the values before the batch, then the batch writes."""
    V = [float(x) for x in J]
    n, m = mdp.n, mdp.m
    for t0 in range(0, n, b):
        new = {}
        for s in (int(x) for x in order[t0:t0 + b]):
            vals = []
            for a in range(m):
                r = s * m + a
                g = float(mdp.cost[r])
                if np.isinf(g):
                    vals.append(np.inf)
                    continue
                if mdp.fmt == "dense":
                    succ = [(j, float(mdp.P[s, a, j])) for j in range(n)]
                else:
                    succ = [(int(mdp.col[e]), float(mdp.prob[e])) for e in range(mdp.row_ptr[r], mdp.row_ptr[r + 1])]
                vals.append(g + sum(mdp.gamma * p * V[j] for j, p in succ))
            new[s] = min(vals)
        for s, v in new.items():
            V[s] = v
    return np.array(V)


@pytest.mark.parametrize("idx", [0, 1, 6])
def test_with_replacement_sweep_matches_definition(idx):
    mdp = _tiny_mdps()[idx]
    J = mdpgen.random_values(mdp.n, seed=idx).astype(np.float64)
    w = (np.arange(mdp.n, dtype=np.uint32) % 3) + 1
    for b in range(1, mdp.n + 1):
        for select in (1, 2):
            for sweep in (0, 4):
                order = oracle.sweep_order(mdp.n, 77, sweep, select, w)
                r = oracle.mbvi(mdp, b, 77, eps=0.0, max_sweeps=1, V0=J, start_sweep=sweep, select=select,
                                weights=w)
                assert np.allclose(r["V"], _definition_draws(mdp, J, b, order), rtol=0, atol=1e-12)


def test_with_replacement_converges_under_the_stop_rule():
    mdp = mdpgen.csr_uniform_k(300, 4, 8, gamma=0.9, seed=13)
    jstar, _, _ = exact.policy_iteration(mdp)
    w = mdpgen._rng(3).integers(1, 20, size=mdp.n).astype(np.uint32)
    for select in (1, 2):
        for b in (1, 16, 300):
            r = oracle.mbvi(mdp, b, 5, eps=1e-9, max_sweeps=100000, select=select, weights=w)
            resid = float(np.max(np.abs(exact.bellman_pass(mdp, r["V"])[0] - r["V"])))
            assert resid <= 1e-9 and abs(resid - r["resid"]) < 1e-12
            assert np.max(np.abs(r["V"] - jstar)) <= 0.9 / 0.1 * resid + 1e-12
        m = oracle.mpi(mdp, 16, K=5, seed=2, eps=1e-10, select=select, weights=w)
        assert m["resid"][-1] <= 1e-10 and np.max(np.abs(m["V"] - jstar)) < 1e-8


def test_bellman_residual_stop_rule():
    """residual_kind 1: a sweep change <= eps is confirmed by ||TV - V||_inf <= eps (eq. (7))."""
    mdp = mdpgen.csr_uniform_k(300, 4, 8, gamma=0.95, seed=17)
    for b in (1, 30, 300):
        r0 = oracle.mbvi(mdp, b, 5, eps=1e-8, max_sweeps=100000)
        r1 = oracle.mbvi(mdp, b, 5, eps=1e-8, max_sweeps=100000, residual_kind=1)
        full0 = float(np.max(np.abs(exact.bellman_pass(mdp, r0["V"])[0] - r0["V"])))
        full1 = float(np.max(np.abs(exact.bellman_pass(mdp, r1["V"])[0] - r1["V"])))
        assert full1 <= 1e-8 and abs(full1 - r1["resid"]) < 1e-13
        assert r1["sweeps"] >= r0["sweeps"]
        # the sweep-change rule can stop with a larger full residual; the trajectories agree up to there
        assert np.array_equal(r1["deltas"][:r0["sweeps"]], r0["deltas"])
        assert full0 >= 0.0


# ------------------------------------------------------------------------------------------------
# The dense certificate (exact policy iteration over rows read in chunks), used at n = 16384 where
# the transition rows (17 GB) never sit in host memory at once.
def _dense_accessors(mdp):
    R = mdp.P.reshape(mdp.n * mdp.m, mdp.n)
    return (lambda r0, r1: R[r0:r1]), (lambda idx: R[np.asarray(idx)])


def _peaked_tiny(seed):
    # the n = 16384 recipe in miniature: Dirichlet(0.1) rows, N(0,1) costs, gamma = 0.999
    return mdpgen.dense_dirichlet(6, 3, alpha=0.1, gamma=0.999, seed=40 + seed, cost_dist="normal")


def test_dense_policy_iteration_matches_brute_force(ex=exact):
    for seed in range(4):
        mdp = _peaked_tiny(seed)
        rows_of, rows_at = _dense_accessors(mdp)
        jstar = exact.brute_force(mdp)
        for chunk in (1, 4, 6):
            r = ex.dense_policy_iteration(rows_of, rows_at, mdp.cost, mdp.gamma, mdp.n, mdp.m, chunk_states=chunk)
            assert np.max(np.abs(r["J"] - jstar)) <= 1e-9 * np.abs(jstar).max(), (seed, chunk)
            assert r["resid"] <= 1e-10 * np.abs(jstar).max()
            J_pi = exact.policy_value(mdp, r["pi"])
            assert np.max(np.abs(J_pi - jstar)) <= 1e-9 * np.abs(jstar).max()


def test_dense_policy_iteration_matches_converged_mbvi(ex=exact):
    """Against the C oracle's MB-VI run to its FP64 floor (independent code), from any start policy."""
    mdp = mdpgen.dense_dirichlet(300, 5, alpha=0.1, gamma=0.99, seed=12, cost_dist="normal")
    rows_of, rows_at = _dense_accessors(mdp)
    ref = oracle.mbvi(mdp, mdp.n, seed=1, eps=1e-12, max_sweeps=100000)
    scale = np.abs(ref["V"]).max()
    _, pi_ref, gap_ref, _ = oracle.greedy(mdp, ref["V"])
    for pi0 in (None, np.random.default_rng(3).integers(0, mdp.m, mdp.n)):
        r = ex.dense_policy_iteration(rows_of, rows_at, mdp.cost, mdp.gamma, mdp.n, mdp.m, pi0=pi0, chunk_states=37)
        assert np.max(np.abs(r["J"] - ref["V"])) <= 1e-9 * scale
        clear = gap_ref > 1e-8 * scale
        assert np.array_equal(r["pi"][clear], pi_ref[clear])
        assert np.allclose(r["gap"][clear], gap_ref[clear], rtol=1e-6, atol=1e-8 * scale)


def test_dense_bellman_pass_matches_the_oracle(ex=exact):
    mdp = mdpgen.dense_dirichlet(50, 4, alpha=0.1, gamma=0.999, seed=13, cost_dist="normal")
    rows_of, _ = _dense_accessors(mdp)
    J = mdpgen.random_values(mdp.n, seed=2).astype(np.float64) * 30
    TJ_ref, _, _, _ = oracle.greedy(mdp, J)
    for chunk in (1, 7, 50):
        TJ, Q = ex.dense_bellman_pass(rows_of, mdp.cost, mdp.gamma, J, mdp.n, mdp.m, chunk)
        assert np.max(np.abs(TJ - TJ_ref)) <= 1e-12 * np.abs(TJ_ref).max()
        assert np.max(np.abs(Q[7] - [oracle.q_factor(mdp, 7, a, J) for a in range(mdp.m)])) <= 1e-12 * 100

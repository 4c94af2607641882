"""Closed forms that pin the iterative oracle (TEST INFRASTRUCTURE ONLY).

* ``policy_value``: J_mu from the Bellman equation for mu (eq. (4)) as the linear system
  (I - alpha P_mu) J = g_mu, solved directly (LAPACK / SuperLU) or, for large sparse chains,
  by GMRES to a 1e-14 relative residual (the system's inf-norm condition is <= (1+alpha)/(1-alpha)).
* ``brute_force``: J* = min over all deterministic stationary policies of J_mu (eq. (2)), by
  enumeration on tiny problems (m^n policies).
* ``policy_iteration``: exact PI (Sec. II-C) with direct solves, ending when the greedy policy of
  J_mu is mu itself; its result is certified by one Bellman pass (J = TJ, eq. (5)).
* ``dense_policy_iteration``: the same PI for dense transition rows that are too large to hold in
  host memory at once (they are read in row chunks from a caller-supplied accessor); the policy
  solve is a dense LU of (I - alpha P_mu) and every Bellman pass streams all rows once.

Everything here is numpy/scipy FP64 and is independent of ``oracle.c``.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _rows(mdp, pi):
    return np.arange(mdp.n, dtype=np.int64) * mdp.m + np.asarray(pi, dtype=np.int64)


def policy_matrix(mdp, pi):
    """(P_mu, g_mu): the transition matrix and stage costs under the policy mu = pi."""
    rows = _rows(mdp, pi)
    g = mdp.cost.astype(np.float64)[rows]
    if mdp.fmt == "dense":
        Pm = mdp.P.reshape(mdp.n * mdp.m, mdp.n)[rows].astype(np.float64)
        return Pm, g
    rp = mdp.row_ptr
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    idx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    indptr = np.zeros(mdp.n + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    Pm = sp.csr_matrix((mdp.prob[idx].astype(np.float64), mdp.col[idx].astype(np.int64), indptr),
                       shape=(mdp.n, mdp.n))
    return Pm, g


def policy_value(mdp, pi, method: str = "auto"):
    """Exact J_mu = (I - alpha P_mu)^{-1} g_mu (eq. (4))."""
    Pm, g = policy_matrix(mdp, pi)
    if np.isinf(g).any():
        raise ValueError("policy uses an inadmissible action")
    n = mdp.n
    a = float(mdp.gamma)
    if sp.issparse(Pm):
        A = (sp.identity(n, format="csr") - a * Pm).tocsc()
        # sparse LU fills in badly on random successor structure: GMRES beyond small n
        if method == "gmres" or (method == "auto" and n > 1000):
            return _gmres(A, g)
        return spla.spsolve(A, g)
    A = np.eye(n) - a * Pm
    return np.linalg.solve(A, g)


def bellman_pass(mdp, J):
    """Vectorised Bellman pass (eq. (7)): returns (TJ, greedy policy, Q-gap, Q[n,m])."""
    J = np.asarray(J, dtype=np.float64)
    c = mdp.cost.astype(np.float64).reshape(mdp.n, mdp.m)
    if mdp.fmt == "dense":
        PJ = mdp.P.reshape(mdp.n * mdp.m, mdp.n).astype(np.float64) @ J
    else:
        A = sp.csr_matrix((mdp.prob.astype(np.float64), mdp.col.astype(np.int64), mdp.row_ptr),
                          shape=(mdp.n * mdp.m, mdp.n))
        PJ = A @ J
    Q = c + mdp.gamma * PJ.reshape(mdp.n, mdp.m)
    Q = np.where(np.isinf(c), np.inf, Q)
    order = np.argsort(Q, axis=1, kind="stable")
    pi = order[:, 0].astype(np.int32)
    TJ = Q[np.arange(mdp.n), pi]
    if mdp.m > 1:
        gap = Q[np.arange(mdp.n), order[:, 1]] - TJ
    else:
        gap = np.full(mdp.n, np.inf)
    return TJ, pi, gap, Q


def brute_force(mdp):
    """J* by enumerating every admissible deterministic policy (tiny problems only)."""
    n, m = mdp.n, mdp.m
    if m ** n > 20000:
        raise ValueError("too many policies for brute force")
    c = mdp.cost.reshape(n, m)
    best = np.full(n, np.inf)
    for pol in itertools.product(range(m), repeat=n):
        pi = np.array(pol, dtype=np.int32)
        if np.isinf(c[np.arange(n), pi]).any():
            continue
        J = policy_value(mdp, pi)
        best = np.minimum(best, J)
    return best


def policy_iteration(mdp, max_iters: int = 200):
    """Exact PI with direct solves; returns (J*, pi*, ||T J* - J*||_inf)."""
    c = mdp.cost.reshape(mdp.n, mdp.m)
    pi = np.argmin(np.where(np.isinf(c), np.inf, c), axis=1).astype(np.int32)
    for _ in range(max_iters):
        J = policy_value(mdp, pi)
        TJ, new_pi, gap, Q = bellman_pass(mdp, J)
        # keep the current action when it ties the minimum up to the rounding of the policy solve
        # (symmetric moves give exact ties; an iterative solve can tip them either way and cycle)
        tie = 1e-11 * max(1.0, float(np.max(np.abs(J))))
        keep = Q[np.arange(mdp.n), pi] <= TJ + tie
        new_pi = np.where(keep, pi, new_pi).astype(np.int32)
        if np.array_equal(new_pi, pi):
            return J, pi, float(np.max(np.abs(TJ - J)))
        pi = new_pi
    raise RuntimeError("policy iteration did not terminate")


def dense_bellman_pass(rows_of, cost, gamma, J, n, m, chunk_states=512):
    """One FP64 Bellman pass (eq. (7)) over dense rows read in chunks: rows_of(r0, r1) returns the
    rows r0..r1-1 (row r = s*m + a, each of length n, any float dtype).  Returns (TJ, Q [n, m])."""
    J = np.asarray(J, dtype=np.float64)
    c = np.asarray(cost, dtype=np.float64).reshape(n, m)
    Q = np.empty((n, m), dtype=np.float64)
    for s0 in range(0, n, chunk_states):
        s1 = min(n, s0 + chunk_states)
        R = np.asarray(rows_of(s0 * m, s1 * m), dtype=np.float64).reshape((s1 - s0) * m, n)
        Q[s0:s1] = c[s0:s1] + gamma * (R @ J).reshape(s1 - s0, m)
    Q = np.where(np.isinf(c), np.inf, Q)
    return Q.min(axis=1), Q


def dense_policy_iteration(rows_of, rows_at, cost, gamma, n, m, pi0=None, chunk_states=512, max_iters=100):
    """Exact policy iteration (Sec. II-C) for a dense MDP whose rows come from accessors:
    rows_of(r0, r1) -> rows r0..r1-1 and rows_at(idx) -> the rows with the given indices.
    Evaluation: J_mu = (I - alpha P_mu)^{-1} g_mu by a dense LU (eq. (4)); improvement: the greedy
    policy of J_mu, keeping the current action where it ties the minimum up to the rounding of the
    solve.  Ends when the policy repeats; then T J = J (eq. (5)) certifies J = J*.
    Returns dict(J, pi, resid = ||TJ - J||_inf, gap = second smallest minus smallest Q, iters)."""
    c = np.asarray(cost, dtype=np.float64).reshape(n, m)
    if pi0 is None:
        pi = np.argmin(np.where(np.isinf(c), np.inf, c), axis=1).astype(np.int64)
    else:
        pi = np.asarray(pi0, dtype=np.int64).copy()
    states = np.arange(n, dtype=np.int64)
    for it in range(1, max_iters + 1):
        g = c[states, pi]
        if np.isinf(g).any():
            raise ValueError("policy uses an inadmissible action")
        A = np.asarray(rows_at(states * m + pi), dtype=np.float64).reshape(n, n)
        A *= -gamma
        A[states, states] += 1.0
        J = np.linalg.solve(A, g)
        del A
        TJ, Q = dense_bellman_pass(rows_of, cost, gamma, J, n, m, chunk_states)
        tie = 1e-11 * max(1.0, float(np.max(np.abs(J))))
        keep = Q[states, pi] <= TJ + tie
        new_pi = np.where(keep, pi, np.argmin(Q, axis=1))
        if np.array_equal(new_pi, pi):
            part = np.sort(Q, axis=1)
            gap = part[:, 1] - part[:, 0] if m > 1 else np.full(n, np.inf)
            return {"J": J, "pi": pi.astype(np.int32), "resid": float(np.max(np.abs(TJ - J))), "gap": gap,
                    "iters": it}
        pi = new_pi
    raise RuntimeError("policy iteration did not terminate")


def softmax_rows(logits, row_ptr):
    """P(.|s,a) = softmax of the row's logits over its successors, in FP64."""
    z = np.asarray(logits, dtype=np.float64)
    rows = len(row_ptr) - 1
    if rows and len(z) % rows == 0 and np.array_equal(row_ptr, np.arange(rows + 1) * (len(z) // rows)):
        zz = z.reshape(rows, -1)
        e = np.exp(zz - zz.max(axis=1, keepdims=True))
        return (e / e.sum(axis=1, keepdims=True)).reshape(-1)
    out = np.empty_like(z)
    for r in range(rows):
        a, b = int(row_ptr[r]), int(row_ptr[r + 1])
        e = np.exp(z[a:b] - z[a:b].max())
        out[a:b] = e / e.sum()
    return out


def fixed_point_gradient(mdp, w, jstar=None, pistar=None):
    """Gradient of L = w . J* (implicit function theorem on the Bellman equation, eq. (5), at a policy
    mu* with no ties):  J* = g_mu + alpha P_mu J*  =>  lambda solves (I - alpha P_mu)^T lambda = w,
      dL/dg(s,a)   = lambda(s) [a = mu(s)],
      dL/dz(s,a,t) = alpha lambda(s) [a = mu(s)] p_t (J*(j_t) - sum_u p_u J*(j_u))   (p = softmax(z)).
    Returns (lambda, dL/dcost [n*m], dL/dlogits [nnz] (CSR only), J*, mu*)."""
    if jstar is None or pistar is None:
        jstar, pistar, _ = policy_iteration(mdp)
    Pm, _ = policy_matrix(mdp, pistar)
    n = mdp.n
    w = np.asarray(w, dtype=np.float64)
    if sp.issparse(Pm):
        A = (sp.identity(n, format="csr") - mdp.gamma * Pm).T.tocsc()
        lam = spla.spsolve(A, w) if n <= 1000 else _gmres(A, w)
    else:
        lam = np.linalg.solve((np.eye(n) - mdp.gamma * Pm).T, w)
    gc = np.zeros(n * mdp.m)
    rows = np.arange(n, dtype=np.int64) * mdp.m + pistar
    gc[rows] = lam
    gz = None
    if mdp.fmt == "csr":
        gz = np.zeros(int(mdp.row_ptr[-1]))
        p = mdp.prob.astype(np.float64)
        k = int(mdp.row_ptr[-1]) // (n * mdp.m) if n * mdp.m else 0
        if k and np.array_equal(mdp.row_ptr, np.arange(n * mdp.m + 1) * k):
            idx = rows[:, None] * k + np.arange(k)[None, :]
            pv = p[idx]
            jv = jstar[mdp.col[idx]]
            gz[idx] = mdp.gamma * lam[:, None] * pv * (jv - (pv * jv).sum(axis=1, keepdims=True))
            return lam, gc, gz, jstar, pistar
        for s in range(n):
            r = int(rows[s])
            a, b = int(mdp.row_ptr[r]), int(mdp.row_ptr[r + 1])
            pv = p[a:b]
            jv = jstar[mdp.col[a:b]]
            gz[a:b] = mdp.gamma * lam[s] * pv * (jv - pv @ jv)
    return lam, gc, gz, jstar, pistar


def _gmres(A, b):
    """GMRES to a 1e-14 relative residual; (I - alpha P) has inf-norm condition <= (1+alpha)/(1-alpha)."""
    x, info = spla.gmres(A, b, rtol=1e-14, atol=0.0, restart=200, maxiter=10000)
    if info != 0:
        raise RuntimeError(f"gmres did not converge (info={info})")
    return x

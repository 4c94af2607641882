"""FP64 CPU oracle for the randomized mini-batch operator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product path (``paper_2110_02901_b300``) never imports it and shares no code
with it; the two meet only through the seeded generators of ``mdpgen``.

Two parts:
  * ``oracle.c`` (loaded here with ctypes): the mini-batch operator B_b / B_{pi,b} of eqs. (11)-(12)
    with the per-sweep random re-indexing of Sec. III-A, MB-VI, MB-MPI (Alg. 1), the greedy pass,
    Philox4x32-10 and the Feistel permutation, batch selection with replacement (uniform or by
    integer weights, the Sec. V extension), all in FP64;
  * ``exact.py``: closed forms from linear algebra (policy values by direct solve, brute force over
    all deterministic policies, optimality certificates) used to pin the iterative part.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

_LIB = None


class _OrcMDP(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("m", ctypes.c_int32), ("dense", ctypes.c_int32),
        ("P", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("prob", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("gamma", ctypes.c_double),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i64, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_perm.argtypes = [i64, u64, u64, i64]
        L.orc_perm.restype = i64
        L.orc_perm_all.argtypes = [i64, u64, u64, vp]
        L.orc_perm_half_bits.argtypes = [i64]
        L.orc_perm_half_bits.restype = ctypes.c_int
        L.orc_q.argtypes = [P(_OrcMDP), i64, i32, vp]
        L.orc_q.restype = f64
        L.orc_greedy.argtypes = [P(_OrcMDP), vp, vp, vp, vp]
        L.orc_greedy.restype = f64
        L.orc_mb_apply.argtypes = [P(_OrcMDP), vp, i64, u64, u64, vp, vp, vp]
        L.orc_mb_apply.restype = f64
        L.orc_mbvi.argtypes = [P(_OrcMDP), vp, i64, u64, i64, f64, i64, vp, vp, vp]
        L.orc_mbvi.restype = i64
        L.orc_mpi.argtypes = [P(_OrcMDP), i64, i32, u64, i64, f64, i64, vp, vp, vp, vp]
        L.orc_mpi.restype = i64
        L.orc_sweep_order.argtypes = [i64, u64, u64, i32, vp, vp]
        L.orc_sweep_order.restype = ctypes.c_int
        L.orc_mbvi_select.argtypes = [P(_OrcMDP), vp, i64, u64, i64, f64, i64, i32, vp, i32, vp, vp, vp, vp]
        L.orc_mbvi_select.restype = i64
        L.orc_mpi_select.argtypes = [P(_OrcMDP), i64, i32, u64, i64, f64, i64, i32, vp, vp, vp, vp, vp]
        L.orc_mpi_select.restype = i64
        L.orc_bellman_T.argtypes = [P(_OrcMDP), vp, vp]
        L.orc_gauss_seidel_F.argtypes = [P(_OrcMDP), vp, vp]
        L.orc_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Holds the ctypes view of an MDP and keeps its arrays alive."""

    def __init__(self, mdp):
        self.mdp = mdp
        self.cost = np.ascontiguousarray(mdp.cost, dtype=np.float32)
        s = _OrcMDP()
        s.n, s.m, s.gamma = int(mdp.n), int(mdp.m), float(mdp.gamma)
        s.cost = _ptr(self.cost)
        if mdp.fmt == "dense":
            self.P = np.ascontiguousarray(mdp.P, dtype=np.float32)
            s.dense, s.P = 1, _ptr(self.P)
        else:
            self.row_ptr = np.ascontiguousarray(mdp.row_ptr, dtype=np.int64)
            self.col = np.ascontiguousarray(mdp.col, dtype=np.int32)
            self.prob = np.ascontiguousarray(mdp.prob, dtype=np.float32)
            s.dense = 0
            s.row_ptr, s.col, s.prob = _ptr(self.row_ptr), _ptr(self.col), _ptr(self.prob)
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


_BOUND_CACHE = {}


def _bind(mdp) -> _Bound:
    key = id(mdp)
    b = _BOUND_CACHE.get(key)
    if b is None or b.mdp is not mdp:
        b = _Bound(mdp)
        _BOUND_CACHE.clear()
        _BOUND_CACHE[key] = b
    return b


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------------------------------
# Philox / permutation
# ----------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def perm_half_bits(n: int) -> int:
    return int(lib().orc_perm_half_bits(int(n)))


def perm(n: int, seed: int, sweep: int) -> np.ndarray:
    """sigma_{seed,sweep}(p) for p = 0..n-1 (the processing order of that sweep)."""
    out = np.empty(int(n), dtype=np.int64)
    lib().orc_perm_all(int(n), int(seed), int(sweep), _ptr(out))
    return out


def perm_at(n: int, seed: int, sweep: int, p: int) -> int:
    return int(lib().orc_perm(int(n), int(seed), int(sweep), int(p)))


SELECT_PERMUTATION, SELECT_UNIFORM, SELECT_WEIGHTED = 0, 1, 2


def _weights(select: int, weights, n: int):
    if select != SELECT_WEIGHTED:
        return None
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    if w.shape != (n,):
        raise ValueError("weights must be uint32 [n]")
    return w


def sweep_order(n: int, seed: int, sweep: int, select: int = 0, weights=None) -> np.ndarray:
    """States of the n positions of one sweep: sigma (select 0) or draws with replacement (1, 2)."""
    out = np.empty(int(n), dtype=np.int64)
    w = _weights(select, weights, int(n))
    if lib().orc_sweep_order(int(n), int(seed), int(sweep), int(select), _ptr(w), _ptr(out)) != 0:
        raise ValueError("bad select or zero total weight")
    return out


# ----------------------------------------------------------------------------------------------
# Operators and schemes
# ----------------------------------------------------------------------------------------------
def q_factor(mdp, s: int, a: int, J: np.ndarray) -> float:
    B = _bind(mdp)
    J = np.ascontiguousarray(J, dtype=np.float64)
    return float(lib().orc_q(B.ref, int(s), int(a), _ptr(J)))


def greedy(mdp, V: np.ndarray):
    """Full Bellman pass: returns (TV, pi, gap, ||TV - V||_inf)."""
    B = _bind(mdp)
    V = np.ascontiguousarray(V, dtype=np.float64)
    TV = np.empty(mdp.n, dtype=np.float64)
    pi = np.empty(mdp.n, dtype=np.int32)
    gap = np.empty(mdp.n, dtype=np.float64)
    r = lib().orc_greedy(B.ref, _ptr(V), _ptr(TV), _ptr(pi), _ptr(gap))
    return TV, pi, gap, float(r)


def mb_apply(mdp, J: np.ndarray, b: int, seed: int, sweep: int, pi: Optional[np.ndarray] = None):
    """One application of B_b (pi None) or B_{pi,b}; returns (new J, max |change|)."""
    B = _bind(mdp)
    V = np.array(J, dtype=np.float64, copy=True)
    perm_buf = np.empty(mdp.n, dtype=np.int64)
    W = np.empty(max(1, min(int(b), mdp.n)), dtype=np.float64)
    pi_c = None if pi is None else np.ascontiguousarray(pi, dtype=np.int32)
    d = lib().orc_mb_apply(B.ref, _ptr(pi_c), int(b), int(seed), int(sweep), _ptr(V), _ptr(perm_buf), _ptr(W))
    return V, float(d)


def mbvi(mdp, b: int, seed: int, eps: float = 1e-6, max_sweeps: int = 100000, V0=None,
         start_sweep: int = 0, pi: Optional[np.ndarray] = None, traj: bool = False, select: int = 0,
         weights=None, residual_kind: int = 0):
    """MB-VI (pi None) or mini-batch policy evaluation (pi given) until delta <= eps.

    select 1 / 2: batches drawn with replacement (uniform / by the uint32 weights); there, and with
    residual_kind 1, the stop also needs the full residual <= eps.
    Returns dict(V, sweeps, deltas, resid[, traj]).
    """
    B = _bind(mdp)
    n = mdp.n
    V = np.zeros(n, dtype=np.float64) if V0 is None else np.array(V0, dtype=np.float64, copy=True)
    deltas = np.zeros(int(max_sweeps), dtype=np.float64)
    T = np.zeros((int(max_sweeps), n), dtype=np.float64) if traj else None
    pi_c = None if pi is None else np.ascontiguousarray(pi, dtype=np.int32)
    w = _weights(select, weights, n)
    resid = ctypes.c_double(0.0)
    k = lib().orc_mbvi_select(B.ref, _ptr(pi_c), int(b), int(seed), int(start_sweep), float(eps),
                              int(max_sweeps), int(select), _ptr(w), int(residual_kind), _ptr(V), _ptr(deltas),
                              _ptr(T), ctypes.byref(resid))
    if k < 0:
        raise ValueError("bad select or zero total weight")
    out = {"V": V, "sweeps": int(k), "deltas": deltas[:k], "resid": float(resid.value)}
    if traj:
        out["traj"] = T[:k]
    return out


def eval_policy(mdp, pi, b: int, seed: int, eps: float = 1e-6, max_sweeps: int = 100000, V0=None,
                start_sweep: int = 0, traj: bool = False):
    return mbvi(mdp, b, seed, eps, max_sweeps, V0, start_sweep, pi=pi, traj=traj)


def mpi(mdp, b: int, K: int, seed: int, eps: float = 1e-6, max_iters: int = 100000, V0=None,
        start_sweep: int = 0, select: int = 0, weights=None):
    """MB-MPI (Alg. 1 with B_{pi,b}); returns dict(V, pi, iters, sweeps, resid)."""
    B = _bind(mdp)
    n = mdp.n
    V = np.zeros(n, dtype=np.float64) if V0 is None else np.array(V0, dtype=np.float64, copy=True)
    pi = np.zeros(n, dtype=np.int32)
    sw = ctypes.c_int64(0)
    res = np.zeros(int(max_iters), dtype=np.float64)
    w = _weights(select, weights, n)
    it = lib().orc_mpi_select(B.ref, int(b), int(K), int(seed), int(start_sweep), float(eps), int(max_iters),
                              int(select), _ptr(w), _ptr(V), _ptr(pi), ctypes.byref(sw), _ptr(res))
    if it < 0:
        raise ValueError("bad select or zero total weight")
    return {"V": V, "pi": pi, "iters": int(it), "sweeps": int(sw.value), "resid": res[:it]}


def bellman_T(mdp, J):
    B = _bind(mdp)
    J = np.ascontiguousarray(J, dtype=np.float64)
    out = np.empty(mdp.n, dtype=np.float64)
    lib().orc_bellman_T(B.ref, _ptr(J), _ptr(out))
    return out


def gauss_seidel_F(mdp, order, J):
    B = _bind(mdp)
    V = np.array(J, dtype=np.float64, copy=True)
    o = np.ascontiguousarray(order, dtype=np.int64)
    lib().orc_gauss_seidel_F(B.ref, _ptr(o), _ptr(V))
    return V


from . import exact  # noqa: E402  (closed forms; numpy/scipy only)

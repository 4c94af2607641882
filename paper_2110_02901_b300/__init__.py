"""Python binding of librmb (include/rmb.h): the randomized mini-batch operator on a B300.

Thin ctypes marshalling only: every step of a solve runs in the CUDA kernels of ``librmb.so``.
PyTorch supplies device memory and streams.  The C entry points keep their names here
(``rmb_vi``, ``rmb_mpi``, ``rmb_eval_policy``, ``rmb_greedy``, ``rmb_permutation``,
``rmb_validate``, ``rmb_workspace_bytes``, ``rmb_status_string``); they take torch CUDA tensors.

There is no CPU fallback: if ``librmb.so`` is missing or cannot be loaded, importing the library
handle raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librmb.so")

RMB_OK = 0
RMB_ERR_ARG = -1
RMB_ERR_CUDA = -2
RMB_ERR_NOT_CONVERGED = -3
RMB_ERR_BARRIER_TIMEOUT = -4
RMB_ERR_INVALID_MDP = -5
RMB_ERR_WORKSPACE = -6
RMB_ERR_UNSUPPORTED = -7
RMB_ERR_NONFINITE = -8
RMB_ERR_TOO_LARGE = -9
RMB_NOALLOC_SCRATCH_BYTES = 8 << 20
RMB_DENSE = 0
RMB_CSR = 1
RMB_P_F32 = 0
RMB_P_BF16 = 1
RMB_P_FP8E4M3 = 2
RMB_FLAG_INJECT_BARRIER_STALL = 1
RMB_FLAG_RAW_ROWS = 2
RMB_FLAG_ASYNC = 4
RMB_FLAG_NO_CLUSTER = 8
RMB_SELECT_PERMUTATION, RMB_SELECT_UNIFORM, RMB_SELECT_WEIGHTED = 0, 1, 2
RMB_RESIDUAL_SWEEP, RMB_RESIDUAL_BELLMAN = 0, 1
PATH_NAMES = {0: "dense", 1: "csr-vec", 2: "csr-generic", 3: "dense-tma", 4: "cluster"}


class rmb_mdp(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("m", ctypes.c_int32), ("format", ctypes.c_int32),
        ("P", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("prob", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("gamma", ctypes.c_double),
        ("k_uniform", ctypes.c_int32), ("p_dtype", ctypes.c_int32), ("row_scale", ctypes.c_void_p),
    ]


class rmb_opts(ctypes.Structure):
    _fields_ = [
        ("batch", ctypes.c_int64), ("seed", ctypes.c_uint64), ("eps", ctypes.c_double),
        ("max_sweeps", ctypes.c_int64), ("start_sweep", ctypes.c_int64),
        ("eval_sweeps", ctypes.c_int32), ("validate", ctypes.c_int32),
        ("barrier_timeout_ns", ctypes.c_int64), ("grid_ctas", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("trace", ctypes.c_void_p),
        ("select", ctypes.c_int32), ("residual_kind", ctypes.c_int32), ("weights", ctypes.c_void_p),
    ]


class rmb_stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64), ("iters", ctypes.c_int64), ("barriers", ctypes.c_int64),
        ("residual", ctypes.c_double), ("v_shift", ctypes.c_double), ("status", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32), ("path", ctypes.c_int32), ("lanes_per_state", ctypes.c_int32),
        ("ms", ctypes.c_float), ("batch", ctypes.c_int32), ("start_ms", ctypes.c_float),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["path"] = PATH_NAMES.get(d["path"], d["path"])
        d["status_text"] = rmb_status_string(d["status"])
        return d


class rmb_batch_item(ctypes.Structure):
    _fields_ = [("mdp", rmb_mdp), ("batch", ctypes.c_int64), ("V", ctypes.c_void_p), ("pi", ctypes.c_void_p),
                ("qgap", ctypes.c_void_p)]


class rmb_batch_plan_item(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("group_ctas", ctypes.c_int32), ("first_cta", ctypes.c_int32),
                ("est_ms", ctypes.c_double)]


class rmb_batch_handle(ctypes.Structure):
    _fields_ = [("workspace", ctypes.c_void_p), ("count", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("ntasks", ctypes.c_int32), ("nqueue", ctypes.c_int32), ("ctrl_offset", ctypes.c_int64),
                ("kp_offset", ctypes.c_int64), ("toff_offset", ctypes.c_int64), ("tasks_offset", ctypes.c_int64),
                ("est_ms", ctypes.c_double)]


_LIB = None


def lib():
    """The loaded librmb.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librmb.so not built at {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, vp, sz = ctypes.POINTER, ctypes.c_void_p, ctypes.c_size_t
        L.rmb_workspace_bytes.argtypes = [P(rmb_mdp), P(rmb_opts)]
        L.rmb_workspace_bytes.restype = sz
        L.rmb_vi.argtypes = [P(rmb_mdp), P(rmb_opts), vp, vp, vp, vp, sz, P(rmb_stats), vp]
        L.rmb_mpi.argtypes = [P(rmb_mdp), P(rmb_opts), vp, vp, vp, vp, sz, P(rmb_stats), vp]
        L.rmb_eval_policy.argtypes = [P(rmb_mdp), vp, P(rmb_opts), vp, vp, sz, P(rmb_stats), vp]
        L.rmb_greedy.argtypes = [P(rmb_mdp), P(rmb_opts), vp, vp, vp, vp, vp, sz, P(rmb_stats), vp]
        L.rmb_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, vp, vp]
        L.rmb_validate.argtypes = [P(rmb_mdp), vp, sz, vp]
        L.rmb_status_string.argtypes = [ctypes.c_int]
        L.rmb_status_string.restype = ctypes.c_char_p
        L.rmb_kernel_launches.restype = ctypes.c_uint64
        L.rmb_version.restype = ctypes.c_int
        for f in ("rmb_vi", "rmb_mpi", "rmb_eval_policy", "rmb_greedy", "rmb_permutation", "rmb_validate"):
            getattr(L, f).restype = ctypes.c_int
        _LIB = L
    return _LIB


class RmbError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {rmb_status_string(status)} ({status})")


def rmb_status_string(status: int) -> str:
    return lib().rmb_status_string(int(status)).decode()


def rmb_kernel_launches() -> int:
    return int(lib().rmb_kernel_launches())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _check(t, dtype, n, name):
    import torch
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor with >= {n} elements")


def _check_mdp_tensors(n, m, fmt, cost, P, row_ptr, col, prob, p_dtype, row_scale):
    """The kernels read these arrays as flat, contiguous device memory of the types include/rmb.h
    names; anything else (a strided view, another dtype, a host tensor) is refused here, because the
    C ABI cannot see it.  Values are checked on the device by rmb_validate."""
    import torch
    if fmt not in ("dense", "csr"):
        raise ValueError(f"format must be 'dense' or 'csr', not {fmt!r}")
    if n < 1 or m < 1:
        raise ValueError("need n >= 1 and m >= 1")
    dt = {RMB_P_F32: torch.float32, RMB_P_BF16: torch.bfloat16, RMB_P_FP8E4M3: torch.uint8}.get(p_dtype)
    if dt is None:
        raise ValueError(f"p_dtype {p_dtype} is not one of RMB_P_F32 / RMB_P_BF16 / RMB_P_FP8E4M3")
    _need(cost, torch.float32, n * m, "cost")
    if fmt == "dense":
        if p_dtype == RMB_P_FP8E4M3 and P is not None and P.dtype == getattr(torch, "float8_e4m3fn", None):
            dt = P.dtype                     # e4m3 codes may also come as torch's own fp8 type
        _need(P, dt, n * m * n, "P")
        if row_scale is not None:
            _check(row_scale, torch.float32, n * m, "row_scale")
    else:
        if p_dtype != RMB_P_F32:
            raise ValueError("CSR rows are float32 (p_dtype = RMB_P_F32)")
        _need(row_ptr, torch.int64, n * m + 1, "row_ptr")
        _need(col, torch.int32, 0, "col")
        _need(prob, torch.float32, col.numel(), "prob")


def _need(t, dtype, n, name):
    if t is None:
        raise ValueError(f"{name} is required")
    _check(t, dtype, n, name)


# ----------------------------------------------------------------------------------------------
class DeviceMDP:
    """An MDP resident in device memory (torch tensors) plus its rmb_mdp descriptor."""

    def __init__(self, n, m, gamma, fmt, cost, P=None, row_ptr=None, col=None, prob=None,
                 k_uniform: int = 0, name: str = "", p_dtype: int = 0, row_scale=None):
        self.n, self.m, self.gamma, self.fmt, self.name = int(n), int(m), float(gamma), fmt, name
        self.cost, self.P, self.row_ptr, self.col, self.prob = cost, P, row_ptr, col, prob
        _check_mdp_tensors(self.n, self.m, fmt, cost, P, row_ptr, col, prob, int(p_dtype), row_scale)
        self.k_uniform = int(k_uniform)
        d = rmb_mdp()
        d.n, d.m, d.gamma = self.n, self.m, self.gamma
        d.format = RMB_DENSE if fmt == "dense" else RMB_CSR
        d.cost = _ptr(cost)
        d.P, d.row_ptr, d.col, d.prob = _ptr(P), _ptr(row_ptr), _ptr(col), _ptr(prob)
        d.k_uniform = self.k_uniform
        self.p_dtype, self.row_scale = int(p_dtype), row_scale
        d.p_dtype = self.p_dtype
        d.row_scale = _ptr(row_scale)
        self.desc = d

    @classmethod
    def from_host(cls, mdp, device="cuda", non_blocking=False):
        """Upload an ``mdpgen.MDP`` (numpy arrays) to the device."""
        import torch

        def up(a):
            if a is None:
                return None
            return torch.from_numpy(np.ascontiguousarray(a)).to(device, non_blocking=non_blocking)

        return cls(mdp.n, mdp.m, mdp.gamma, mdp.fmt, up(mdp.cost), P=up(mdp.P), row_ptr=up(mdp.row_ptr),
                   col=up(mdp.col), prob=up(mdp.prob),
                   k_uniform=mdp.uniform_k() if mdp.fmt == "csr" else 0, name=getattr(mdp, "name", ""))

    @property
    def nnz(self) -> int:
        return self.n * self.m * self.n if self.fmt == "dense" else int(self.prob.numel())


@dataclasses.dataclass
class Opts:
    batch: int
    seed: int = 12345
    eps: float = 1e-6
    max_sweeps: int = 100000
    start_sweep: int = 0
    eval_sweeps: int = 10
    validate: bool = True
    barrier_timeout_ns: int = 0
    grid_ctas: int = 0
    flags: int = 0
    trace: object = None       # optional torch float64 CUDA tensor [max_sweeps]
    select: int = 0            # RMB_SELECT_PERMUTATION / _UNIFORM / _WEIGHTED
    weights: object = None     # RMB_SELECT_WEIGHTED: torch int32 (read as uint32) CUDA tensor [n]
    residual_kind: int = 0     # RMB_RESIDUAL_SWEEP / RMB_RESIDUAL_BELLMAN (stop test of rmb_vi)

    def desc(self) -> rmb_opts:
        o = rmb_opts()
        o.batch, o.seed, o.eps = int(self.batch), int(self.seed) & (2 ** 64 - 1), float(self.eps)
        o.max_sweeps, o.start_sweep = int(self.max_sweeps), int(self.start_sweep)
        o.eval_sweeps, o.validate = int(self.eval_sweeps), int(bool(self.validate))
        o.barrier_timeout_ns, o.grid_ctas, o.flags = int(self.barrier_timeout_ns), int(self.grid_ctas), int(self.flags)
        o.trace = _ptr(self.trace)
        o.select = int(self.select)
        o.residual_kind = int(self.residual_kind)
        o.weights = _ptr(self.weights)
        return o


def rmb_workspace_bytes(mdp: DeviceMDP, opts: Opts) -> int:
    o = opts.desc()
    return int(lib().rmb_workspace_bytes(ctypes.byref(mdp.desc), ctypes.byref(o)))


def workspace(mdp: DeviceMDP, opts: Opts, device="cuda"):
    import torch
    nb = rmb_workspace_bytes(mdp, opts)
    if nb == 0:
        raise RmbError(RMB_ERR_ARG, "rmb_workspace_bytes")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def _finish(st: int, stats: Optional[rmb_stats], what: str, allow=(RMB_OK, RMB_ERR_NOT_CONVERGED)):
    if st not in allow:
        raise RmbError(st, what)
    return stats.as_dict() if stats is not None else None


def rmb_vi(mdp: DeviceMDP, opts: Opts, V, pi=None, qgap=None, ws=None, stats: bool = True, stream=None,
           check: bool = True):
    """MB-VI in place on V (float32 [n]); returns the stats dict (or None when stats=False)."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(pi, torch.int32, mdp.n, "pi")
    _check(qgap, torch.float32, mdp.n, "qgap")
    ws = workspace(mdp, opts) if ws is None else ws
    o = opts.desc()
    s = rmb_stats() if stats else None
    st = lib().rmb_vi(ctypes.byref(mdp.desc), ctypes.byref(o), _ptr(V), _ptr(pi), _ptr(qgap), _ptr(ws),
                      ws.numel(), ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    return _finish(st, s, "rmb_vi") if check else (st, s.as_dict() if s is not None else None)


def rmb_mpi(mdp: DeviceMDP, opts: Opts, V, pi, qgap=None, ws=None, stats: bool = True, stream=None,
            check: bool = True):
    """MB-MPI in place on V; pi (int32 [n]) receives the final greedy policy."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(pi, torch.int32, mdp.n, "pi")
    _check(qgap, torch.float32, mdp.n, "qgap")
    ws = workspace(mdp, opts) if ws is None else ws
    o = opts.desc()
    s = rmb_stats() if stats else None
    st = lib().rmb_mpi(ctypes.byref(mdp.desc), ctypes.byref(o), _ptr(V), _ptr(pi), _ptr(qgap), _ptr(ws),
                       ws.numel(), ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    return _finish(st, s, "rmb_mpi") if check else (st, s.as_dict() if s is not None else None)


def rmb_eval_policy(mdp: DeviceMDP, pi, opts: Opts, V, ws=None, stats: bool = True, stream=None,
                    check: bool = True):
    """Mini-batch policy evaluation (B_{pi,b} sweeps) in place on V."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(pi, torch.int32, mdp.n, "pi")
    ws = workspace(mdp, opts) if ws is None else ws
    o = opts.desc()
    s = rmb_stats() if stats else None
    st = lib().rmb_eval_policy(ctypes.byref(mdp.desc), _ptr(pi), ctypes.byref(o), _ptr(V), _ptr(ws), ws.numel(),
                               ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    return _finish(st, s, "rmb_eval_policy") if check else (st, s.as_dict() if s is not None else None)


def rmb_residual_weights(mdp: DeviceMDP, V, floor_frac: float = 0.05, out=None, ws=None, stream=None):
    """Importance weights (uint32 in an int32 tensor [n]) from the Bellman residual at V (see rmb.h)."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    L = lib()
    L.rmb_residual_weights_workspace_bytes.argtypes = [ctypes.POINTER(rmb_mdp)]
    L.rmb_residual_weights_workspace_bytes.restype = ctypes.c_size_t
    L.rmb_residual_weights.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.rmb_residual_weights.restype = ctypes.c_int
    if ws is None:
        nb = int(L.rmb_residual_weights_workspace_bytes(ctypes.byref(mdp.desc)))
        if nb == 0:
            raise RmbError(RMB_ERR_ARG, "rmb_residual_weights_workspace_bytes")
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.empty(mdp.n, dtype=torch.int32, device="cuda") if out is None else out
    _check(out, torch.int32, mdp.n, "weights")
    st = L.rmb_residual_weights(ctypes.byref(mdp.desc), _ptr(V), float(floor_frac), _ptr(out), _ptr(ws), ws.numel(),
                                _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_residual_weights")
    return out


def rmb_vi_prioritized(mdp: DeviceMDP, opts: Opts, V, refresh: int = 4, floor_frac: float = 0.05, pi=None, qgap=None,
                       ws=None, stats: bool = True, stream=None, check: bool = True):
    """MB-VI whose batches are drawn by residual weights, refreshed every `refresh` sweeps (the
    importance-sampled selection suggested in Sec. V); stops when a sweep's change and
    ||TV - V||_inf are <= opts.eps.  Returns the stats dict (iters = rounds)."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(pi, torch.int32, mdp.n, "pi")
    _check(qgap, torch.float32, mdp.n, "qgap")
    L = lib()
    L.rmb_vi_prioritized_workspace_bytes.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_opts)]
    L.rmb_vi_prioritized_workspace_bytes.restype = ctypes.c_size_t
    L.rmb_vi_prioritized.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_opts), ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.POINTER(rmb_stats), ctypes.c_void_p]
    L.rmb_vi_prioritized.restype = ctypes.c_int
    o = opts.desc()
    if ws is None:
        nb = int(L.rmb_vi_prioritized_workspace_bytes(ctypes.byref(mdp.desc), ctypes.byref(o)))
        if nb == 0:
            raise RmbError(RMB_ERR_ARG, "rmb_vi_prioritized_workspace_bytes")
        ws = torch.empty(nb, dtype=torch.uint8, device=V.device)
    s = rmb_stats() if stats else None
    st = L.rmb_vi_prioritized(ctypes.byref(mdp.desc), ctypes.byref(o), int(refresh), float(floor_frac), _ptr(V),
                              _ptr(pi), _ptr(qgap), _ptr(ws), ws.numel(), ctypes.byref(s) if s is not None else None,
                              _stream_handle(stream))
    return _finish(st, s, "rmb_vi_prioritized") if check else (st, s.as_dict() if s is not None else None)


def prioritized_vi(mdp: DeviceMDP, V, batch: int, eps: float, refresh: int = 4, floor_frac: float = 0.05,
                   seed: int = 12345, max_sweeps: int = 1000000, pi=None, stream=None):
    """rmb_vi_prioritized with the options spelled out; returns dict(sweeps, rounds, residual, status)."""
    st = rmb_vi_prioritized(mdp, Opts(batch=batch, seed=seed, eps=eps, max_sweeps=max_sweeps, validate=False), V,
                            refresh=refresh, floor_frac=floor_frac, pi=pi, stream=stream)
    return {"sweeps": st["sweeps"], "rounds": st["iters"], "residual": st["residual"], "status": st["status"],
            "ms": st["ms"]}


def rmb_greedy(mdp: DeviceMDP, V, TV=None, pi=None, qgap=None, opts: Optional[Opts] = None, ws=None,
               stats: bool = True, stream=None, check: bool = True):
    """One Bellman pass at V: TV, greedy policy, Q-gap; stats['residual'] = ||TV - V||_inf."""
    import torch
    opts = opts or Opts(batch=mdp.n)
    _check(V, torch.float32, mdp.n, "V")
    _check(TV, torch.float32, mdp.n, "TV")
    _check(pi, torch.int32, mdp.n, "pi")
    _check(qgap, torch.float32, mdp.n, "qgap")
    ws = workspace(mdp, opts) if ws is None else ws
    o = opts.desc()
    s = rmb_stats() if stats else None
    st = lib().rmb_greedy(ctypes.byref(mdp.desc), ctypes.byref(o), _ptr(V), _ptr(TV), _ptr(pi), _ptr(qgap),
                          _ptr(ws), ws.numel(), ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    return _finish(st, s, "rmb_greedy", allow=(RMB_OK,)) if check else (st, s.as_dict() if s is not None else None)


def rmb_vi_noalloc(mdp: DeviceMDP, opts: Opts, V, pi=None, qgap=None, stats: bool = True, stream=None,
                   check: bool = True):
    """MB-VI in place on V using the library's fixed scratch array instead of a workspace.

    For callers that cannot allocate device memory (see rmb.h): no workspace argument, problems
    needing more than RMB_NOALLOC_SCRATCH_BYTES of scratch are rejected (RMB_ERR_TOO_LARGE), and
    calls that overlap on the GPU race on the shared array.
    """
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(pi, torch.int32, mdp.n, "pi")
    _check(qgap, torch.float32, mdp.n, "qgap")
    f = lib().rmb_vi_noalloc
    f.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_opts), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    o = opts.desc()
    s = rmb_stats() if stats else None
    st = f(ctypes.byref(mdp.desc), ctypes.byref(o), _ptr(V), _ptr(pi), _ptr(qgap),
           ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    return _finish(st, s, "rmb_vi_noalloc") if check else (st, s.as_dict() if s is not None else None)


def rmb_backup_states(mdp: DeviceMDP, V, states, pi=None, out=None, stream=None):
    """W[i] = min_a Q(states[i], a) at V (or Q at pi[states[i]]); float32 CUDA tensors, states int32."""
    import torch
    _check(V, torch.float32, mdp.n, "V")
    _check(states, torch.int32, 0, "states")
    _check(pi, torch.int32, mdp.n, "pi")
    out = torch.empty(states.numel(), dtype=torch.float32, device=V.device) if out is None else out
    _check(out, torch.float32, states.numel(), "out")
    f = lib().rmb_backup_states
    f.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(ctypes.byref(mdp.desc), _ptr(V), _ptr(states), states.numel(), _ptr(pi), _ptr(out), _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_backup_states")
    return out


def rmb_softmax_rows(mdp: DeviceMDP, logits, prob_out, stream=None):
    """prob_out = softmax of each (s,a) row of logits (CSR, uniform k)."""
    import torch
    nnz = mdp.n * mdp.m * mdp.k_uniform
    _check(logits, torch.float32, nnz, "logits")
    _check(prob_out, torch.float32, nnz, "prob_out")
    f = lib().rmb_softmax_rows
    f.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(ctypes.byref(mdp.desc), _ptr(logits), _ptr(prob_out), _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_softmax_rows")
    return prob_out


def rmb_fixed_point_grad(mdp: DeviceMDP, pi, V, w, opts: Opts, lam=None, grad_cost=None, grad_logits=None,
                         want_cost: bool = True, want_logits: bool = True, stats: bool = True, stream=None):
    """Adjoint lambda of (I - gamma P_pi)^T lambda = w and the gradients of w . V* (see rmb.h).
    Returns (lambda, dL/dcost, dL/dlogits, stats)."""
    import torch
    n, m, k = mdp.n, mdp.m, mdp.k_uniform
    dev = V.device
    lam = torch.empty(n, dtype=torch.float32, device=dev) if lam is None else lam
    if want_cost and grad_cost is None:
        grad_cost = torch.empty(n * m, dtype=torch.float32, device=dev)
    if want_logits and grad_logits is None:
        grad_logits = torch.empty(n * m * k, dtype=torch.float32, device=dev)
    for t, dt, sz, nm in ((pi, torch.int32, n, "pi"), (V, torch.float32, n, "V"), (w, torch.float32, n, "w"),
                          (lam, torch.float32, n, "lambda"), (grad_cost, torch.float32, n * m, "grad_cost"),
                          (grad_logits, torch.float32, n * m * k, "grad_logits")):
        _check(t, dt, sz, nm)
    L = lib()
    L.rmb_fixed_point_grad_workspace_bytes.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_opts)]
    L.rmb_fixed_point_grad_workspace_bytes.restype = ctypes.c_size_t
    o = opts.desc()
    nb = int(L.rmb_fixed_point_grad_workspace_bytes(ctypes.byref(mdp.desc), ctypes.byref(o)))
    if nb == 0:
        raise RmbError(RMB_ERR_ARG, "rmb_fixed_point_grad_workspace_bytes")
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    f = L.rmb_fixed_point_grad
    f.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(rmb_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_size_t, ctypes.POINTER(rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    s = rmb_stats() if stats else None
    st = f(ctypes.byref(mdp.desc), _ptr(pi), _ptr(V), _ptr(w), ctypes.byref(o), _ptr(lam), _ptr(grad_cost),
           _ptr(grad_logits), _ptr(ws), nb, ctypes.byref(s) if s is not None else None, _stream_handle(stream))
    d = _finish(st, s, "rmb_fixed_point_grad")
    return lam, grad_cost, grad_logits, d


def rmb_quantize_rows(P, rows: int, cols: int, p_dtype: int, codes=None, scale=None, stream=None):
    """Quantise float32 rows to bf16 / fp8-e4m3 codes with per-row scales (see rmb.h)."""
    import torch
    _check(P, torch.float32, rows * cols, "P")
    dt = torch.bfloat16 if p_dtype == RMB_P_BF16 else torch.uint8
    codes = torch.empty(rows * cols, dtype=dt, device=P.device) if codes is None else codes
    scale = torch.empty(rows, dtype=torch.float32, device=P.device) if scale is None else scale
    f = lib().rmb_quantize_rows
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(_ptr(P), int(rows), int(cols), int(p_dtype), _ptr(codes), _ptr(scale), _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_quantize_rows")
    return codes, scale


def dense_lowp(dm: DeviceMDP, p_dtype: int, stream=None) -> DeviceMDP:
    """The same dense MDP with its rows stored as bf16 / fp8-e4m3 codes (quantised on the device)."""
    rows = dm.n * dm.m
    codes, scale = rmb_quantize_rows(dm.P.reshape(-1), rows, dm.n, p_dtype, stream=stream)
    return DeviceMDP(dm.n, dm.m, dm.gamma, "dense", dm.cost, P=codes, p_dtype=p_dtype, row_scale=scale,
                     name=f"{dm.name}-{'bf16' if p_dtype == RMB_P_BF16 else 'fp8'}")


def rmb_vi_refined(lowp: DeviceMDP, ref: DeviceMDP, opts: Opts, eps_low: float, V, pi=None, qgap=None, ws=None,
                   stream=None):
    """Low-precision MB-VI to eps_low, then float32 refinement sweeps to opts.eps (see rmb.h).
    Returns (stats of the low-precision phase, stats of the refinement phase)."""
    import torch
    _check(V, torch.float32, ref.n, "V")
    ws = workspace(ref, opts) if ws is None else ws
    f = lib().rmb_vi_refined
    f.argtypes = [ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_mdp), ctypes.POINTER(rmb_opts), ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                  ctypes.POINTER(rmb_stats), ctypes.POINTER(rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    o = opts.desc()
    s1, s2 = rmb_stats(), rmb_stats()
    st = f(ctypes.byref(lowp.desc), ctypes.byref(ref.desc), ctypes.byref(o), float(eps_low), _ptr(V), _ptr(pi),
           _ptr(qgap), _ptr(ws), ws.numel(), ctypes.byref(s1), ctypes.byref(s2), _stream_handle(stream))
    if st not in (RMB_OK, RMB_ERR_NOT_CONVERGED):
        raise RmbError(st, "rmb_vi_refined")
    return s1.as_dict(), s2.as_dict()


def rmb_diag_gather_probe(src, idx, reps: int = 1, stream=None):
    """Diagnostic: gather src[idx] (reps times) with one 512-thread CTA per SM; returns the checksums."""
    import torch
    _check(src, torch.float32, 1, "src")
    _check(idx, torch.int32, 4, "idx")
    out = torch.empty(torch.cuda.get_device_properties(src.device).multi_processor_count * 512,
                      dtype=torch.float32, device=src.device)
    f = lib().rmb_diag_gather_probe
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(_ptr(src), src.numel(), _ptr(idx), idx.numel(), int(reps), _ptr(out), _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_diag_gather_probe")
    return out


def rmb_diag_gather_probe_tma(src, idx, reps: int = 1, stream=None):
    """Diagnostic: the same gathers through the tensor-memory-access unit (tile::gather4 of 16-byte
    rows); one 256-thread CTA per SM; returns the checksums (NaN where a wait ran out)."""
    import torch
    _check(src, torch.float32, 4, "src")
    _check(idx, torch.int32, 128, "idx")
    out = torch.empty(torch.cuda.get_device_properties(src.device).multi_processor_count * 256,
                      dtype=torch.float32, device=src.device)
    f = lib().rmb_diag_gather_probe_tma
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(_ptr(src), src.numel(), _ptr(idx), idx.numel(), int(reps), _ptr(out), _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_diag_gather_probe_tma")
    return out


def rmb_permutation(n: int, seed: int, sweep: int, out=None, stream=None):
    """sigma_{seed,sweep}(p) for p = 0..n-1 as an int32 CUDA tensor."""
    import torch
    out = torch.empty(int(n), dtype=torch.int32, device="cuda") if out is None else out
    _check(out, torch.int32, n, "out")
    st = lib().rmb_permutation(int(n), int(seed) & (2 ** 64 - 1), int(sweep) & (2 ** 64 - 1), _ptr(out),
                               _stream_handle(stream))
    if st != RMB_OK:
        raise RmbError(st, "rmb_permutation")
    return out


def rmb_validate(mdp: DeviceMDP, ws=None, stream=None) -> int:
    """Synchronous device validation; returns RMB_OK or RMB_ERR_INVALID_MDP."""
    import torch
    ws = torch.empty(256, dtype=torch.uint8, device="cuda") if ws is None else ws
    return int(lib().rmb_validate(ctypes.byref(mdp.desc), _ptr(ws), ws.numel(), _stream_handle(stream)))


# ----------------------------------------------------------------------------------------------
# Convenience: allocate outputs with torch and run a solve.
# ----------------------------------------------------------------------------------------------
def vi(mdp: DeviceMDP, opts: Opts, V0=None, want_policy: bool = True):
    import torch
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda") if V0 is None else V0.clone()
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda") if want_policy else None
    gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda") if want_policy else None
    st = rmb_vi(mdp, opts, V, pi, gap)
    return {"V": V, "pi": pi, "qgap": gap, "stats": st}


def mpi(mdp: DeviceMDP, opts: Opts, V0=None):
    import torch
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda") if V0 is None else V0.clone()
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb_mpi(mdp, opts, V, pi, gap)
    return {"V": V, "pi": pi, "qgap": gap, "stats": st}


def eval_policy(mdp: DeviceMDP, pi, opts: Opts, V0=None):
    import torch
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda") if V0 is None else V0.clone()
    st = rmb_eval_policy(mdp, pi, opts, V)
    return {"V": V, "stats": st}


# ----------------------------------------------------------------------------------------------
# Batched MB-VI (many independent MDPs in one persistent launch).
# ----------------------------------------------------------------------------------------------
class Batch:
    """A planned batched solve: holds the descriptors, the workspace and the handle."""

    def __init__(self, mdps, Vs, opts: Opts, pis=None, gaps=None, batches=None, stream=None):
        import torch
        L = lib()
        n = len(mdps)
        self.mdps, self.Vs, self.pis, self.gaps = mdps, Vs, pis, gaps
        arr = (rmb_batch_item * n)()
        for i, dm in enumerate(mdps):
            _check(Vs[i], torch.float32, dm.n, "V")
            arr[i].mdp = dm.desc
            arr[i].batch = 0 if batches is None else int(batches[i])
            arr[i].V = _ptr(Vs[i])
            arr[i].pi = _ptr(pis[i]) if pis is not None else None
            arr[i].qgap = _ptr(gaps[i]) if gaps is not None else None
        self.items = arr
        self.opts = opts
        o = opts.desc()
        L.rmb_batched_workspace_bytes.argtypes = [ctypes.POINTER(rmb_batch_item), ctypes.c_int, ctypes.POINTER(rmb_opts)]
        L.rmb_batched_workspace_bytes.restype = ctypes.c_size_t
        nb = int(L.rmb_batched_workspace_bytes(arr, n, ctypes.byref(o)))
        if nb == 0:
            raise RmbError(RMB_ERR_ARG, "rmb_batched_workspace_bytes")
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        self.handle = rmb_batch_handle()
        self.plan = (rmb_batch_plan_item * n)()
        f = L.rmb_batched_plan
        f.argtypes = [ctypes.POINTER(rmb_batch_item), ctypes.c_int, ctypes.POINTER(rmb_opts), ctypes.c_void_p,
                      ctypes.c_size_t, ctypes.POINTER(rmb_batch_handle), ctypes.POINTER(rmb_batch_plan_item),
                      ctypes.c_void_p]
        f.restype = ctypes.c_int
        st = f(arr, n, ctypes.byref(o), _ptr(self.ws), nb, ctypes.byref(self.handle), self.plan,
               _stream_handle(stream))
        if st != RMB_OK:
            raise RmbError(st, "rmb_batched_plan")
        self.graph = None

    def plan_table(self):
        return [{"batch": p.batch, "group_ctas": p.group_ctas, "first_cta": p.first_cta, "est_ms": p.est_ms}
                for p in self.plan]

    def run(self, stream=None):
        f = lib().rmb_batched_run
        f.argtypes = [ctypes.POINTER(rmb_batch_handle), ctypes.c_void_p]
        f.restype = ctypes.c_int
        st = f(ctypes.byref(self.handle), _stream_handle(stream))
        if st != RMB_OK:
            raise RmbError(st, "rmb_batched_run")

    def results(self, stream=None, check: bool = True):
        n = self.handle.count
        out = (rmb_stats * n)()
        f = lib().rmb_batched_results
        f.argtypes = [ctypes.POINTER(rmb_batch_handle), ctypes.POINTER(rmb_stats), ctypes.c_void_p]
        f.restype = ctypes.c_int
        st = f(ctypes.byref(self.handle), out, _stream_handle(stream))
        if check and st not in (RMB_OK, RMB_ERR_NOT_CONVERGED):
            raise RmbError(st, "rmb_batched_results")
        return [out[i].as_dict() for i in range(n)]

    def capture(self, stream):
        """Capture the solve into a CUDA graph on `stream` (a torch.cuda.Stream, not the default)."""
        L = lib()
        ex = ctypes.c_void_p()
        L.rmb_batched_graph_create.argtypes = [ctypes.POINTER(rmb_batch_handle), ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_void_p)]
        L.rmb_batched_graph_create.restype = ctypes.c_int
        st = L.rmb_batched_graph_create(ctypes.byref(self.handle), _stream_handle(stream), ctypes.byref(ex))
        if st != RMB_OK:
            raise RmbError(st, "rmb_batched_graph_create")
        self.graph = ex

    def replay(self, stream):
        L = lib()
        L.rmb_batched_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.rmb_batched_graph_launch.restype = ctypes.c_int
        st = L.rmb_batched_graph_launch(self.graph, _stream_handle(stream))
        if st != RMB_OK:
            raise RmbError(st, "rmb_batched_graph_launch")

    def __del__(self):
        try:
            if self.graph is not None:
                L = lib()
                L.rmb_batched_graph_destroy.argtypes = [ctypes.c_void_p]
                L.rmb_batched_graph_destroy(self.graph)
        except Exception:
            pass

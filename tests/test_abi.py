"""C-ABI checks that need no GPU: the library loads, exports every function include/rmb.h declares,
its structs have the header's layout, and argument errors come back before anything touches CUDA."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2110_02901_b300 as rmb
from paper_2110_02901_b300 import build as rbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmb.h")
DIAG_HEADER = os.path.join(ROOT, "include", "rmb_diag.h")


@pytest.fixture(scope="module")
def L():
    rbuild.build()
    return rmb.lib()


def declared_functions(header=HEADER):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("rmb_vi", "rmb_mpi", "rmb_eval_policy", "rmb_greedy", "rmb_permutation", "rmb_validate",
              "rmb_workspace_bytes", "rmb_status_string", "rmb_kernel_launches", "rmb_version"):
        assert f in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", rmb.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (rmb_\w+)", out))
    declared = declared_functions() + declared_functions(DIAG_HEADER)
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(L, f)


def test_diagnostics_stay_out_of_the_boundary():
    """The gather-rate probes are measurement tools, declared in rmb_diag.h only."""
    diag = declared_functions(DIAG_HEADER)
    assert diag == ["rmb_diag_gather_probe", "rmb_diag_gather_probe_tma"]
    assert not set(diag) & set(declared_functions())
    assert all(not f.startswith("rmb_diag_") for f in declared_functions())


def test_struct_layouts_match_header():
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "rmb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rmb_mdp), sizeof(rmb_opts), sizeof(rmb_stats),
         offsetof(rmb_mdp, gamma), offsetof(rmb_mdp, k_uniform), offsetof(rmb_opts, trace),
         offsetof(rmb_stats, ms), offsetof(rmb_opts, flags), offsetof(rmb_mdp, row_scale),
         sizeof(rmb_batch_item), sizeof(rmb_batch_handle), sizeof(rmb_batch_plan_item),
         offsetof(rmb_opts, select), offsetof(rmb_opts, weights));
  return 0;
}'''
    d = tempfile.mkdtemp()
    c = os.path.join(d, "t.c")
    open(c, "w").write(code)
    exe = os.path.join(d, "t")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    mine = [ctypes.sizeof(rmb.rmb_mdp), ctypes.sizeof(rmb.rmb_opts), ctypes.sizeof(rmb.rmb_stats),
            rmb.rmb_mdp.gamma.offset, rmb.rmb_mdp.k_uniform.offset, rmb.rmb_opts.trace.offset,
            rmb.rmb_stats.ms.offset, rmb.rmb_opts.flags.offset, rmb.rmb_mdp.row_scale.offset,
            ctypes.sizeof(rmb.rmb_batch_item), ctypes.sizeof(rmb.rmb_batch_handle),
            ctypes.sizeof(rmb.rmb_batch_plan_item), rmb.rmb_opts.select.offset, rmb.rmb_opts.weights.offset]
    assert vals == mine


def test_status_strings_and_version(L):
    assert rmb.rmb_status_string(0) == "ok"
    assert "wait timed out" in rmb.rmb_status_string(rmb.RMB_ERR_BARRIER_TIMEOUT)
    assert rmb.rmb_status_string(12345) == "unknown status"
    assert L.rmb_version() >> 16 == 1


def _fake_mdp(n=100, m=4, gamma=0.9, fmt=rmb.RMB_CSR):
    d = rmb.rmb_mdp()
    d.n, d.m, d.gamma, d.format = n, m, gamma, fmt
    # non-null stand-in addresses: every call below is rejected before any pointer is used
    d.cost = d.row_ptr = d.col = d.prob = d.P = 4096
    d.k_uniform = 0
    return d


def _opts(b=10, max_sweeps=10, eps=1e-6):
    return rmb.Opts(batch=b, max_sweeps=max_sweeps, eps=eps).desc()


@pytest.mark.parametrize("bad", ["null_mdp", "n0", "m0", "gamma1", "gamma0", "fmt", "b_neg", "sweeps0", "eps_neg",
                                 "eps_nan", "no_v", "ws_null", "ws_misaligned", "ws_small", "n_huge", "no_cost"])
def test_argument_errors_need_no_gpu(L, bad):
    d, o = _fake_mdp(), _opts()
    V, ws, wsb = 4096, 8192, 1 << 30
    mdp_ptr = ctypes.byref(d)
    if bad == "null_mdp":
        mdp_ptr = None
    elif bad == "n0":
        d.n = 0
    elif bad == "m0":
        d.m = 0
    elif bad == "gamma1":
        d.gamma = 1.0
    elif bad == "gamma0":
        d.gamma = 0.0
    elif bad == "fmt":
        d.format = 7
    elif bad == "b_neg":
        o.batch = -1
    elif bad == "sweeps0":
        o.max_sweeps = 0
    elif bad == "eps_neg":
        o.eps = -1.0
    elif bad == "eps_nan":
        o.eps = float("nan")
    elif bad == "no_v":
        V = None
    elif bad == "ws_null":
        ws = None
    elif bad == "ws_misaligned":
        ws = 8192 + 16
    elif bad == "ws_small":
        wsb = 16
    elif bad == "n_huge":
        d.n = 1 << 31
    elif bad == "no_cost":
        d.cost = None
    st = L.rmb_vi(mdp_ptr, ctypes.byref(o), V, None, None, ws, wsb, None, None)
    want = {"ws_null": rmb.RMB_ERR_WORKSPACE, "ws_misaligned": rmb.RMB_ERR_WORKSPACE,
            "ws_small": rmb.RMB_ERR_WORKSPACE, "n_huge": rmb.RMB_ERR_UNSUPPORTED}.get(bad, rmb.RMB_ERR_ARG)
    assert st == want


def test_mpi_and_eval_require_their_policy_arrays(L):
    d, o = _fake_mdp(), _opts()
    o.eval_sweeps = 5
    assert L.rmb_mpi(ctypes.byref(d), ctypes.byref(o), 4096, None, None, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    o.eval_sweeps = 0
    assert L.rmb_mpi(ctypes.byref(d), ctypes.byref(o), 4096, 4096, None, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    assert L.rmb_eval_policy(ctypes.byref(d), None, ctypes.byref(o), 4096, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    assert L.rmb_permutation(0, 1, 2, 4096, None) == rmb.RMB_ERR_ARG
    assert L.rmb_permutation(10, 1, 2, None, None) == rmb.RMB_ERR_ARG


def test_workspace_size_formula(L):
    d = _fake_mdp(n=1000)
    o = _opts(b=64)
    nb = L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o))
    # control block + two value buffers + two position caches + two value caches, 256-byte aligned,
    # + the precomputed permutation when T = ceil(n/b) >= 16, or 2 <= T and n < T * 65536
    assert nb == 256 + 2 * 4096 + 4 * 256 + 4096
    o.batch = 67            # 15 batches, n small: precomputed too
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == 256 + 2 * 4096 + 4 * 512 + 4096
    o.batch = 5000          # b > n means b = n: one batch, no permutation
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == 256 + 6 * 4096
    big = _fake_mdp(n=1 << 20)
    o.batch = 1 << 18       # 4 batches of a large MDP: evaluated on the fly
    assert L.rmb_workspace_bytes(ctypes.byref(big), ctypes.byref(o)) == 256 + 2 * (4 << 20) + 4 * (1 << 20)
    o.batch = 1 << 16       # 16 batches
    assert L.rmb_workspace_bytes(ctypes.byref(big), ctypes.byref(o)) == 256 + 2 * (4 << 20) + 4 * (1 << 18) + (4 << 20)
    o.batch = 70000         # 15 batches and n >= 15 * 65536: on the fly
    bb = (70000 * 4 + 255) // 256 * 256
    assert L.rmb_workspace_bytes(ctypes.byref(big), ctypes.byref(o)) == 256 + 2 * (4 << 20) + 4 * bb
    d.gamma = 2.0
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == 0


def test_batch_selection_arguments(L):
    d, o = _fake_mdp(), _opts()
    o.select = 3
    assert L.rmb_vi(ctypes.byref(d), ctypes.byref(o), 4096, None, None, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    o.select = rmb.RMB_SELECT_WEIGHTED       # weights missing
    assert L.rmb_vi(ctypes.byref(d), ctypes.byref(o), 4096, None, None, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    o.select = rmb.RMB_SELECT_UNIFORM        # policy evaluation has no full-residual stop rule for draws
    assert L.rmb_eval_policy(ctypes.byref(d), 4096, ctypes.byref(o), 4096, 8192, 1 << 30, None, None) == \
        rmb.RMB_ERR_UNSUPPORTED
    # draws add 16 bytes per state of batch marks when b < n; weights another 8 per state of
    # cumulative weights (+ 8 per 8192 states of tile sums)
    o.select = rmb.RMB_SELECT_PERMUTATION
    base = L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o))
    o.select = rmb.RMB_SELECT_WEIGHTED
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == base + 1792 + 1024 + 256
    o.select = rmb.RMB_SELECT_UNIFORM
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == base + 1792
    o.batch = 100           # b = n: one batch, no marks
    base = L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o))
    o.select = rmb.RMB_SELECT_PERMUTATION
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) == base


def test_residual_weights_arguments(L):
    d = _fake_mdp(n=1000)
    L.rmb_residual_weights_workspace_bytes.argtypes = [ctypes.POINTER(rmb.rmb_mdp)]
    L.rmb_residual_weights_workspace_bytes.restype = ctypes.c_size_t
    nb = L.rmb_residual_weights_workspace_bytes(ctypes.byref(d))
    # a Bellman pass (b = n: control + 6 arrays of n floats) + TV + the maximum
    assert nb == 256 + 6 * 4096 + 4096 + 256
    f = L.rmb_residual_weights
    f.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_size_t, ctypes.c_void_p]
    for frac in (-0.1, 1.5, float("nan")):
        assert f(ctypes.byref(d), 4096, frac, 8192, 1 << 20, nb, None) == rmb.RMB_ERR_ARG
    assert f(ctypes.byref(d), None, 0.1, 8192, 1 << 20, nb, None) == rmb.RMB_ERR_ARG
    assert f(ctypes.byref(d), 4096, 0.1, 8192, 1 << 20, nb - 1, None) == rmb.RMB_ERR_WORKSPACE


def test_residual_kind_arguments(L):
    d, o = _fake_mdp(), _opts()
    o.residual_kind = 2
    assert L.rmb_vi(ctypes.byref(d), ctypes.byref(o), 4096, None, None, 8192, 1 << 30, None, None) == rmb.RMB_ERR_ARG
    o.residual_kind = rmb.RMB_RESIDUAL_BELLMAN   # evaluation keeps the sweep-change test
    assert L.rmb_eval_policy(ctypes.byref(d), 4096, ctypes.byref(o), 4096, 8192, 1 << 30, None, None) == \
        rmb.RMB_ERR_UNSUPPORTED


def test_device_mdp_refuses_unreadable_tensors():
    """The descriptor holds raw pointers, so DeviceMDP refuses host tensors, strided views and
    wrong element types before any of them reaches the C ABI (checked without a GPU: a host tensor
    is refused first)."""
    import torch
    n, m = 4, 2
    cost = torch.zeros(n * m)
    P = torch.zeros(n * m * n)
    with pytest.raises(ValueError, match="cost"):
        rmb.DeviceMDP(n, m, 0.9, "dense", cost, P=P)
    with pytest.raises(ValueError, match="format"):
        rmb.DeviceMDP(n, m, 0.9, "coo", cost, P=P)
    with pytest.raises(ValueError, match="p_dtype"):
        rmb.DeviceMDP(n, m, 0.9, "dense", cost, P=P, p_dtype=7)
    with pytest.raises(ValueError, match="n >= 1"):
        rmb.DeviceMDP(0, m, 0.9, "dense", cost, P=P)


def test_gather_probe_tma_arguments(L):
    """Argument checks of the gather4 probe, taken before any device work."""
    f = L.rmb_diag_gather_probe_tma
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(4096, 1001, 8192, 1024, 1, 4096, None) == rmb.RMB_ERR_ARG      # n_src not a multiple of 4
    assert f(4096, 1000, 8192, 1000, 1, 4096, None) == rmb.RMB_ERR_ARG      # n_idx not a multiple of 128
    assert f(4096, 1000, 8200, 1024, 1, 4096, None) == rmb.RMB_ERR_ARG      # idx not 16-byte aligned
    assert f(4100, 1000, 8192, 1024, 1, 4096, None) == rmb.RMB_ERR_ARG      # src not 16-byte aligned
    assert f(4096, 1000, 8192, 1024, 0, 4096, None) == rmb.RMB_ERR_ARG      # reps < 1
    assert f(None, 1000, 8192, 1024, 1, 4096, None) == rmb.RMB_ERR_ARG


def test_noalloc_rejects_problems_beyond_the_fixed_scratch(L):
    """rmb_vi_noalloc checks the scratch its solve needs on the host, before any CUDA call."""
    n = 1 << 20                          # needs 8n + 16n bytes of scratch at b = n: 24 MiB > 8 MiB
    d = rmb.rmb_mdp()
    d.n, d.m, d.gamma, d.format = n, 8, 0.99, rmb.RMB_CSR
    d.cost = d.row_ptr = d.col = d.prob = 4096   # never dereferenced: rejected on the host
    o = rmb.Opts(batch=n).desc()
    f = L.rmb_vi_noalloc
    f.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.POINTER(rmb.rmb_opts), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(rmb.rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(d), ctypes.byref(o), 4096, None, None, None, None) == rmb.RMB_ERR_TOO_LARGE
    d.n = 400000                         # 12n bytes at b = 4096 (fits); draws add 16n of batch marks
    o = rmb.Opts(batch=4096).desc()
    assert L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(o)) <= 8 << 20
    o = rmb.Opts(batch=4096, select=rmb.RMB_SELECT_UNIFORM).desc()
    assert f(ctypes.byref(d), ctypes.byref(o), 4096, None, None, None, None) == rmb.RMB_ERR_TOO_LARGE
    assert "no-allocation" in rmb.rmb_status_string(rmb.RMB_ERR_TOO_LARGE)


def test_prioritized_arguments(L):
    """rmb_vi_prioritized rejects bad arguments on the host."""
    d = _fake_mdp()
    f = L.rmb_vi_prioritized
    f.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.POINTER(rmb.rmb_opts), ctypes.c_int32, ctypes.c_float,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                  ctypes.POINTER(rmb.rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    g = L.rmb_vi_prioritized_workspace_bytes
    g.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.POINTER(rmb.rmb_opts)]
    g.restype = ctypes.c_size_t
    o = rmb.Opts(batch=10).desc()
    need = g(ctypes.byref(d), ctypes.byref(o))
    wo = rmb.Opts(batch=10, select=rmb.RMB_SELECT_WEIGHTED).desc()
    assert need > L.rmb_workspace_bytes(ctypes.byref(d), ctypes.byref(wo)) + 4 * d.n
    call = lambda refresh, frac, ws_bytes, V=4096, ws=1 << 20: f(ctypes.byref(d), ctypes.byref(o), refresh, frac, V,
                                                                   None, None, ws, ws_bytes, None, None)
    assert call(0, 0.05, need) == rmb.RMB_ERR_ARG                  # refresh < 1
    assert call(4, 1.5, need) == rmb.RMB_ERR_ARG                   # floor_frac outside [0, 1]
    assert call(4, 0.05, need, V=None) == rmb.RMB_ERR_ARG          # no values
    assert call(4, 0.05, need - 1) == rmb.RMB_ERR_WORKSPACE        # workspace too small
    assert call(4, 0.05, need, ws=(1 << 20) + 8) == rmb.RMB_ERR_WORKSPACE   # not 256-byte aligned


def test_backup_states_arguments(L):
    """rmb_backup_states: argument checks on the host; count 0 launches nothing."""
    d = _fake_mdp()
    f = L.rmb_backup_states
    f.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(d), 4096, 8192, -1, None, 4096, None) == rmb.RMB_ERR_ARG      # negative count
    assert f(ctypes.byref(d), None, 8192, 5, None, 4096, None) == rmb.RMB_ERR_ARG      # no values
    assert f(ctypes.byref(d), 4096, None, 5, None, 4096, None) == rmb.RMB_ERR_ARG      # no states
    assert f(ctypes.byref(d), 4096, 8192, 5, None, None, None) == rmb.RMB_ERR_ARG      # no output
    assert f(ctypes.byref(d), None, None, 0, None, None, None) == rmb.RMB_OK           # nothing to do
    dd = _fake_mdp(fmt=rmb.RMB_DENSE)
    dd.p_dtype = rmb.RMB_P_BF16
    assert f(ctypes.byref(dd), 4096, 8192, 5, None, 4096, None) == rmb.RMB_ERR_UNSUPPORTED

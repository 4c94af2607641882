"""rmb_vi_noalloc: MB-VI for callers that cannot allocate device memory.

Some callers only receive device pointers for their inputs and outputs from a host application
that owns all device memory (a plugin in a simulator or a serving process, a C caller without an
allocator handle), or run control loops that forbid cudaMalloc after start-up.  This entry point
takes no workspace: its scratch is a fixed array inside the library.  These tests call it through
the C ABI and compare it with rmb_vi (which takes a caller-provided workspace), on consecutive calls
so that whatever the previous call left in the shared array is exercised.
"""
import ctypes

import numpy as np
import pytest

import mdpgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402

RTOL = 1e-5   # the value tolerance of the GPU parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


def _close(a, b):
    a = a.detach().cpu().numpy().astype(np.float64)
    b = b.detach().cpu().numpy().astype(np.float64)
    scale = max(1.0, float(np.abs(b).max()))
    assert float(np.abs(a - b).max()) <= RTOL * scale


def _solve_both(mdp, b, seed):
    dm = rmb.DeviceMDP.from_host(mdp)
    opts = rmb.Opts(batch=b, seed=seed, eps=1e-6, max_sweeps=20000)
    V_ref = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi_ref = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    gap_ref = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
    st_ref = rmb.rmb_vi(dm, opts, V_ref, pi_ref, gap_ref)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi_noalloc(dm, opts, V, pi, gap)
    assert st["status"] == rmb.RMB_OK == st_ref["status"]
    assert st["sweeps"] == st_ref["sweeps"]
    _close(V, V_ref)
    clear = gap_ref > 1e-6 * max(1.0, float(V_ref.abs().max()))
    assert torch.equal(pi[clear], pi_ref[clear])


def test_noalloc_matches_rmb_vi_on_consecutive_calls():
    # two different problems back to back: the second call starts from the first call's leftovers
    _solve_both(mdpgen.csr_uniform_k(20000, 8, 32, gamma=0.99, seed=1), 512, 12345)
    _solve_both(mdpgen.csr_uniform_k(7001, 4, 16, gamma=0.95, seed=2), 100, 7)
    _solve_both(mdpgen.dense_dirichlet(500, 4, gamma=0.95, seed=0), 50, 12345)


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    n = 1 << 20                          # needs 8n + 16n bytes of scratch at b = n: 24 MiB > 8 MiB
    d = rmb.rmb_mdp()
    d.n, d.m, d.gamma, d.format = n, 8, 0.99, rmb.RMB_CSR
    d.cost = d.row_ptr = d.col = d.prob = 4096   # never dereferenced: rejected on the host
    o = rmb.Opts(batch=n).desc()
    f = rmb.lib().rmb_vi_noalloc
    f.argtypes = [ctypes.POINTER(rmb.rmb_mdp), ctypes.POINTER(rmb.rmb_opts), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(rmb.rmb_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(d), ctypes.byref(o), 4096, None, None, None, None) == rmb.RMB_ERR_TOO_LARGE
    assert "no-allocation" in rmb.rmb_status_string(rmb.RMB_ERR_TOO_LARGE)

"""rmb_vi_noalloc: MB-VI for callers that cannot allocate device memory.

Some callers only receive device pointers for their inputs and outputs from a host application
that owns all device memory (a plugin in a simulator or a serving process, a C caller without an
allocator handle), or run control loops that forbid cudaMalloc after start-up.  This entry point
takes no workspace: its scratch is a fixed array inside the library.  These tests call it through
the C ABI and compare it with rmb_vi (which takes a caller-provided workspace), on consecutive calls
so that whatever the previous call left in the shared array is exercised.
"""

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


def _solve_both(mdp, b, seed, select=rmb.RMB_SELECT_PERMUTATION, weights=None):
    dm = rmb.DeviceMDP.from_host(mdp)
    w = None if weights is None else torch.as_tensor(weights, dtype=torch.int32, device="cuda")
    opts = rmb.Opts(batch=b, seed=seed, eps=1e-6, max_sweeps=20000, select=select, weights=w)
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
    assert st["batch"] == st_ref["batch"] == min(b, mdp.n)
    _close(V, V_ref)
    clear = gap_ref > 1e-6 * max(1.0, float(V_ref.abs().max()))
    assert torch.equal(pi[clear], pi_ref[clear])


def test_noalloc_matches_rmb_vi_on_consecutive_calls():
    # two different problems back to back: the second call starts from the first call's leftovers
    _solve_both(mdpgen.csr_uniform_k(20000, 8, 32, gamma=0.99, seed=1), 512, 12345)
    _solve_both(mdpgen.csr_uniform_k(7001, 4, 16, gamma=0.95, seed=2), 100, 7)
    _solve_both(mdpgen.dense_dirichlet(500, 4, gamma=0.95, seed=0), 50, 12345)


def test_noalloc_draws_clear_the_shared_scratch():
    """Draws with replacement keep per-state batch marks (and, with weights, cumulative weights) in
    the scratch array; a call must not see the stamps of the call before it.  Two uniform and two
    weighted solves back to back, each against rmb_vi with its own fresh workspace."""
    mdp = mdpgen.csr_uniform_k(6000, 4, 16, gamma=0.95, seed=3)
    _solve_both(mdp, 500, 11, select=rmb.RMB_SELECT_UNIFORM)
    _solve_both(mdp, 500, 11, select=rmb.RMB_SELECT_UNIFORM)
    wts = np.random.default_rng(5).integers(1, 1000, mdp.n)
    _solve_both(mdp, 700, 13, select=rmb.RMB_SELECT_WEIGHTED, weights=wts)
    _solve_both(mdp, 700, 13, select=rmb.RMB_SELECT_WEIGHTED, weights=wts)


def test_noalloc_allocates_no_device_memory():
    """Once its set-up has run, a call takes no device memory: the free memory the driver reports is
    the same before and after a solve (torch's caching allocator is not involved in the call)."""
    mdp = mdpgen.csr_uniform_k(5000, 8, 32, gamma=0.99, seed=4)
    dm = rmb.DeviceMDP.from_host(mdp)
    opts = rmb.Opts(batch=256, seed=1, eps=1e-6, max_sweeps=20000)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    rmb.rmb_vi_noalloc(dm, opts, V, pi)          # set-up: the scratch address is looked up once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        V.zero_()
        st = rmb.rmb_vi_noalloc(dm, opts, V, pi, stats=False)
        assert st is None
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0

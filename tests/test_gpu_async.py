"""Asynchronous sweeps (RMB_FLAG_ASYNC): no barrier between batches, values written in place at once.
Trajectories are not reproducible, so parity is against the fixed point: the exact optimum / policy
value (policy iteration, direct solves), within the FP32 value tolerance."""
import numpy as np
import pytest

import mdpgen
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


def close(a, b, tol=1e-5):
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(np.asarray(a, np.float64) - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"


@pytest.mark.parametrize("kind", ["vec", "ragged"])
def test_async_vi_reaches_the_optimum(kind):
    mdp = (mdpgen.csr_uniform_k(5000, 8, 32, gamma=0.99, seed=1) if kind == "vec"
           else mdpgen.csr_ragged(2000, 4, 12, gamma=0.95, seed=2, inadmissible_frac=0.2))
    jstar, pistar, _ = exact.policy_iteration(mdp)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=1, seed=3, eps=1e-7, max_sweeps=100000, flags=rmb.RMB_FLAG_ASYNC), V, pi)
    assert st["status"] == rmb.RMB_OK
    # one grid-wide barrier per sweep, one more per re-centring, none between batches
    assert st["barriers"] <= 2 * st["sweeps"] + 8
    close(V.cpu().numpy(), jstar)
    _, _, gap, _ = exact.bellman_pass(mdp, jstar)
    sel = gap > 1e-6 * max(1.0, np.abs(jstar).max())
    assert np.array_equal(pi.cpu().numpy()[sel], pistar[sel])


def test_async_evaluation_and_mpi():
    mdp = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.97, seed=4)
    pol = mdpgen.random_policy(mdp.n, mdp.m, seed=2)
    J = exact.policy_value(mdp, pol)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_eval_policy(dm, torch.from_numpy(pol).cuda(),
                             rmb.Opts(batch=1, eps=1e-8, max_sweeps=100000, flags=rmb.RMB_FLAG_ASYNC), V)
    assert st["status"] == rmb.RMB_OK
    close(V.cpu().numpy(), J)
    jstar, _, _ = exact.policy_iteration(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_mpi(dm, rmb.Opts(batch=1, eps=1e-7, max_sweeps=100000, eval_sweeps=10, flags=rmb.RMB_FLAG_ASYNC), V, pi)
    assert st["status"] == rmb.RMB_OK
    close(V.cpu().numpy(), jstar)


def test_async_needs_csr():
    mdp = mdpgen.dense_dirichlet(64, 2, seed=1)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(64, dtype=torch.float32, device="cuda")
    st, _ = rmb.rmb_vi(dm, rmb.Opts(batch=8, flags=rmb.RMB_FLAG_ASYNC), V, check=False)
    assert st == rmb.RMB_ERR_UNSUPPORTED


def test_async_without_allocation_and_batched_rejection():
    mdp = mdpgen.csr_uniform_k(4096, 4, 16, gamma=0.95, seed=8)
    jstar, _, _ = exact.policy_iteration(mdp)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi_noalloc(dm, rmb.Opts(batch=1, eps=1e-7, max_sweeps=100000, flags=rmb.RMB_FLAG_ASYNC), V)
    assert st["status"] == rmb.RMB_OK
    close(V.cpu().numpy(), jstar)
    with pytest.raises(rmb.RmbError):
        rmb.Batch([dm], [torch.zeros(mdp.n, dtype=torch.float32, device="cuda")],
                  rmb.Opts(batch=1, flags=rmb.RMB_FLAG_ASYNC))

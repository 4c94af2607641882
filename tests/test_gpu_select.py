"""Batch selection with replacement (the Sec. V extension) on the GPU against the FP64 oracle.

* the draws are integer work, checked exactly: at b = n from random start values exactly the drawn
  states change, and that set equals the oracle's draws for the sweep;
* trajectories (several sweeps, ragged batches, CSR vectorised / generic and dense rows, the
  precomputed and the on-the-fly order) equal the oracle's within the FP32 value tolerance;
* converged solves satisfy the full-residual stop rule and reach J*; MPI with drawn evaluation
  sweeps reaches J*; zero total weight, policy evaluation and the batched API are refused.
"""
import numpy as np
import pytest

import mdpgen
import oracle
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


def close(a, b, tol=RTOL):
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(np.asarray(a, np.float64) - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"


def weights_for(n, seed, zero_frac=0.0):
    g = np.random.default_rng(seed)
    w = g.integers(1, 1000, size=n).astype(np.uint32)
    if zero_frac:
        w[g.random(n) < zero_frac] = 0
        w[0] = 1
    return w


def dev_w(w):
    return torch.from_numpy(w.view(np.int32)).cuda()


@pytest.mark.parametrize("select", [1, 2])
@pytest.mark.parametrize("n", [1000, 70001])
def test_drawn_states_are_exactly_the_oracles(select, n):
    mdp = mdpgen.csr_uniform_k(n, 4, 8, gamma=0.9, seed=n)
    w = weights_for(n, 3, zero_frac=0.3)
    # values near -100: a drawn state moves by about 10, and the centred storage round-trips every
    # other value exactly (V - mu is exact in float32 when V and mu are within a factor 2)
    V0 = mdpgen.random_values(n, seed=5, scale=0.1, offset=-100.0)
    dm = rmb.DeviceMDP.from_host(mdp)
    for sweep in (0, 7):
        V = torch.from_numpy(V0).cuda()
        rmb.rmb_vi(dm, rmb.Opts(batch=n, seed=99, eps=0.0, max_sweeps=1, start_sweep=sweep, select=select,
                                weights=dev_w(w) if select == 2 else None), V)
        changed = np.flatnonzero(V.cpu().numpy() != V0)
        drawn = np.unique(oracle.sweep_order(n, 99, sweep, select, w))
        assert np.array_equal(changed, drawn)
        if select == 2:
            assert (w[changed] > 0).all()


CASES = [("csr-vec", lambda: mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.95, seed=1)),
         ("csr-generic", lambda: mdpgen.csr_ragged(1200, 3, 9, gamma=0.9, seed=2, inadmissible_frac=0.2)),
         ("dense", lambda: mdpgen.dense_dirichlet(400, 4, gamma=0.95, seed=3))]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("select", [1, 2])
def test_trajectories_match_oracle(name, make, select):
    mdp = make()
    w = weights_for(mdp.n, 8, zero_frac=0.1)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=2)
    for b in (1, 37, mdp.n // 3, mdp.n):
        if b == 1 and mdp.n > 1500:
            continue
        ref = oracle.mbvi(mdp, b, 11, eps=0.0, max_sweeps=4, V0=V0, select=select, weights=w)
        V = torch.from_numpy(V0).cuda()
        st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=11, eps=0.0, max_sweeps=4, select=select,
                                     weights=dev_w(w) if select == 2 else None), V)
        assert st["sweeps"] == 4 and st["path"].startswith(name.split("-")[0])
        close(V.cpu().numpy(), ref["V"])


@pytest.mark.parametrize("select", [1, 2])
def test_converged_solve_meets_the_full_residual_stop_rule(select):
    mdp = mdpgen.csr_uniform_k(4000, 8, 32, gamma=0.95, seed=4)
    jstar, pistar, _ = exact.policy_iteration(mdp)
    w = weights_for(mdp.n, 1)
    dm = rmb.DeviceMDP.from_host(mdp)
    for b in (64, 4000):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=3, eps=1e-6, max_sweeps=100000, select=select,
                                     weights=dev_w(w) if select == 2 else None), V, pi)
        assert st["status"] == rmb.RMB_OK and st["residual"] <= 1e-6
        v = V.cpu().numpy().astype(np.float64)
        resid = float(np.abs(exact.bellman_pass(mdp, v)[0] - v).max())
        assert resid <= 2e-6
        close(v, jstar)
        _, _, gap, _ = exact.bellman_pass(mdp, jstar)
        sel = gap > 1e-5
        assert np.array_equal(pi.cpu().numpy()[sel], pistar[sel])


def test_mpi_with_drawn_evaluation_sweeps():
    mdp = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.95, seed=6)
    jstar, _, _ = exact.policy_iteration(mdp)
    w = weights_for(mdp.n, 2)
    dm = rmb.DeviceMDP.from_host(mdp)
    for select in (1, 2):
        ref = oracle.mpi(mdp, 100, K=5, seed=4, eps=1e-6, select=select, weights=w)
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_mpi(dm, rmb.Opts(batch=100, seed=4, eps=1e-6, max_sweeps=10000, eval_sweeps=5, select=select,
                                      weights=dev_w(w) if select == 2 else None), V, pi)
        assert st["status"] == rmb.RMB_OK
        close(V.cpu().numpy(), jstar)
        assert abs(st["iters"] - ref["iters"]) <= 1


def test_async_noalloc_and_order_buffer_with_draws():
    mdp = mdpgen.csr_uniform_k(20000, 4, 8, gamma=0.9, seed=9)
    jstar, _, _ = exact.policy_iteration(mdp)
    w = weights_for(mdp.n, 4)
    dm = rmb.DeviceMDP.from_host(mdp)
    # 40 batches: the drawn order is precomputed into the order buffer; compare with the oracle
    ref = oracle.mbvi(mdp, 500, 21, eps=0.0, max_sweeps=3, select=2, weights=w)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    rmb.rmb_vi(dm, rmb.Opts(batch=500, seed=21, eps=0.0, max_sweeps=3, select=2, weights=dev_w(w)), V)
    close(V.cpu().numpy(), ref["V"])
    for flags in (rmb.RMB_FLAG_ASYNC, 0):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        o = rmb.Opts(batch=1, seed=5, eps=1e-6, max_sweeps=100000, select=1, flags=flags)
        st = (rmb.rmb_vi(dm, o, V) if flags else rmb.rmb_vi_noalloc(dm, o, V))
        assert st["status"] == rmb.RMB_OK
        close(V.cpu().numpy(), jstar)


def test_refusals():
    mdp = mdpgen.csr_uniform_k(500, 4, 8, gamma=0.9, seed=1)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    zero = dev_w(np.zeros(mdp.n, dtype=np.uint32))
    assert rmb.rmb_vi(dm, rmb.Opts(batch=10, select=2, weights=zero), V, check=False)[0] == rmb.RMB_ERR_ARG
    assert rmb.rmb_vi(dm, rmb.Opts(batch=10, select=2, weights=None), V, check=False)[0] == rmb.RMB_ERR_ARG
    assert rmb.rmb_vi(dm, rmb.Opts(batch=10, select=3), V, check=False)[0] == rmb.RMB_ERR_ARG
    pol = torch.zeros(mdp.n, dtype=torch.int32, device="cuda")
    assert rmb.rmb_eval_policy(dm, pol, rmb.Opts(batch=10, select=1), V, check=False)[0] == rmb.RMB_ERR_UNSUPPORTED
    with pytest.raises(rmb.RmbError):
        rmb.Batch([dm], [V], rmb.Opts(batch=1, select=1))
    # the solver still works afterwards
    st = rmb.rmb_vi(dm, rmb.Opts(batch=10, select=1, eps=1e-6), V)
    assert st["status"] == rmb.RMB_OK


def test_residual_weights_match_the_oracles_residual():
    mdp = mdpgen.csr_uniform_k(5000, 4, 16, gamma=0.95, seed=12)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=3)
    f = 0.05
    w = rmb.rmb_residual_weights(dm, torch.from_numpy(V0).cuda(), f).cpu().numpy().view(np.uint32).astype(np.int64)
    TV, _, _, _ = oracle.greedy(mdp, V0.astype(np.float64))
    r = np.abs(TV - V0)
    R = r.max()
    want = np.floor(2.0 ** 20 * (f + (1 - f) * r / R))
    # TV is rounded to float32 on the device: r moves by up to ~2 ulp of max(|TV|, |V|)
    tol = 2.0 + 2.0 ** 20 * (1 - f) * 4 * np.finfo(np.float32).eps * max(np.abs(TV).max(), np.abs(V0).max()) / R
    assert np.abs(w - want).max() <= tol
    assert w.min() >= int(np.floor(2.0 ** 20 * f)) - 1 and w.max() <= 2 ** 20
    assert r[np.argmax(w)] >= R * (1 - 1e-5)


def test_prioritized_vi_reaches_the_optimum():
    mdp = mdpgen.maze(40, 1500, gamma=0.95, slip=0.2, seed=9)
    jstar, _, _ = exact.policy_iteration(mdp)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    res = rmb.prioritized_vi(dm, V, batch=64, eps=1e-6, refresh=4, floor_frac=0.05)
    assert res["status"] == rmb.RMB_OK and res["residual"] <= 1e-6
    close(V.cpu().numpy(), jstar)


def test_prioritized_entry_point_equals_its_rounds():
    """rmb_vi_prioritized is the loop of rounds {residual weights; <= refresh weighted sweeps}: the same
    rounds run one by one through rmb_residual_weights and rmb_vi give the same values bit for bit."""
    mdp = mdpgen.maze(30, 800, gamma=0.95, slip=0.2, seed=4)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    # eps above the float32 floor of this maze (|V| ~ 20: ||TV - V||_inf settles at a few 1e-6 under draws)
    st = rmb.rmb_vi_prioritized(dm, rmb.Opts(batch=50, seed=21, eps=1e-5, max_sweeps=100000, validate=False), V,
                                refresh=3, floor_frac=0.1)
    assert st["status"] == rmb.RMB_OK and st["iters"] >= 2
    U = torch.zeros_like(V)
    sweeps, rounds = 0, 0
    while True:
        w = rmb.rmb_residual_weights(dm, U, 0.1)
        r = rmb.rmb_vi(dm, rmb.Opts(batch=50, seed=21, eps=1e-5, max_sweeps=3, start_sweep=sweeps, validate=False,
                                    select=rmb.RMB_SELECT_WEIGHTED, weights=w), U)
        sweeps += r["sweeps"]
        rounds += 1
        if r["status"] == rmb.RMB_OK:
            break
    assert (sweeps, rounds) == (st["sweeps"], st["iters"])
    assert torch.equal(U, V)


@pytest.mark.parametrize("n", [1, 2, 3, 37])
def test_tiny_problems_with_draws_and_stop_tests(n):
    mdp = mdpgen.csr_ragged(n, 3, 3, gamma=0.9, seed=n)
    dm = rmb.DeviceMDP.from_host(mdp)
    w = (np.arange(n, dtype=np.uint32) % 4) + 1
    V0 = mdpgen.random_values(n, seed=1)
    for b in sorted({1, 2, n}):
        b = min(b, n)
        for select in (1, 2):
            ref = oracle.mbvi(mdp, b, 3, eps=0.0, max_sweeps=5, V0=V0, select=select, weights=w)
            V = torch.from_numpy(V0).cuda()
            rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=3, eps=0.0, max_sweeps=5, select=select,
                                    weights=dev_w(w) if select == 2 else None), V)
            close(V.cpu().numpy(), ref["V"])
        for rk in (0, 1):
            # both stop tests end the solve; values are compared at the oracle's stopping sweep (the
            # float32 and FP64 residuals may cross eps a sweep apart)
            ref = oracle.mbvi(mdp, b, 3, eps=1e-6, max_sweeps=10000, V0=V0, residual_kind=rk)
            V = torch.from_numpy(V0).cuda()
            st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=3, eps=1e-6, max_sweeps=10000, residual_kind=rk), V)
            assert st["status"] == rmb.RMB_OK and abs(st["sweeps"] - ref["sweeps"]) <= 2
            V = torch.from_numpy(V0).cuda()
            rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=3, eps=0.0, max_sweeps=ref["sweeps"]), V)
            close(V.cpu().numpy(), ref["V"])
    jstar, _, _ = exact.policy_iteration(mdp)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=1, eps=1e-7, max_sweeps=100000, flags=rmb.RMB_FLAG_ASYNC), V)
    assert st["status"] == rmb.RMB_OK
    close(V.cpu().numpy(), jstar)

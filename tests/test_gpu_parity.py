"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerance (FP32 values): max |V_gpu - V_oracle| <= 1e-5 * max(1, ||V_oracle||_inf); greedy policies
equal wherever the oracle's Q-gap exceeds 1e-6 (relative to the same scale); permutations bit-exact.
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


def close(v_gpu, v_ref, rtol=RTOL):
    v_gpu = np.asarray(v_gpu, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(v_ref))))
    err = float(np.max(np.abs(v_gpu - v_ref))) if len(v_ref) else 0.0
    assert err <= rtol * scale, f"max abs err {err:.3e} > {rtol:.0e} * {scale:.3e}"
    return err


def to_np(t):
    return t.detach().cpu().numpy()


def gpu_vi(dm, b, seed, eps, max_sweeps, V0=None, start_sweep=0, validate=True, want_policy=True, flags=0):
    V = torch.zeros(dm.n, dtype=torch.float32, device="cuda") if V0 is None else \
        torch.from_numpy(np.asarray(V0, np.float32)).cuda()
    pi = torch.empty(dm.n, dtype=torch.int32, device="cuda") if want_policy else None
    gap = torch.empty(dm.n, dtype=torch.float32, device="cuda") if want_policy else None
    st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=seed, eps=eps, max_sweeps=max_sweeps, start_sweep=start_sweep,
                                 validate=validate, flags=flags), V, pi, gap)
    return to_np(V), (to_np(pi) if pi is not None else None), (to_np(gap) if gap is not None else None), st


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 500, 1000, 4097, 65536, 1 << 20, 3000017])
def test_permutation_bit_exact(n):
    for seed, sweep in ((12345, 0), (7, 1), (2 ** 63 + 11, 2 ** 33 + 5)):
        got = to_np(rmb.rmb_permutation(n, seed, sweep)).astype(np.int64)
        want = oracle.perm(n, seed, sweep)
        assert np.array_equal(got, want)


# ------------------------------------------------------------------------------------------------
CSR_CASES = [
    # (n, m, k, gamma, seed)  -- vectorised row path shapes
    (5000, 8, 32, 0.99, 1),     # cfg2-shaped, ragged batch tails for most b
    (3001, 3, 16, 0.95, 2),     # m not a power of two
    (2000, 16, 16, 0.9, 3),     # two row passes per state
    (1500, 2, 4, 0.9, 4),       # one float4 per row
    (1200, 1, 8, 0.9, 5),       # single action
    (700, 5, 256, 0.95, 6),     # k/4 = 64 > 32: two chunks per lane
]


@pytest.mark.parametrize("case", CSR_CASES)
def test_csr_vi_trajectory_parity(case):
    n, m, k, g, seed = case
    mdp = mdpgen.csr_uniform_k(n, m, k, gamma=g, seed=seed)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(n, seed=seed, scale=0.5)
    for b in sorted({1, 7, 64, 333, n - 1, n}):
        if b < 1:
            continue
        ref = oracle.mbvi(mdp, b, seed=99, eps=0.0, max_sweeps=6, V0=V0, traj=True)
        for s in (1, 2, 6):
            V, _, _, st = gpu_vi(dm, b, 99, 0.0, s, V0=V0, want_policy=False)
            assert st["sweeps"] == s
            close(V, ref["traj"][s - 1])


@pytest.mark.parametrize("case", CSR_CASES[:3])
def test_csr_vi_converged_parity_and_policy(case):
    n, m, k, g, seed = case
    mdp = mdpgen.csr_uniform_k(n, m, k, gamma=g, seed=seed)
    dm = rmb.DeviceMDP.from_host(mdp)
    for b in (16, 512, n):
        ref = oracle.mbvi(mdp, b, seed=5, eps=1e-6, max_sweeps=20000)
        V, pi, gap, st = gpu_vi(dm, b, 5, 1e-6, 20000)
        assert st["status"] == rmb.RMB_OK and st["residual"] <= 1e-6
        # near eps the residual shrinks by only ~(1 - gamma) per sweep, so float32 rounding noise in
        # the residual (a few 1e-8 here) moves the stopping sweep by a few sweeps
        assert abs(st["sweeps"] - ref["sweeps"]) <= max(2, 0.02 * ref["sweeps"])
        scale = max(1.0, float(np.abs(ref["V"]).max()))
        close(V, ref["V"])
        # greedy policy at the oracle's own final values, compared where the oracle's gap is clear
        _, opi, ogap, _ = oracle.greedy(mdp, ref["V"])
        sel = ogap > 1e-6 * scale
        assert np.array_equal(pi[sel], opi[sel])
        # and at the GPU's values, both sides deciding from the same V
        _, opi2, ogap2, _ = oracle.greedy(mdp, V.astype(np.float64))
        sel2 = ogap2 > 1e-6 * scale
        assert np.array_equal(pi[sel2], opi2[sel2])
        close(gap[sel2], ogap2[sel2], rtol=1e-5)


def test_csr_vi_matches_certified_optimum():
    mdp = mdpgen.csr_uniform_k(4000, 8, 32, gamma=0.99, seed=11)
    jstar, pistar, cert = exact.policy_iteration(mdp)
    assert cert < 1e-10
    dm = rmb.DeviceMDP.from_host(mdp)
    V, pi, gap, st = gpu_vi(dm, 256, 12345, 1e-7, 50000)
    scale = float(np.abs(jstar).max())
    close(V, jstar)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    sel = jgap > 1e-6 * scale
    assert np.array_equal(pi[sel], pistar[sel])


def test_csr_generic_rows_ragged_and_inadmissible():
    mdp = mdpgen.csr_ragged(1500, 4, 12, gamma=0.9, seed=3, inadmissible_frac=0.3)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=1)
    for b in (1, 50, 1500):
        ref = oracle.mbvi(mdp, b, seed=3, eps=0.0, max_sweeps=4, V0=V0, traj=True)
        for flags, path in ((rmb.RMB_FLAG_NO_CLUSTER, "csr-generic"), (0, "cluster" if b <= 512 else "csr-generic")):
            V, _, _, st = gpu_vi(dm, b, 3, 0.0, 4, V0=V0, want_policy=False, flags=flags)
            assert st["path"] == path
            close(V, ref["traj"][3])
    ref = oracle.mbvi(mdp, 50, seed=3, eps=1e-6, max_sweeps=5000)
    for flags in (rmb.RMB_FLAG_NO_CLUSTER, 0):
        V, pi, gap, st = gpu_vi(dm, 50, 3, 1e-6, 5000, flags=flags)
        close(V, ref["V"])
        assert np.all(np.isfinite(mdp.cost[np.arange(mdp.n) * mdp.m + pi]))


@pytest.mark.parametrize("k", [12, 30])
def test_csr_generic_path_for_uniform_rows_not_vectorisable(k):
    mdp = mdpgen.csr_uniform_k(900, 3, k, gamma=0.9, seed=k)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 40, seed=1, eps=0.0, max_sweeps=3, traj=True)
    # uniform rows that are not vectorisable take the cluster path only when a state fits one lane per entry
    for flags, path in ((rmb.RMB_FLAG_NO_CLUSTER, "csr-generic"), (0, "cluster" if 3 * k <= 32 else "csr-generic")):
        V, _, _, st = gpu_vi(dm, 40, 1, 0.0, 3, want_policy=False, flags=flags)
        assert st["path"] == path
        close(V, ref["traj"][2])


# ------------------------------------------------------------------------------------------------
def test_dense_config1_full_size():
    mdp = mdpgen.config1()
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 50, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=5, traj=True)
    # both solvers: the one-cluster solve this workload takes by default, and the grid-wide one
    for flags, path in ((0, "cluster"), (rmb.RMB_FLAG_NO_CLUSTER, "dense")):
        for s in (1, 5):
            V, _, _, st = gpu_vi(dm, 50, mdpgen.PERM_SEED, 0.0, s, want_policy=False, flags=flags)
            assert st["path"] == path
            close(V, ref["traj"][s - 1])
    ref = oracle.mbvi(mdp, 50, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=100000)
    jstar, pistar, _ = exact.policy_iteration(mdp)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    sel = jgap > 1e-6 * max(1.0, float(np.abs(jstar).max()))
    for flags in (0, rmb.RMB_FLAG_NO_CLUSTER):
        V, pi, gap, st = gpu_vi(dm, 50, mdpgen.PERM_SEED, 1e-6, 100000, flags=flags)
        assert st["status"] == rmb.RMB_OK and abs(st["sweeps"] - ref["sweeps"]) <= 2
        if st["sweeps"] != ref["sweeps"]:   # compare at the oracle's stopping sweep
            V, pi, gap, st = gpu_vi(dm, 50, mdpgen.PERM_SEED, 0.0, ref["sweeps"], flags=flags)
        close(V, ref["V"])
        close(V, jstar)
        assert np.array_equal(pi[sel], pistar[sel])


@pytest.mark.parametrize("n,m,stage", [(333, 3, None), (1000, 12, None), (1000, 4, "128"), (999, 2, "100")])
def test_dense_paths(n, m, stage, monkeypatch):
    """n % 4 != 0 takes the scalar row path; RMB_DENSE_STAGE < n stages values chunk by chunk."""
    if stage:
        monkeypatch.setenv("RMB_DENSE_STAGE", stage)
    mdp = mdpgen.dense_dirichlet(n, m, alpha=0.5, gamma=0.95, seed=n + m, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(n, seed=2)
    for b in (1, 37, n):
        ref = oracle.mbvi(mdp, b, seed=8, eps=0.0, max_sweeps=3, V0=V0, traj=True)
        for flags in (rmb.RMB_FLAG_NO_CLUSTER, 0):
            V, _, _, st = gpu_vi(dm, b, 8, 0.0, 3, V0=V0, want_policy=False, flags=flags)
            assert st["path"] != "cluster" if flags else st["path"] == ("cluster" if b < n else "dense")
            close(V, ref["traj"][2])


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("flags", [0, rmb.RMB_FLAG_NO_CLUSTER], ids=["auto", "grid"])
@pytest.mark.parametrize("fmt", ["csr", "dense"])
def test_policy_evaluation_parity_and_closed_form(fmt, flags):
    mdp = (mdpgen.csr_uniform_k(3000, 8, 32, gamma=0.97, seed=21) if fmt == "csr"
           else mdpgen.dense_dirichlet(600, 4, gamma=0.95, seed=22))
    dm = rmb.DeviceMDP.from_host(mdp)
    pi = mdpgen.random_policy(mdp.n, mdp.m, seed=3)
    pit = torch.from_numpy(pi).cuda()
    for b in (1, 100, mdp.n):
        ref = oracle.eval_policy(mdp, pi, b, seed=4, eps=0.0, max_sweeps=5, traj=True)
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_eval_policy(dm, pit, rmb.Opts(batch=b, seed=4, eps=0.0, max_sweeps=5, flags=flags), V)
        assert st["sweeps"] == 5
        assert (st["path"] == "cluster") == (flags == 0 and b < mdp.n), (b, st["path"])
        close(to_np(V), ref["traj"][4])
    J = exact.policy_value(mdp, pi)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_eval_policy(dm, pit, rmb.Opts(batch=128, seed=4, eps=1e-7, max_sweeps=100000, flags=flags), V)
    assert st["status"] == rmb.RMB_OK
    close(to_np(V), J)


@pytest.mark.parametrize("flags", [0, rmb.RMB_FLAG_NO_CLUSTER], ids=["auto", "grid"])
@pytest.mark.parametrize("fmt", ["csr", "dense"])
def test_mpi_parity(fmt, flags):
    mdp = (mdpgen.csr_uniform_k(4000, 8, 32, gamma=0.99, seed=31) if fmt == "csr"
           else mdpgen.dense_dirichlet(500, 4, gamma=0.95, seed=32))
    dm = rmb.DeviceMDP.from_host(mdp)
    for b, K in ((64, 10), (mdp.n, 3), (1, 2)):
        for iters in (1, 2, 4):
            ref = oracle.mpi(mdp, b, K, seed=6, eps=0.0, max_iters=iters)
            V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
            pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
            st = rmb.rmb_mpi(dm, rmb.Opts(batch=b, seed=6, eps=0.0, max_sweeps=iters, eval_sweeps=K, flags=flags), V, pi)
            assert st["iters"] == iters and st["sweeps"] == K * (iters - 1)
            close(to_np(V), ref["V"])
            close([st["residual"]], np.array([ref["resid"][-1]]), rtol=1e-5)
    jstar, pistar, _ = exact.policy_iteration(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_mpi(dm, rmb.Opts(batch=64, seed=6, eps=1e-6, max_sweeps=100000, eval_sweeps=10, flags=flags), V, pi)
    assert st["status"] == rmb.RMB_OK
    close(to_np(V), jstar)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    sel = jgap > 1e-6 * max(1.0, float(np.abs(jstar).max()))
    assert np.array_equal(to_np(pi)[sel], pistar[sel])


@pytest.mark.parametrize("fmt", ["csr", "dense"])
def test_greedy_pass_parity(fmt):
    mdp = (mdpgen.csr_uniform_k(5000, 8, 32, gamma=0.99, seed=41) if fmt == "csr"
           else mdpgen.dense_dirichlet(800, 6, gamma=0.9, seed=42, cost_dist="normal"))
    dm = rmb.DeviceMDP.from_host(mdp)
    Vh = mdpgen.random_values(mdp.n, seed=9, scale=0.3, offset=11.0)
    TVr, pir, gapr, resr = oracle.greedy(mdp, Vh.astype(np.float64))
    V = torch.from_numpy(Vh).cuda()
    TV = torch.empty_like(V)
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    gap = torch.empty_like(V)
    st = rmb.rmb_greedy(dm, V, TV, pi, gap)
    close(to_np(TV), TVr)
    sel = gapr > 1e-6 * 11
    assert np.array_equal(to_np(pi)[sel], pir[sel])
    close([st["residual"]], np.array([resr]))


# ------------------------------------------------------------------------------------------------
def test_edge_cases_tiny_and_clamped_batch():
    # n = 1: one state with a self loop
    mdp = mdpgen.csr_uniform_k(1, 2, 1, gamma=0.5, seed=0)
    dm = rmb.DeviceMDP.from_host(mdp)
    V, pi, gap, st = gpu_vi(dm, 5, 1, 1e-7, 1000)      # b > n is clamped to n
    c = mdp.cost.astype(np.float64)
    assert abs(V[0] - c.min() / 0.5) < 1e-5 and pi[0] == int(np.argmin(c))
    # tiny dense
    mdp = mdpgen.dense_dirichlet(3, 2, gamma=0.9, seed=1)
    dm = rmb.DeviceMDP.from_host(mdp)
    jstar = exact.brute_force(mdp)
    for b in (1, 2, 3):
        V, _, _, _ = gpu_vi(dm, b, 2, 1e-8, 100000)
        close(V, jstar)


def test_resume_from_start_sweep_and_determinism():
    mdp = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.95, seed=51)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 100, seed=77, eps=0.0, max_sweeps=8, traj=True)
    V3, _, _, _ = gpu_vi(dm, 100, 77, 0.0, 3, want_policy=False)
    V8, _, _, st = gpu_vi(dm, 100, 77, 0.0, 5, V0=V3, start_sweep=3, want_policy=False)
    close(V8, ref["traj"][7])
    a = gpu_vi(dm, 100, 77, 1e-6, 10000)
    b = gpu_vi(dm, 100, 77, 1e-6, 10000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[3]["sweeps"] == b[3]["sweeps"]


def test_trace_records_sweep_residuals():
    mdp = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.9, seed=61)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 77, seed=5, eps=1e-6, max_sweeps=1000)
    trace = torch.zeros(1000, dtype=torch.float64, device="cuda")
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=77, seed=5, eps=1e-6, max_sweeps=1000, trace=trace), V)
    t = to_np(trace)[: st["sweeps"]]
    k = min(len(t), len(ref["deltas"]))
    assert np.allclose(t[:k], ref["deltas"][:k], rtol=1e-3, atol=2e-6)
    assert t[-1] <= 1e-6 and st["residual"] == t[-1]


def test_not_converged_status():
    mdp = mdpgen.csr_uniform_k(500, 4, 8, gamma=0.99, seed=71)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=10, eps=1e-9, max_sweeps=3), V)
    assert st["status"] == rmb.RMB_ERR_NOT_CONVERGED and st["sweeps"] == 3


# ------------------------------------------------------------------------------------------------
def test_validation_rejects_bad_mdps():
    good = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81)
    assert rmb.rmb_validate(rmb.DeviceMDP.from_host(good)) == rmb.RMB_OK
    bads = []
    m1 = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81); m1.prob[5] = 1.5; bads.append(m1)
    m2 = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81); m2.col[7] = 300; bads.append(m2)
    m3 = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81); m3.prob[8:16] *= 0.9; bads.append(m3)
    m4 = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81); m4.cost[4] = np.nan; bads.append(m4)
    m5 = mdpgen.csr_uniform_k(300, 3, 8, gamma=0.9, seed=81); m5.cost[6:9] = np.inf; bads.append(m5)
    d6 = mdpgen.dense_dirichlet(50, 2, seed=1); d6.P[3, 1, 4] = -0.1; bads.append(d6)
    for bad in bads:
        dm = rmb.DeviceMDP.from_host(bad)
        assert rmb.rmb_validate(dm) == rmb.RMB_ERR_INVALID_MDP
        V = torch.zeros(bad.n, dtype=torch.float32, device="cuda")
        st, stats = rmb.rmb_vi(dm, rmb.Opts(batch=16, max_sweeps=10), V, check=False)
        assert st == rmb.RMB_ERR_INVALID_MDP == stats["status"]


def test_barrier_timeout_is_reported_and_context_survives():
    mdp = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.9, seed=91)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    o = rmb.Opts(batch=64, max_sweeps=5, barrier_timeout_ns=50_000_000, flags=rmb.RMB_FLAG_INJECT_BARRIER_STALL)
    st, stats = rmb.rmb_vi(dm, o, V, check=False)
    assert st == rmb.RMB_ERR_BARRIER_TIMEOUT == stats["status"]
    # the context still works
    ref = oracle.mbvi(mdp, 64, seed=12345, eps=0.0, max_sweeps=2, traj=True)
    V2, _, _, st2 = gpu_vi(dm, 64, 12345, 0.0, 2, want_policy=False)
    close(V2, ref["traj"][1])


def test_grid_size_does_not_change_results():
    mdp = mdpgen.csr_uniform_k(3000, 8, 32, gamma=0.99, seed=95)
    dm = rmb.DeviceMDP.from_host(mdp)
    outs = []
    for ctas in (1, 3, 0):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=200, seed=3, eps=0.0, max_sweeps=4, grid_ctas=ctas), V)
        outs.append(to_np(V))
    ref = oracle.mbvi(mdp, 200, seed=3, eps=0.0, max_sweeps=4)
    for o in outs:
        close(o, ref["V"])


def test_bellman_residual_stop_test_matches_oracle():
    """residual_kind = RMB_RESIDUAL_BELLMAN: the solve ends on a confirmed ||TV - V||_inf <= eps; the
    values equal the oracle's under the same rule, and the full residual really is below eps."""
    from oracle import exact
    for mdp in (mdpgen.csr_uniform_k(3000, 8, 32, gamma=0.95, seed=3),
                mdpgen.csr_ragged(1500, 4, 9, gamma=0.9, seed=4), mdpgen.dense_dirichlet(300, 4, gamma=0.95, seed=5)):
        dm = rmb.DeviceMDP.from_host(mdp)
        for b in (37, mdp.n):
            ref = oracle.mbvi(mdp, b, 9, eps=1e-5, max_sweeps=100000, residual_kind=1)
            V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
            st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=9, eps=1e-5, max_sweeps=100000,
                                         residual_kind=rmb.RMB_RESIDUAL_BELLMAN), V)
            assert st["status"] == rmb.RMB_OK and st["residual"] <= 1e-5
            v = V.cpu().numpy().astype(np.float64)
            assert float(np.abs(exact.bellman_pass(mdp, v)[0] - v).max()) <= 1.2e-5
            assert abs(st["sweeps"] - ref["sweeps"]) <= 2
            assert np.abs(v - ref["V"]).max() <= 1e-4 * max(1.0, np.abs(ref["V"]).max())


def test_nonfinite_inputs_are_reported():
    """A NaN start value ends the solve with RMB_ERR_NONFINITE and a NaN cost is rejected by the
    validation pass (statuses, not faults); the library keeps working afterwards."""
    mdp = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.9, seed=2)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=1)
    V0[17] = np.nan
    V = torch.from_numpy(V0).cuda()
    st, _ = rmb.rmb_vi(dm, rmb.Opts(batch=100, eps=1e-6, max_sweeps=50), V, check=False)
    assert st == rmb.RMB_ERR_NONFINITE
    bad = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.9, seed=2)
    bad.cost = bad.cost.copy()
    bad.cost[4 * 33] = np.nan
    dbad = rmb.DeviceMDP.from_host(bad)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st, _ = rmb.rmb_vi(dbad, rmb.Opts(batch=100, eps=1e-6, max_sweeps=50, validate=True), V, check=False)
    assert st == rmb.RMB_ERR_INVALID_MDP
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    assert rmb.rmb_vi(dm, rmb.Opts(batch=100, eps=1e-6), V)["status"] == rmb.RMB_OK


@pytest.mark.parametrize("make", [lambda: mdpgen.csr_uniform_k(20000, 8, 32, gamma=0.95, seed=8),
                                  lambda: mdpgen.csr_ragged(3000, 4, 9, gamma=0.9, seed=9),
                                  lambda: mdpgen.dense_dirichlet(700, 4, gamma=0.95, seed=10)])
def test_batch_zero_uses_the_time_model_choice(make):
    """opts.batch = 0: the library picks b (reported in stats['batch']); the solve equals the oracle
    at that b, and the workspace sized for batch = 0 is the one the solve needs."""
    mdp = make()
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=0, seed=4, eps=0.0, max_sweeps=6), V)
    b = st["batch"]
    assert 1 <= b <= mdp.n and st["sweeps"] == 6
    ref = oracle.mbvi(mdp, b, 4, eps=0.0, max_sweeps=6)
    close(V.cpu().numpy(), ref["V"])
    V2 = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st2 = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=4, eps=0.0, max_sweeps=6), V2)
    assert st2["batch"] == b and torch.equal(V, V2)


def test_csr_headline_config_full_size():
    """The bench's workload at full size (n = 2^20, m = 8, k = 32, gamma = 0.99) in its launch
    configuration (b = 262144): the whole value vector after 3 sweeps, and the converged solve (sweep
    residual 1e-6), against the FP64 oracle's MB-VI element by element (the GPU trajectory is taken at
    the oracle's stopping sweep), and the greedy policy against the oracle's wherever its Q-gap is
    clear."""
    mdp = mdpgen.config2()
    dm = rmb.DeviceMDP.from_host(mdp)
    b = 262144
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=3, validate=False), V)
    ref = oracle.mbvi(mdp, b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=3)
    close(V.cpu().numpy(), ref["V"])
    ref = oracle.mbvi(mdp, b, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=5000)
    k = ref["sweeps"]
    V.zero_()
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000, validate=False), V, pi)
    assert st["status"] == rmb.RMB_OK
    # the float32 and FP64 sweep changes cross 1e-6 within a sweep or two of each other
    assert abs(st["sweeps"] - k) <= 2, (st["sweeps"], k)
    if st["sweeps"] != k:
        V.zero_()
        rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=k, validate=False), V, pi)
    close(V.cpu().numpy(), ref["V"])
    _, opi, ogap, _ = oracle.greedy(mdp, ref["V"])
    sel = ogap > 1e-6 * max(1.0, float(np.abs(ref["V"]).max()))
    assert sel.mean() > 0.99
    assert np.array_equal(pi.cpu().numpy()[sel], opi[sel])

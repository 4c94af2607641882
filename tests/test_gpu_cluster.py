"""The one-cluster solve of small MDPs (stats path "cluster"): values and orders in shared memory, batch
values stored into every CTA's copy, hardware cluster barriers between batches.  Trajectories equal the
FP64 oracle's MB-VI (eq. (11), sigma_{seed,k} of Sec. III-A) within 1e-5 of ||V||_inf, for every row
form it reads; converged values and greedy policies equal the oracle's; statuses and edge cases."""
import numpy as np
import pytest

import mdpgen
import oracle
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
    a = np.asarray(a, np.float64)
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"


CASES = [
    ("dense n%4", lambda: mdpgen.dense_dirichlet(333, 3, alpha=0.5, gamma=0.95, seed=1, cost_dist="normal")),
    ("dense m=11", lambda: mdpgen.dense_dirichlet(640, 11, alpha=0.2, gamma=0.99, seed=2)),
    ("csr k=32", lambda: mdpgen.csr_uniform_k(5000, 8, 32, gamma=0.99, seed=3)),
    ("csr ragged", lambda: mdpgen.csr_ragged(4000, 5, 9, gamma=0.95, seed=4, inadmissible_frac=0.3)),
    ("csr >32 per state", lambda: mdpgen.csr_ragged(1200, 6, 40, gamma=0.9, seed=5)),
    ("csr m=40", lambda: mdpgen.csr_uniform_k(700, 40, 4, gamma=0.9, seed=6)),
    ("maze", lambda: mdpgen.maze(40, 1500, gamma=0.95, slip=0.2, seed=9)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_cluster_trajectories_match_oracle(name, make):
    mdp = make()
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=7) * 3
    for b in sorted({1, 7, 64, 1000, mdp.n // 2 + 1}):
        if b >= mdp.n or (b == 1 and mdp.n > 2000):
            continue
        ref = oracle.mbvi(mdp, b, seed=19, eps=0.0, max_sweeps=5, V0=V0, start_sweep=2)
        V = torch.from_numpy(V0).cuda()
        st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=19, eps=0.0, max_sweeps=5, start_sweep=2), V)
        T = -(-mdp.n // b)
        expect = "cluster" if b <= 512 else "grid"
        if expect == "cluster":
            assert st["path"] == "cluster" and st["sweeps"] == 5, (b, st)
            assert st["barriers"] == 5 * T          # one cluster barrier per batch
        close(V.cpu().numpy(), ref["V"])


def test_cluster_converged_policy_trace_and_determinism():
    mdp = mdpgen.csr_ragged(3000, 4, 12, gamma=0.97, seed=11, inadmissible_frac=0.2)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 100, seed=5, eps=1e-6, max_sweeps=100000)
    trace = torch.zeros(100000, dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(2):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
        gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=100, seed=5, eps=1e-6, max_sweeps=100000, trace=trace), V, pi, gap)
        assert st["status"] == rmb.RMB_OK and st["path"] == "cluster"
        assert abs(st["sweeps"] - ref["sweeps"]) <= 2
        runs.append((V.clone(), pi.clone(), gap.clone(), st))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])   # reproducible
    V, pi, gap, st = runs[0]
    tr = trace.cpu().numpy()[:st["sweeps"]]
    k = min(st["sweeps"], ref["sweeps"])
    assert np.allclose(tr[:k], ref["deltas"][:k], rtol=1e-3, atol=2e-6)
    assert tr[-1] <= 1e-6 and st["residual"] == tr[-1]
    jstar, pistar, _ = exact.policy_iteration(mdp)
    close(V.cpu().numpy(), jstar)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    sel = jgap > 1e-6 * max(1.0, float(np.abs(jstar).max()))
    assert np.array_equal(pi.cpu().numpy()[sel], pistar[sel])
    _, opi, ogap, _ = oracle.greedy(mdp, V.cpu().numpy().astype(np.float64))
    clear = ogap > 1e-5
    assert np.array_equal(pi.cpu().numpy()[clear], opi[clear])
    fin = clear & np.isfinite(ogap)          # one admissible action: the gap is +inf on both sides
    assert np.array_equal(np.isinf(gap.cpu().numpy()), np.isinf(ogap))
    assert np.max(np.abs(gap.cpu().numpy()[fin] - ogap[fin])) <= 1e-4


def test_cluster_recentring_and_sizes_near_the_limit():
    # start values far from the solution: the centre moves between sweeps (every CTA shifts its copies)
    mdp = mdpgen.csr_uniform_k(14000, 4, 8, gamma=0.95, seed=12)
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = np.full(mdp.n, 500.0, np.float32) + mdpgen.random_values(mdp.n, seed=3)
    ref = oracle.mbvi(mdp, 509, seed=8, eps=0.0, max_sweeps=40, V0=V0)
    V = torch.from_numpy(V0).cuda()
    st = rmb.rmb_vi(dm, rmb.Opts(batch=509, seed=8, eps=0.0, max_sweeps=40), V)
    assert st["path"] == "cluster" and st["sweeps"] == 40
    assert abs(st["v_shift"] - 500.0) > 10.0   # the centre moved from ~500 towards the solution
    close(V.cpu().numpy(), ref["V"])


def test_cluster_statuses():
    mdp = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.99, seed=13)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=100, seed=1, eps=1e-9, max_sweeps=3), V, check=False)[1]
    assert st["status"] == rmb.RMB_ERR_NOT_CONVERGED and st["sweeps"] == 3 and st["path"] == "cluster"
    V[17] = float("nan")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=100, seed=1, eps=1e-6, max_sweeps=30), V, check=False)[1]
    assert st["status"] == rmb.RMB_ERR_NONFINITE
    # a bad index: device validation rejects the MDP before the cluster solve starts
    bad = mdpgen.csr_uniform_k(2000, 4, 8, gamma=0.99, seed=13)
    bad.col = bad.col.copy()
    bad.col[5] = bad.n + 3
    dbad = rmb.DeviceMDP.from_host(bad)
    V = torch.zeros(bad.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dbad, rmb.Opts(batch=100, seed=1, eps=1e-6, max_sweeps=30, validate=True), V, check=False)[1]
    assert st["status"] == rmb.RMB_ERR_INVALID_MDP
    # the context still works afterwards
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    assert rmb.rmb_vi(dm, rmb.Opts(batch=100, seed=1, eps=1e-6, max_sweeps=100000), V)["status"] == rmb.RMB_OK


def test_cluster_is_not_taken_outside_its_scope():
    mdp = mdpgen.csr_uniform_k(3000, 4, 8, gamma=0.95, seed=14)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    for o in (rmb.Opts(batch=3000, eps=0.0, max_sweeps=2),                      # one batch: the grid solve
              rmb.Opts(batch=1000, eps=0.0, max_sweeps=2),                      # more than 2 states per warp
              rmb.Opts(batch=100, eps=0.0, max_sweeps=2, grid_ctas=16),          # explicit grid
              rmb.Opts(batch=100, eps=0.0, max_sweeps=2, select=rmb.RMB_SELECT_UNIFORM),
              rmb.Opts(batch=100, eps=0.0, max_sweeps=2, residual_kind=rmb.RMB_RESIDUAL_BELLMAN),
              rmb.Opts(batch=100, eps=0.0, max_sweeps=2, flags=rmb.RMB_FLAG_NO_CLUSTER)):
        assert rmb.rmb_vi(dm, o, V, check=False)[1]["path"] != "cluster"
    assert rmb.rmb_mpi(dm, rmb.Opts(batch=100, eps=0.0, max_sweeps=2, flags=rmb.RMB_FLAG_NO_CLUSTER), V, pi,
                       check=False)[1]["path"] != "cluster"
    big = mdpgen.csr_uniform_k(15000, 2, 4, gamma=0.9, seed=15)        # 16 bytes per state do not fit
    V = torch.zeros(big.n, dtype=torch.float32, device="cuda")
    assert rmb.rmb_vi(rmb.DeviceMDP.from_host(big), rmb.Opts(batch=100, eps=0.0, max_sweeps=1), V,
                      check=False)[1]["path"] != "cluster"


MPI_CASES = [c for c in CASES if c[0] in ("dense m=11", "csr k=32", "csr ragged", "csr >32 per state", "maze")]


@pytest.mark.parametrize("name,make", MPI_CASES, ids=[c[0] for c in MPI_CASES])
def test_cluster_mpi_matches_oracle_per_iteration(name, make):
    """MB-MPI (Alg. 1) on the cluster: improvement pass (greedy policy at V, ||TV - V||_inf), then K
    sweeps of B_{pi,b} (eq. (12)) over sigma with the sweep counter running on; values after 1 and 3
    outer iterations, the last residual and the policy equal the oracle's MB-MPI, and the grid solve's."""
    mdp = make()
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=8) * 2
    for b, K in ((7, 3), (64, 2)):
        for iters in (1, 3):
            ref = oracle.mpi(mdp, b, K, seed=23, eps=0.0, max_iters=iters, V0=V0, start_sweep=1)
            out = {}
            for flags in (0, rmb.RMB_FLAG_NO_CLUSTER):
                V = torch.from_numpy(V0).cuda()
                pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
                gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
                st = rmb.rmb_mpi(dm, rmb.Opts(batch=b, seed=23, eps=0.0, max_sweeps=iters, eval_sweeps=K,
                                              start_sweep=1, flags=flags), V, pi, gap)
                assert (st["path"] == "cluster") == (flags == 0), (flags, st)
                assert st["iters"] == iters and st["sweeps"] == K * (iters - 1), (b, K, iters, st)
                close(V.cpu().numpy(), ref["V"])
                close([st["residual"]], np.array([ref["resid"][-1]]), tol=1e-5)
                out[flags] = (V.cpu().numpy(), pi.cpu().numpy(), gap.cpu().numpy())
            # the policy of the last improvement pass where it is not a near tie
            Vc, pic, gapc = out[0]
            sel = gapc > 1e-5 * max(1.0, float(np.abs(Vc).max()))
            assert np.array_equal(pic[sel], ref["pi"][sel])
            close(out[0][0], out[rmb.RMB_FLAG_NO_CLUSTER][0])


def test_cluster_mpi_converges_to_the_optimum():
    mdp = mdpgen.csr_uniform_k(3000, 6, 16, gamma=0.97, seed=31)
    dm = rmb.DeviceMDP.from_host(mdp)
    jstar, pistar, _ = exact.policy_iteration(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_mpi(dm, rmb.Opts(batch=128, seed=6, eps=1e-6, max_sweeps=100000, eval_sweeps=10), V, pi)
    assert st["status"] == rmb.RMB_OK and st["path"] == "cluster"
    close(V.cpu().numpy(), jstar)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    sel = jgap > 1e-6 * max(1.0, float(np.abs(jstar).max()))
    assert np.array_equal(pi.cpu().numpy()[sel], pistar[sel])


EVAL_CASES = [c for c in CASES if c[0] in ("dense n%4", "dense m=11", "csr k=32", "csr >32 per state", "csr m=40")]
# rows staged per warp by cp.async (m n <= 2048, n % 4 == 0): the policy's row is picked by its cost
EVAL_CASES.append(("dense staged", lambda: mdpgen.dense_dirichlet(500, 4, gamma=0.95, seed=7)))


@pytest.mark.parametrize("name,make", EVAL_CASES, ids=[c[0] for c in EVAL_CASES])
def test_cluster_policy_evaluation_matches_oracle(name, make):
    """Sweeps of B_{pi,b} (eq. (12)) for a fixed policy on the cluster: trajectories equal the oracle's;
    converged values equal J_pi (eq. (4), a direct solve)."""
    mdp = make()
    dm = rmb.DeviceMDP.from_host(mdp)
    pi = mdpgen.random_policy(mdp.n, mdp.m, seed=5)
    pit = torch.from_numpy(pi).cuda()
    V0 = mdpgen.random_values(mdp.n, seed=4)
    for b in (5, 100):
        ref = oracle.eval_policy(mdp, pi, b, seed=12, eps=0.0, max_sweeps=4, V0=V0)
        V = torch.from_numpy(V0).cuda()
        st = rmb.rmb_eval_policy(dm, pit, rmb.Opts(batch=b, seed=12, eps=0.0, max_sweeps=4), V, check=False)[1]
        assert st["path"] == "cluster" and st["sweeps"] == 4, (b, st)
        close(V.cpu().numpy(), ref["V"])
    J = exact.policy_value(mdp, pi)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_eval_policy(dm, pit, rmb.Opts(batch=64, seed=4, eps=1e-7, max_sweeps=100000), V)
    assert st["status"] == rmb.RMB_OK and st["path"] == "cluster"
    close(V.cpu().numpy(), J)

"""2D-maze stand-ins of Sec. IV-A on the GPU: trajectories equal the FP64 oracle's, and the sweep
counts to ||V - J*||_inf <= 1e-4 (the accuracy of the paper's speed-ups, Sec. IV-B) equal the
oracle's, with J* from exact policy iteration.  The maze rows are ragged (2..5 successors), so this
also covers the generic CSR path, including the one-pass form for states with <= 32 entries."""
import numpy as np
import pytest

import mdpgen
import oracle
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


@pytest.mark.parametrize("b", [1, 64, 700, 1500])
def test_maze_trajectory_matches_oracle(b):
    mdp = mdpgen.maze(40, 1500, gamma=0.95, slip=0.2, seed=9)
    ref = oracle.mbvi(mdp, b, seed=31, eps=0.0, max_sweeps=12, traj=True)
    dm = rmb.DeviceMDP.from_host(mdp)
    want = ref["traj"][-1]
    for flags, path in ((rmb.RMB_FLAG_NO_CLUSTER, "csr-generic"), (0, "cluster" if b <= 512 else "csr-generic")):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=31, eps=0.0, max_sweeps=12, flags=flags), V)
        assert st["path"] == path and st["sweeps"] == 12
        assert np.max(np.abs(V.cpu().numpy() - want)) <= 1e-5 * max(1.0, np.abs(want).max())


def test_maze80_sweeps_to_accuracy_match_oracle():
    mdp = mdpgen.maze80()
    jstar, pistar, _ = exact.policy_iteration(mdp)
    dm = rmb.DeviceMDP.from_host(mdp)
    for b in (512, mdp.n):
        ref = oracle.mbvi(mdp, b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=400, traj=True)
        errs = np.abs(ref["traj"] - jstar).max(axis=1)
        k = int(np.argmax(errs <= TOL)) + 1
        assert errs[k - 1] <= TOL < errs[k - 2]
        for cap in (k - 1, k):
            V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
            rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=cap), V)
            e = float(np.abs(V.cpu().numpy() - jstar).max())
            assert abs(e - errs[cap - 1]) <= 2e-5, (b, cap, e, errs[cap - 1])
    # converged solve: policy equals pi* where the Q-gap is clear
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=512, seed=1, eps=1e-6, max_sweeps=100000), V, pi)
    assert st["status"] == rmb.RMB_OK
    assert np.abs(V.cpu().numpy() - jstar).max() <= 2e-5
    _, _, gap, _ = exact.bellman_pass(mdp, jstar)
    sel = gap > 1e-4
    assert np.array_equal(pi.cpu().numpy()[sel], pistar[sel])


def test_maze100_mpi_k50():
    mdp = mdpgen.maze100()
    jstar, _, _ = exact.policy_iteration(mdp)
    dm = rmb.DeviceMDP.from_host(mdp)
    for b in (512, mdp.n):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_mpi(dm, rmb.Opts(batch=b, seed=2, eps=1e-6, max_sweeps=1000, eval_sweeps=50), V, pi)
        assert st["status"] == rmb.RMB_OK
        assert np.abs(V.cpu().numpy() - jstar).max() <= 2e-5

"""GPU pieces of the row-partitioned form: rmb_backup_states (one backup of a list of states, eq. (7)
restricted to the list, or T_pi) against the FP64 oracle's Q-factors, and partitioned_vi on one rank
(order from rmb_permutation, backups from rmb_backup_states) against the oracle's MB-VI trajectory.
Tolerance: 1e-5 of ||V||_inf (float32 values)."""
import numpy as np
import pytest

import mdpgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402
from paper_2110_02901_b300.partitioned import partitioned_vi  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


@pytest.mark.parametrize("make", [lambda: mdpgen.csr_ragged(3001, 5, 40, gamma=0.95, seed=2, inadmissible_frac=0.2),
                                  lambda: mdpgen.csr_uniform_k(5000, 8, 32, gamma=0.99, seed=3),
                                  lambda: mdpgen.dense_dirichlet(700, 4, gamma=0.95, seed=4)])
def test_backup_states_matches_oracle(make):
    mdp = make()
    dm = rmb.DeviceMDP.from_host(mdp)
    V0 = mdpgen.random_values(mdp.n, seed=8) * 10
    V = torch.from_numpy(V0).cuda()
    states = np.random.default_rng(1).integers(0, mdp.n, 777).astype(np.int32)
    W = rmb.rmb_backup_states(dm, V, torch.from_numpy(states).cuda()).cpu().numpy()
    Vd = V0.astype(np.float64)
    want = np.array([min(oracle.q_factor(mdp, int(s), a, Vd) for a in range(mdp.m)) for s in states])
    scale = max(1.0, float(np.abs(want[np.isfinite(want)]).max()))
    assert np.max(np.abs(W - want)) <= 1e-5 * scale
    pi = oracle.greedy(mdp, Vd)[1]
    Wp = rmb.rmb_backup_states(dm, V, torch.from_numpy(states).cuda(), pi=torch.from_numpy(pi).cuda()).cpu().numpy()
    want_p = np.array([oracle.q_factor(mdp, int(s), int(pi[s]), Vd) for s in states])
    assert np.max(np.abs(Wp - want_p)) <= 1e-5 * scale
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    assert rmb.rmb_backup_states(dm, V, empty).numel() == 0


def test_partitioned_vi_single_rank_matches_oracle():
    mdp = mdpgen.csr_uniform_k(6000, 4, 16, gamma=0.95, seed=6)
    dm = rmb.DeviceMDP.from_host(mdp)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    res = partitioned_vi(dm, rmb.Opts(batch=1000, seed=9, eps=0.0, max_sweeps=8, start_sweep=2), V)
    ref = oracle.mbvi(mdp, 1000, seed=9, eps=0.0, max_sweeps=8, start_sweep=2)
    assert res["sweeps"] == 8
    scale = max(1.0, float(np.abs(ref["V"]).max()))
    assert float(np.abs(V.cpu().numpy() - ref["V"]).max()) <= 1e-5 * scale

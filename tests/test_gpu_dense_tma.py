"""Dense rows through the TMA pipeline (n >= 2048): parity with the FP64 oracle for float32 rows and for
bf16 / fp8 codes (on the decoded, renormalised rows), VI, MPI and policy evaluation, ragged tiles and
row groups, and batches larger than one CTA's state list."""
import numpy as np
import pytest

import mdpgen
import oracle

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
    a = np.asarray(a, np.float64)
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"


def decoded(mdp, lp):
    """Decoded, renormalised rows of a coded MDP (read back from the device; the codes themselves were
    checked against torch's CPU conversion in test_gpu_lowp)."""
    c = lp.P.cpu()
    d = (c.view(torch.float8_e4m3fn) if lp.p_dtype == rmb.RMB_P_FP8E4M3 else c).to(torch.float64).numpy()
    d = d.reshape(mdp.n * mdp.m, mdp.n)
    d = d / d.sum(axis=1, keepdims=True)
    return mdpgen.MDP(n=mdp.n, m=mdp.m, gamma=mdp.gamma, fmt="dense", cost=mdp.cost,
                      P=d.astype(np.float32).reshape(mdp.n, mdp.m, mdp.n))


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("n,m,b", [(2048, 16, 256), (2064, 5, 700), (4096, 3, 4096)])
def test_tma_vi_trajectory(storage, n, m, b):
    mdp = mdpgen.dense_dirichlet(n, m, alpha=0.1, gamma=0.999, seed=n + m, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    form, ref_mdp = dm, mdp
    if storage != "f32":
        form = rmb.dense_lowp(dm, rmb.RMB_P_BF16 if storage == "bf16" else rmb.RMB_P_FP8E4M3)
        ref_mdp = decoded(mdp, form)
    V0 = mdpgen.random_values(n, seed=2)
    ref = oracle.mbvi(ref_mdp, b, seed=11, eps=0.0, max_sweeps=3, V0=V0, traj=True)
    V = torch.from_numpy(V0).cuda()
    st = rmb.rmb_vi(form, rmb.Opts(batch=b, seed=11, eps=0.0, max_sweeps=3, flags=rmb.RMB_FLAG_NO_CLUSTER), V)
    assert st["path"] == "dense-tma" and st["sweeps"] == 3
    close(V.cpu().numpy(), ref["traj"][2])


@pytest.mark.parametrize("storage", ["f32", "fp8"])
def test_tma_mpi_and_evaluation(storage):
    n, m = 2048, 8
    mdp = mdpgen.dense_dirichlet(n, m, alpha=0.5, gamma=0.95, seed=5, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    form, ref_mdp = dm, mdp
    if storage != "f32":
        form = rmb.dense_lowp(dm, rmb.RMB_P_FP8E4M3)
        ref_mdp = decoded(mdp, form)
    ref = oracle.mpi(ref_mdp, 128, K=5, seed=3, eps=0.0, max_iters=3)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    pi = torch.empty(n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_mpi(form, rmb.Opts(batch=128, seed=3, eps=0.0, max_sweeps=3, eval_sweeps=5,
                                    flags=rmb.RMB_FLAG_NO_CLUSTER), V, pi)
    assert st["path"] == "dense-tma" and st["iters"] == 3
    close(V.cpu().numpy(), ref["V"])
    pol = mdpgen.random_policy(n, m, seed=4)
    ev = oracle.eval_policy(ref_mdp, pol, 300, seed=8, eps=0.0, max_sweeps=4)
    V2 = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_eval_policy(form, torch.from_numpy(pol).cuda(),
                             rmb.Opts(batch=300, seed=8, eps=0.0, max_sweeps=4, flags=rmb.RMB_FLAG_NO_CLUSTER), V2)
    assert st["path"] == "dense-tma"
    close(V2.cpu().numpy(), ev["V"])


def test_tma_converged_with_policy_and_against_the_old_path(monkeypatch):
    n, m = 2048, 4
    mdp = mdpgen.dense_dirichlet(n, m, alpha=1.0, gamma=0.95, seed=9)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, 512, seed=2, eps=1e-6, max_sweeps=100000)
    out = {}
    for tma in (True, False):
        if not tma:
            monkeypatch.setenv("RMB_DENSE_NO_TMA", "1")
        V = torch.zeros(n, dtype=torch.float32, device="cuda")
        pi = torch.empty(n, dtype=torch.int32, device="cuda")
        gap = torch.empty(n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=512, seed=2, eps=1e-6, max_sweeps=100000, flags=rmb.RMB_FLAG_NO_CLUSTER),
                        V, pi, gap)
        assert st["path"] == ("dense-tma" if tma else "dense")
        close(V.cpu().numpy(), ref["V"])
        out[tma] = (pi.cpu().numpy(), gap.cpu().numpy())
    _, opi, ogap, _ = oracle.greedy(mdp, ref["V"])
    sel = ogap > 1e-6 * max(1.0, np.abs(ref["V"]).max())
    for tma in (True, False):
        assert np.array_equal(out[tma][0][sel], opi[sel])


def test_tma_batch_larger_than_one_state_list():
    # b = n = 16384 on 148 CTAs: 111 states per CTA per batch, one chunk; 65536 would need 3 chunks
    n, m = 2048, 2
    mdp = mdpgen.dense_dirichlet(n, m, alpha=1.0, gamma=0.9, seed=12)
    dm = rmb.DeviceMDP.from_host(mdp)
    ref = oracle.mbvi(mdp, n, seed=1, eps=0.0, max_sweeps=2)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=n, seed=1, eps=0.0, max_sweeps=2, grid_ctas=3), V)
    assert st["grid_ctas"] == 3          # 683 states per CTA: two chunks of the state list
    close(V.cpu().numpy(), ref["V"])

"""GPU parity of the differentiable fixed point (softmax-parametrised transitions).

Against the oracle's direct-solve gradient (exact.fixed_point_gradient: adjoint by sparse LU / GMRES)
and against central finite differences in FP64 (h = 1e-4) of the exact value at the greedy policy,
on coordinates whose state has a clear Q-gap (so the optimal policy does not change at +-h).
Tolerance for FP32 gradients: |g_gpu - g_ref| <= 2e-5 * max(1, ||g_ref||_inf) (lambda is summed in
float32 over ~1/(1-gamma) discounted terms of magnitude up to ||w|| / (1-gamma)).
"""
import dataclasses

import numpy as np
import pytest

import mdpgen
from oracle import exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402
from paper_2110_02901_b300.autograd import fixed_point  # noqa: E402

GTOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    rmb.lib()


def close(a, b, tol):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"


def gpu_forward(mdp, b=256, eps=1e-7):
    dm = rmb.DeviceMDP.from_host(mdp)
    z = torch.from_numpy(mdp.logits).cuda()
    rmb.rmb_softmax_rows(dm, z, dm.prob)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    gap = torch.empty(mdp.n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=12345, eps=eps, max_sweeps=100000), V, pi, gap)
    assert st["status"] == rmb.RMB_OK
    return dm, z, V, pi, gap


def test_softmax_rows():
    mdp = mdpgen.csr_uniform_k(3000, 4, 16, gamma=0.95, seed=1, prob_kind="softmax")
    dm = rmb.DeviceMDP.from_host(mdp)
    out = torch.empty_like(dm.prob)
    rmb.rmb_softmax_rows(dm, torch.from_numpy(mdp.logits).cuda(), out)
    want = exact.softmax_rows(mdp.logits, mdp.row_ptr)
    assert np.max(np.abs(out.cpu().numpy() - want)) < 1e-6


@pytest.mark.parametrize("n,m,k,g,b", [(3000, 4, 16, 0.95, 64), (5000, 8, 16, 0.95, 5000), (2000, 3, 32, 0.9, 1)])
def test_gradient_matches_direct_solve(n, m, k, g, b):
    mdp = mdpgen.csr_uniform_k(n, m, k, gamma=g, seed=n + m, prob_kind="softmax")
    dm, z, V, pi, gap = gpu_forward(mdp)
    w = mdpgen.random_values(n, seed=7).astype(np.float64)
    lam, gc, gz, jstar, pistar = exact.fixed_point_gradient(mdp, w)
    scale = max(1.0, float(np.abs(jstar).max()))
    close(V.cpu().numpy(), jstar, 1e-5)
    _, _, jgap, _ = exact.bellman_pass(mdp, jstar)
    clear = jgap > 1e-6 * scale
    assert np.array_equal(pi.cpu().numpy()[clear], pistar[clear])
    if not np.array_equal(pi.cpu().numpy(), pistar):
        pytest.skip("a near-tie changes the greedy policy; gradients differ by construction")
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    lam_g, gc_g, gz_g, st = rmb.rmb_fixed_point_grad(dm, pi, V, wt, rmb.Opts(batch=b, seed=3, eps=1e-7, max_sweeps=100000))
    assert st["status"] == rmb.RMB_OK
    close(lam_g.cpu().numpy(), lam, GTOL)
    close(gc_g.cpu().numpy(), gc, GTOL)
    close(gz_g.cpu().numpy(), gz, GTOL)


def _central_differences(mdp, b, w_seed):
    """64 coordinates: 32 logits of greedy rows, 16 costs of greedy actions, 16 uniform costs (kept
    where the state's Q-gap exceeds 1e-3, so the optimal policy is the same at +-h); each compared
    with (L(theta + h) - L(theta - h)) / 2h, L = w . J_pi* from FP64 solves of the perturbed MDP."""
    n = mdp.n
    dm, z, V, pi, gap = gpu_forward(mdp, b=b)
    pi_h = pi.cpu().numpy()
    w = mdpgen.random_values(n, seed=w_seed).astype(np.float64)
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    _, gc_g, gz_g, _ = rmb.rmb_fixed_point_grad(dm, pi, V, wt, rmb.Opts(batch=b, seed=3, eps=1e-7, max_sweeps=100000))
    gc_g, gz_g = gc_g.cpu().numpy().astype(np.float64), gz_g.cpu().numpy().astype(np.float64)
    z0 = mdp.logits.astype(np.float64)
    base = dataclasses.replace(mdp)
    base.prob = exact.softmax_rows(z0, mdp.row_ptr)
    base.cost = mdp.cost.astype(np.float64)
    jstar, pistar, _ = exact.policy_iteration(base)
    _, _, jgap, _ = exact.bellman_pass(base, jstar)
    assert np.array_equal(pi_h[jgap > 1e-4], pistar[jgap > 1e-4])
    h = 1e-4
    rng = np.random.default_rng(0)
    ok_states = np.nonzero(jgap > 1e-3)[0]
    k = int(mdp.row_ptr[1] - mdp.row_ptr[0])      # uniform row length

    def L_of(mod):
        return float(w @ exact.policy_value(mod, pistar))

    coords = []
    for s in rng.choice(ok_states, 32, replace=False):
        r = s * mdp.m + pistar[s]
        coords.append(("z", int(mdp.row_ptr[r]) + int(rng.integers(0, k))))
    for s in rng.choice(ok_states, 16, replace=False):
        coords.append(("c", int(s * mdp.m + pistar[s])))
    for r in rng.integers(0, n * mdp.m, 16):
        if jgap[r // mdp.m] > 1e-3:
            coords.append(("c", int(r)))
    assert len(coords) >= 56
    gmax = max(np.abs(gc_g).max(), 1.0)
    for kind, i in coords:
        mp, mm = dataclasses.replace(base), dataclasses.replace(base)
        if kind == "c":
            mp.cost = base.cost.copy(); mp.cost[i] += h
            mm.cost = base.cost.copy(); mm.cost[i] -= h
            got = gc_g[i]
        else:
            zp, zm = z0.copy(), z0.copy()
            zp[i] += h
            zm[i] -= h
            mp.prob = exact.softmax_rows(zp, mdp.row_ptr)
            mm.prob = exact.softmax_rows(zm, mdp.row_ptr)
            got = gz_g[i]
        fd = (L_of(mp) - L_of(mm)) / (2 * h)
        assert abs(got - fd) <= GTOL * gmax, (kind, i, got, fd)


def test_gradient_matches_central_differences():
    mdp = mdpgen.csr_uniform_k(4096, 8, 16, gamma=0.95, seed=4, prob_kind="softmax")
    _central_differences(mdp, 256, 11)


def test_gradient_matches_central_differences_full_size():
    """The differentiable fixed point at full size (n = 65536, m = 8, k = 16, gamma = 0.95) in the
    bench's launch configuration (b = 16384 for the forward and the adjoint solve)."""
    _central_differences(mdpgen.config5(), 16384, 13)


def test_autograd_function_and_full_size_config():
    mdp = mdpgen.config5()                       # n = 65536, m = 8, k = 16, gamma = 0.95
    dm = rmb.DeviceMDP.from_host(mdp)
    cost = torch.from_numpy(mdp.cost).cuda().requires_grad_(True)
    logits = torch.from_numpy(mdp.logits).cuda().requires_grad_(True)
    opts = rmb.Opts(batch=16384, seed=12345, eps=1e-7, max_sweeps=100000)     # the bench's launch configuration
    V, pi = fixed_point(cost, logits, dm, opts, rmb.Opts(batch=16384, seed=5, eps=1e-7, max_sweeps=100000))
    w = mdpgen.random_values(mdp.n, seed=13).astype(np.float64)
    loss = (torch.from_numpy(w.astype(np.float32)).cuda() * V).sum()
    gcost, glog = torch.autograd.grad(loss, [cost, logits])
    lam, gc, gz, jstar, pistar = exact.fixed_point_gradient(mdp, w)
    close(V.detach().cpu().numpy(), jstar, 1e-5)
    if not np.array_equal(pi.cpu().numpy(), pistar):
        pytest.skip("a near-tie changes the greedy policy")
    close(gcost.cpu().numpy(), gc, GTOL)
    close(glog.cpu().numpy(), gz, GTOL)

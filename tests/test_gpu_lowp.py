"""Low-precision dense transitions (bf16 / fp8-e4m3 codes with per-row scales) and float32 refinement.

* the device quantiser equals torch's CPU conversion of P / scale bit for bit;
* a low-precision solve equals the FP64 oracle run on the decoded, renormalised rows (that is the
  operator the kernel applies) within the FP32 value tolerance;
* the refined solve (low precision, then float32 sweeps) equals the oracle on the float32 problem;
* the error of the unrefined low-precision solution against the float32 problem is reported.
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
    a = np.asarray(a, np.float64)
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= tol * scale, f"{err:.3e} > {tol:.0e} * {scale:.3e}"
    return err


def cpu_codes(P2d, dt):
    """Reference quantisation with torch on the CPU (a library conversion, not the CUDA path)."""
    P = torch.from_numpy(P2d)
    mx = P.max(dim=1).values
    if dt == rmb.RMB_P_FP8E4M3:
        sc = torch.where(mx > 0, mx / 448.0, torch.ones_like(mx))
        codes = (P / sc[:, None]).to(torch.float8_e4m3fn)
    else:
        sc = torch.where(mx > 0, mx, torch.ones_like(mx))
        codes = (P / sc[:, None]).to(torch.bfloat16)
    return codes, sc


def decoded_mdp(mdp, codes):
    """The MDP the low-precision kernel applies: decoded codes, each row divided by its sum."""
    d = codes.to(torch.float64).numpy()
    d = d / d.sum(axis=1, keepdims=True)
    out = mdpgen.MDP(n=mdp.n, m=mdp.m, gamma=mdp.gamma, fmt="dense", cost=mdp.cost,
                     P=d.astype(np.float32).reshape(mdp.n, mdp.m, mdp.n))
    return out


@pytest.mark.parametrize("dt", [rmb.RMB_P_BF16, rmb.RMB_P_FP8E4M3])
def test_quantiser_matches_cpu_conversion(dt):
    mdp = mdpgen.dense_dirichlet(1024, 4, alpha=0.1, gamma=0.999, seed=3, cost_dist="normal")
    P2 = mdp.P.reshape(-1, mdp.n)
    dm = rmb.DeviceMDP.from_host(mdp)
    codes, scale = rmb.rmb_quantize_rows(dm.P.reshape(-1), P2.shape[0], P2.shape[1], dt)
    want, sc = cpu_codes(P2, dt)
    dec_sum = want.to(torch.float64).sum(dim=1)
    assert torch.allclose(1.0 / scale.cpu().to(torch.float64), dec_sum, rtol=1e-6, atol=0)
    if dt == rmb.RMB_P_FP8E4M3:
        assert torch.equal(codes.cpu().reshape(P2.shape), want.view(torch.uint8))
    else:
        assert torch.equal(codes.cpu().reshape(P2.shape), want)


@pytest.mark.parametrize("dt", [rmb.RMB_P_BF16, rmb.RMB_P_FP8E4M3])
@pytest.mark.parametrize("n,m,b", [(1024, 16, 256), (512, 8, 512), (400, 3, 33)])
def test_lowp_trajectory_matches_oracle_on_decoded_rows(dt, n, m, b):
    mdp = mdpgen.dense_dirichlet(n, m, alpha=0.1, gamma=0.999, seed=n + m, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    lp = rmb.dense_lowp(dm, dt)
    codes, _ = cpu_codes(mdp.P.reshape(-1, n), dt)
    dec = decoded_mdp(mdp, codes)
    V0 = mdpgen.random_values(n, seed=1)
    ref = oracle.mbvi(dec, b, seed=9, eps=0.0, max_sweeps=4, V0=V0, traj=True)
    V = torch.from_numpy(V0).cuda()
    st = rmb.rmb_vi(lp, rmb.Opts(batch=b, seed=9, eps=0.0, max_sweeps=4), V)
    assert st["sweeps"] == 4 and st["path"] == "dense"
    close(V.cpu().numpy(), ref["traj"][3])


@pytest.mark.parametrize("dt", [rmb.RMB_P_BF16, rmb.RMB_P_FP8E4M3])
def test_row_sums_from_quantiser_or_on_the_fly_agree(dt):
    mdp = mdpgen.dense_dirichlet(640, 8, alpha=0.1, gamma=0.99, seed=2, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    lp = rmb.dense_lowp(dm, dt)
    raw = rmb.DeviceMDP(lp.n, lp.m, lp.gamma, "dense", lp.cost, P=lp.P, p_dtype=dt, row_scale=None)
    out = []
    for form in (lp, raw):
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        rmb.rmb_vi(form, rmb.Opts(batch=32, seed=4, eps=0.0, max_sweeps=30), V)
        out.append(V.cpu().numpy())
    close(out[0], out[1].astype(np.float64), tol=1e-6)


@pytest.mark.parametrize("dt", [rmb.RMB_P_BF16, rmb.RMB_P_FP8E4M3])
def test_converged_lowp_and_refined_solutions(dt):
    n, m, b = 512, 8, 64
    mdp = mdpgen.dense_dirichlet(n, m, alpha=0.1, gamma=0.99, seed=7, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    lp = rmb.dense_lowp(dm, dt)
    codes, _ = cpu_codes(mdp.P.reshape(-1, n), dt)
    dec = decoded_mdp(mdp, codes)
    ref_lp = oracle.mbvi(dec, b, seed=5, eps=1e-7, max_sweeps=100000)
    ref = oracle.mbvi(mdp, b, seed=5, eps=1e-7, max_sweeps=100000)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = rmb.rmb_vi(lp, rmb.Opts(batch=b, seed=5, eps=1e-7, max_sweeps=100000), V)
    assert st["status"] == rmb.RMB_OK
    close(V.cpu().numpy(), ref_lp["V"])
    lowp_err = float(np.abs(V.cpu().numpy() - ref["V"]).max()) / float(np.abs(ref["V"]).max())
    V2 = torch.zeros(n, dtype=torch.float32, device="cuda")
    pi = torch.empty(n, dtype=torch.int32, device="cuda")
    s1, s2 = rmb.rmb_vi_refined(lp, dm, rmb.Opts(batch=b, seed=5, eps=1e-7, max_sweeps=100000), 1e-7, V2, pi)
    assert s2["status"] == rmb.RMB_OK
    ref_err = close(V2.cpu().numpy(), ref["V"]) / max(1.0, float(np.abs(ref["V"]).max()))
    print(f"dtype={dt}: relative error vs float32 problem, low precision {lowp_err:.2e}, refined {ref_err:.2e}, "
          f"sweeps {s1['sweeps']} + {s2['sweeps']}")
    assert ref_err < lowp_err


def test_refined_solve_with_model_batch():
    """batch = 0 in rmb_vi_refined: one b (the model's, for the float32 rows) for both solves, in the
    workspace sized for the float32 MDP.  The result equals the oracle's two phases at the same sweep
    counts: MB-VI on the decoded fp8 rows, then MB-VI on the float32 rows from there."""
    n = 2048
    mdp = mdpgen.dense_dirichlet(n, 8, alpha=0.1, gamma=0.99, seed=7, cost_dist="normal")
    dm = rmb.DeviceMDP.from_host(mdp)
    lp = rmb.dense_lowp(dm, rmb.RMB_P_FP8E4M3)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    s1, s2 = rmb.rmb_vi_refined(lp, dm, rmb.Opts(batch=0, seed=5, eps=1e-6, max_sweeps=100000), 1e-6, V)
    assert s2["status"] == rmb.RMB_OK and s1["batch"] == s2["batch"] >= 1
    b = s2["batch"]
    codes, _ = cpu_codes(mdp.P.reshape(-1, n), rmb.RMB_P_FP8E4M3)
    ref1 = oracle.mbvi(decoded_mdp(mdp, codes), b, seed=5, eps=0.0, max_sweeps=s1["sweeps"])
    ref2 = oracle.mbvi(mdp, b, seed=5, eps=0.0, max_sweeps=s2["sweeps"], V0=ref1["V"])
    close(V.cpu().numpy(), ref2["V"])


def _rows_only_mdp(n, m, gamma, s, rows, cost_s):
    """A CSR MDP in the oracle's layout that holds state s's m dense rows (all n successors) and a
    self-loop everywhere else: enough for the oracle to evaluate Q(s, a, J) on the full-size problem."""
    lens = np.ones(n * m, dtype=np.int64)
    lens[s * m:(s + 1) * m] = n
    row_ptr = np.zeros(n * m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.repeat(np.arange(n, dtype=np.int32), m)          # self-loops (row r = t*m + a -> state t)
    prob = np.ones(n * m, dtype=np.float32)
    col = list(np.split(col, np.arange(1, n * m)))
    prob = list(np.split(prob, np.arange(1, n * m)))
    for a in range(m):
        col[s * m + a] = np.arange(n, dtype=np.int32)
        prob[s * m + a] = rows[a].astype(np.float32)
    cost = np.zeros(n * m, dtype=np.float32)
    cost[s * m:(s + 1) * m] = cost_s
    return mdpgen.MDP(n=n, m=m, gamma=gamma, fmt="csr", cost=cost, row_ptr=row_ptr,
                      col=np.concatenate(col), prob=np.concatenate(prob))


@pytest.mark.parametrize("dt", [None, rmb.RMB_P_FP8E4M3])
def test_dense_config4_full_size_sampled(dt):
    """The dense workload at full size (n = 16384, m = 16, Dirichlet(0.1), gamma = 0.999, P drawn on the
    device) in the bench's launch configuration (b = 4096): one sweep from random values.  Every state of
    the first batch reads only the start values, so its new value is min_a Q(s, a, V0); for sampled
    states the FP64 oracle evaluates Q on the state's rows (float32 rows, or the fp8 codes of the same
    rows converted on the CPU by torch and renormalised)."""
    n, m, b, g = 16384, 16, 4096, 0.999
    P, cost = mdpgen.dense_dirichlet_device(n, m, 0.1, g, seed=3)
    d32 = rmb.DeviceMDP(n, m, g, "dense", cost, P=P.reshape(-1))
    dm = d32 if dt is None else rmb.dense_lowp(d32, dt)
    V0 = mdpgen.random_values(n, seed=4)
    V = torch.from_numpy(V0).cuda()
    st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=77, eps=0.0, max_sweeps=1, validate=False), V)
    assert st["path"] == "dense-tma"
    v1 = V.cpu().numpy().astype(np.float64)
    sample = np.random.default_rng(1).choice(oracle.perm(n, 77, 0)[:b], size=4, replace=False)
    rows = P[torch.from_numpy(sample).cuda()].cpu().numpy()
    costs = cost.cpu().numpy().reshape(n, m)
    for i, s in enumerate(sample):
        R = rows[i]
        if dt is not None:
            codes, _ = cpu_codes(R, dt)
            d = codes.to(torch.float64).numpy()
            R = d / d.sum(axis=1, keepdims=True)
        mdp = _rows_only_mdp(n, m, g, int(s), R, costs[s])
        want = min(oracle.q_factor(mdp, int(s), a, V0.astype(np.float64)) for a in range(m))
        assert abs(v1[s] - want) <= 1e-5 * max(1.0, abs(want)), (s, v1[s], want)


def test_dense_config4_full_size_certified():
    """The dense workload at full size (n = 16384, m = 16, Dirichlet(0.1) rows, N(0,1) costs,
    gamma = 0.999, P drawn on the device) in the bench's launch configuration (b = 4096), solved to a
    sweep residual of 1e-6 with float32 rows, with bf16 codes + float32 refinement and with fp8 codes +
    float32 refinement.  The FP64 oracle solves the same MDP exactly: policy iteration from the greedy
    policy of the costs, each policy value by a dense LU of (I - gamma P_pi), each improvement by a
    Bellman pass over all 17 GB of rows streamed to the host in chunks, until the policy repeats; then
    T J = J (eq. (5)) certifies J = J*.  Every storage type's values must equal J* within 1e-5 of
    ||J*||_inf and its greedy policy must be the optimal one wherever J*'s Q-gap is clear."""
    n, m, b, g = 16384, 16, 4096, 0.999
    P, cost = mdpgen.dense_dirichlet_device(n, m, 0.1, g, seed=3)
    d32 = rmb.DeviceMDP(n, m, g, "dense", cost, P=P.reshape(-1))
    opts = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000, validate=False)
    out = {}
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    pi = torch.empty(n, dtype=torch.int32, device="cuda")
    st = rmb.rmb_vi(d32, opts, V, pi)
    assert st["status"] == rmb.RMB_OK and st["path"] == "dense-tma"
    out["f32"] = (V.cpu().numpy().astype(np.float64), pi.cpu().numpy())
    for name, dt in (("bf16", rmb.RMB_P_BF16), ("fp8", rmb.RMB_P_FP8E4M3)):
        lp = rmb.dense_lowp(d32, dt)
        V.zero_()
        s1, s2 = rmb.rmb_vi_refined(lp, d32, opts, 1e-6, V, pi)
        assert s1["status"] == rmb.RMB_OK and s2["status"] == rmb.RMB_OK
        out[name] = (V.cpu().numpy().astype(np.float64), pi.cpu().numpy())
        del lp
    rows = P.reshape(n * m, n)
    cert = exact.dense_policy_iteration(lambda r0, r1: rows[r0:r1].cpu().numpy(),
                                        lambda idx: rows[torch.from_numpy(np.asarray(idx)).cuda()].cpu().numpy(),
                                        cost.cpu().numpy(), g, n, m, chunk_states=256)
    jstar = cert["J"]
    scale = max(1.0, float(np.abs(jstar).max()))
    # the certificate: ||T J - J||_inf at FP64 rounding level, so ||J - J*|| <= resid / (1 - gamma) is tiny
    assert cert["resid"] / (1 - g) <= 1e-8 * scale, cert["resid"]
    clear = cert["gap"] > 1e-6 * scale
    assert clear.mean() > 0.99
    for name, (v, p) in out.items():
        err = float(np.abs(v - jstar).max())
        print(f"dense n=16384 {name}: sup-norm error vs certified J* {err:.3e} (relative {err / scale:.2e}), "
              f"policy iterations {cert['iters']}")
        assert err <= RTOL * scale, (name, err, scale)
        assert np.array_equal(p[clear], cert["pi"][clear]), name

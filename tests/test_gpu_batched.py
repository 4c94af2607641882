"""Batched MB-VI: many uneven MDPs in one persistent launch (autotuned b and CTA groups).

Every MDP's result must equal rmb_vi's on the same MDP with the same b, seed and options bit for bit
(the summation order of a state does not depend on how many CTAs share the solve), and the oracle's
MB-VI within the FP32 value tolerance (1e-5 relative).
"""
import numpy as np
import pytest

import mdpgen
import oracle

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


def _mdps():
    out = mdpgen.batched_uneven(36, 256, 8192, 16, seed=21)          # uneven CSR, k = 16
    out.append(mdpgen.csr_uniform_k(20000, 8, 32, gamma=0.99, seed=3))  # one big one: gets a CTA group
    out.append(mdpgen.csr_ragged(700, 3, 9, gamma=0.9, seed=4))         # ragged rows: generic path
    out.append(mdpgen.csr_uniform_k(900, 5, 12, gamma=0.93, seed=5))    # k % 4 == 0 but k/4 = 3
    out.append(mdpgen.csr_uniform_k(600, 16, 16, gamma=0.95, seed=6))   # two chunks per lane
    return out


def _run_batch(mdps, opts, stream=None):
    dms = [rmb.DeviceMDP.from_host(m) for m in mdps]
    Vs = [torch.zeros(m.n, dtype=torch.float32, device="cuda") for m in mdps]
    pis = [torch.empty(m.n, dtype=torch.int32, device="cuda") for m in mdps]
    B = rmb.Batch(dms, Vs, opts, pis=pis)
    return dms, Vs, pis, B


def test_batched_equals_single_solves_and_oracle():
    mdps = _mdps()
    opts = rmb.Opts(batch=1, seed=12345, eps=1e-6, max_sweeps=100000)
    dms, Vs, pis, B = _run_batch(mdps, opts)
    plan = B.plan_table()
    assert any(p["group_ctas"] > 1 for p in plan)          # the big MDP got a group of CTAs
    # groups have fixed CTAs; MDPs solved alone come from the shared queue
    assert all((p["first_cta"] >= 0) if p["group_ctas"] > 1 else (p["group_ctas"] == 1 and p["first_cta"] == -1)
               for p in plan)
    B.run()
    res = B.results()
    for i, (m, dm) in enumerate(zip(mdps, dms)):
        assert res[i]["status"] == rmb.RMB_OK, (i, res[i])
        V1 = torch.zeros(m.n, dtype=torch.float32, device="cuda")
        pi1 = torch.empty(m.n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=plan[i]["batch"], seed=12345, eps=1e-6, max_sweeps=100000,
                                     flags=rmb.RMB_FLAG_NO_CLUSTER), V1, pi1)
        assert st["sweeps"] == res[i]["sweeps"], i
        assert torch.equal(V1, Vs[i]), i
        assert torch.equal(pi1, pis[i]), i
    for i in (0, 7, len(mdps) - 4, len(mdps) - 3, len(mdps) - 1):
        ref = oracle.mbvi(mdps[i], plan[i]["batch"], seed=12345, eps=1e-6, max_sweeps=100000)
        v = Vs[i].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(v - ref["V"])) <= 1e-5 * max(1.0, np.abs(ref["V"]).max()), i


def test_batched_graph_capture_and_replay():
    mdps = mdpgen.batched_uneven(24, 256, 4096, 16, seed=33)
    opts = rmb.Opts(batch=1, seed=7, eps=1e-6, max_sweeps=100000)
    dms, Vs, pis, B = _run_batch(mdps, opts)
    s = torch.cuda.Stream()
    B.run(stream=s)
    r1 = B.results(stream=s)          # waits for stream s
    first = [v.clone() for v in Vs]
    B.capture(s)
    for _ in range(2):
        with torch.cuda.stream(s):
            for v in Vs:
                v.zero_()
        B.replay(s)
        r2 = B.results(stream=s)
        torch.cuda.synchronize()
        for a, b in zip(first, Vs):
            assert torch.equal(a, b)
        assert [x["sweeps"] for x in r1] == [x["sweeps"] for x in r2]


def test_batched_fixed_batch_sizes_are_respected():
    mdps = mdpgen.batched_uneven(8, 300, 2000, 16, seed=44)
    dms = [rmb.DeviceMDP.from_host(m) for m in mdps]
    Vs = [torch.zeros(m.n, dtype=torch.float32, device="cuda") for m in mdps]
    bs = [1, 7, 64, 100, m_n := mdps[4].n, 3, 1000000, 50]
    B = rmb.Batch(dms, Vs, rmb.Opts(batch=1, seed=1, eps=0.0, max_sweeps=5), batches=bs)
    plan = B.plan_table()
    for p, b, m in zip(plan, bs, mdps):
        assert p["batch"] == min(b, m.n)
    B.run()
    res = B.results()
    for i, m in enumerate(mdps):
        ref = oracle.mbvi(m, min(bs[i], m.n), seed=1, eps=0.0, max_sweeps=5)
        assert res[i]["sweeps"] == 5
        v = Vs[i].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(v - ref["V"])) <= 1e-5 * max(1.0, np.abs(ref["V"]).max())


def test_batched_full_config_against_single_solves_and_oracle():
    """The bench's batched workload at full size (256 MDPs, n log-uniform in [256, 65536], m in 2..16,
    k = 16) in one launch with the autotuned plan: every MDP converges; every MDP's values, policy and
    sweep count equal a single grid-wide rmb_vi solve at its planned b bit for bit; and 64 MDPs, every fourth
    by size, equal the FP64 oracle's MB-VI at their planned b."""
    mdps = mdpgen.config3()
    opts = rmb.Opts(batch=1, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000)
    dms, Vs, pis, B = _run_batch(mdps, opts)
    B.run()
    res = B.results()
    plan = B.plan_table()
    assert all(r["status"] == rmb.RMB_OK for r in res)
    for i, dm in enumerate(dms):
        V1 = torch.zeros(mdps[i].n, dtype=torch.float32, device="cuda")
        pi1 = torch.empty(mdps[i].n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=plan[i]["batch"], seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000,
                                     validate=False, flags=rmb.RMB_FLAG_NO_CLUSTER), V1, pi1)
        assert st["sweeps"] == res[i]["sweeps"], i
        assert torch.equal(V1, Vs[i]), i
        assert torch.equal(pi1, pis[i]), i
    by_size = np.argsort([m.n for m in mdps], kind="stable")
    for i in by_size[::4]:
        ref = oracle.mbvi(mdps[i], plan[i]["batch"], seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000)
        v = Vs[i].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(v - ref["V"])) <= 1e-5 * max(1.0, np.abs(ref["V"]).max()), i


def test_batched_groups_with_shared_memory_values_odd_batch_counts():
    """MDPs solved by a group of CTAs, each with a copy of the values in shared memory: three batches
    per sweep (the two (state, value) lists alternate across sweeps as well), one MDP whose values
    exceed shared memory (the states past 57344 in L2), start values away from zero (re-centring) and
    greedy outputs; values, policies and sweep counts equal rmb_vi's bit for bit."""
    mdps = [mdpgen.csr_uniform_k(30000, 8, 16, gamma=0.97, seed=41),
            mdpgen.csr_uniform_k(70000, 4, 16, gamma=0.95, seed=42)]
    bs = [10001, 23334]
    dms = [rmb.DeviceMDP.from_host(m) for m in mdps]
    V0 = [mdpgen.random_values(m.n, seed=43 + i, scale=0.5, offset=20.0) for i, m in enumerate(mdps)]
    Vs = [torch.from_numpy(v).cuda() for v in V0]
    pis = [torch.empty(m.n, dtype=torch.int32, device="cuda") for m in mdps]
    opts = rmb.Opts(batch=1, seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000)
    B = rmb.Batch(dms, Vs, opts, pis=pis, batches=bs)
    plan = B.plan_table()
    assert [p["batch"] for p in plan] == bs
    assert all(p["group_ctas"] > 1 for p in plan), plan
    B.run()
    res = B.results()
    assert all(r["status"] == rmb.RMB_OK for r in res)
    for i, dm in enumerate(dms):
        V1 = torch.from_numpy(V0[i]).cuda()
        pi1 = torch.empty(mdps[i].n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=bs[i], seed=mdpgen.PERM_SEED, eps=1e-6, max_sweeps=200000,
                                     flags=rmb.RMB_FLAG_NO_CLUSTER), V1, pi1)
        assert st["sweeps"] == res[i]["sweeps"], i
        assert torch.equal(V1, Vs[i]), i
        assert torch.equal(pi1, pis[i]), i

#!/usr/bin/env python3
"""Benchmark: randomized mini-batch value iteration on the 2^20-state CSR MDP.

Workload (synthetic, seeded): n = 2^20 states, m = 8 actions, k = 32 distinct successors per
(s,a) drawn uniformly without replacement, probabilities ~ Dirichlet(1), costs ~ U[0,1],
gamma = 0.99, FP32 values and probabilities, int32 indices.  One step = one complete MB-VI solve
from V = 0 to a sup-norm sweep residual <= 1e-6 at the headline batch size b, plus the greedy
policy; the metric is Bellman backups/s = n * sweeps / time and the time-to-1e-6.
A b-sweep over {1024, 16384, 262144, 2^20} for MB-VI and MB-MPI (K = 10) is reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--b B] [--no-sweep]

Under torchrun every rank solves its own replica (the method does not shard: batch t+1 reads
batch t's writes through random successors); value = all ranks' backups / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import mdpgen  # noqa: E402

METRIC = "time-to-1e-6 residual and Bellman backups/s vs batch b; P-stream HBM GB/s"
N_STATES, M_ACTIONS, K_SUCC, GAMMA = 1 << 20, 8, 32, 0.99
EPS = 1e-6
CSR_DRAM_BYTES_PER_STATE_PASS = (11167719000 + 10510336) / (21 * 262144)
# batched launch: DRAM bytes (read + write) over the algorithmic row bytes, from one ncu capture of the
# 256-MDP launch with every MDP capped at 20 sweeps (72.6275 GB + 0.1440 GB over 72.0046 GB)
BATCHED_DRAM_PER_ALGO_BYTE = (72627516000 + 144032512) / 72004641408
DENSE_DRAM_BYTES_PER_P_BYTE = (4285076000 + 7139328) / (4 * 4096 * 16 * 4096 * 4)
B_SWEEP = [1024, 16384, 262144, 1 << 20]
HEADLINE_B = 262144
MPI_K = 10


def workload_name(b):
    return (f"csr-mdp n=2^20 m=8 k=32 dirichlet(1) c~U[0,1] gamma=0.99; MB-VI from V=0 to sweep "
            f"residual 1e-6 at b={b}, greedy policy included")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def sweep_bytes(n, m, k):
    """Algorithmic bytes of one pass over all rows: prob (4 B) + col (4 B) per entry + cost (4 B) per row."""
    return n * m * k * 8 + n * m * 4


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clk_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


# ------------------------------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------------------
def cpu_baseline(mdp, b, budget_s=15.0, max_sweeps=200):
    """The FP64 oracle as it stands, on this host's cores: MB-VI sweeps of the same workload from
    V = 0 until budget_s seconds are spent; backups/s = n * sweeps / time."""
    import oracle
    V = np.zeros(mdp.n)
    t0 = time.perf_counter()
    sweeps = 0
    while sweeps < max_sweeps:
        r = oracle.mbvi(mdp, b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=1, V0=V, start_sweep=sweeps)
        V = r["V"]
        sweeps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": mdp.n * sweeps / dt, "unit": "Bellman backups/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{sweeps} MB-VI sweeps (b={b}) of the same n=2^20 workload from V=0, FP64, {dt:.1f} s"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    mdp = mdpgen.config2()
    b = args.b
    for _ in range(args.warmup):
        cpu_baseline(mdp, b, budget_s=0.0, max_sweeps=1)
    times, sweeps = [], 0
    import oracle
    V = np.zeros(mdp.n)
    for s in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.mbvi(mdp, b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=args.ref_sweeps, V0=V, start_sweep=sweeps)
        times.append(time.perf_counter() - t0)
        V = r["V"]
        sweeps += r["sweeps"]
    tot = sum(times)
    value = mdp.n * sweeps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Bellman backups/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(b) + f"; each step = {args.ref_sweeps} FP64 oracle sweeps (bounded sample)",
                   "n": mdp.n, "m": mdp.m, "k": K_SUCC, "batch": b},
        "cpu_baseline": {"value": value, "unit": "Bellman backups/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} x {args.ref_sweeps} MB-VI sweeps of the n=2^20 workload"},
        "e2e": {"value": value, "unit": "Bellman backups/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--b", type=int, default=HEADLINE_B)
    ap.add_argument("--no-sweep", action="store_true", help="skip the b-sweep side table")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the other four workloads in the headline line")
    ap.add_argument("--ref-sweeps", type=int, default=3, help="reference arm: oracle sweeps per step")
    ap.add_argument("--n-log2", type=int, default=20, help="states = 2^n_log2 (profiling of smaller cases)")
    ap.add_argument("--profile-case", type=int, default=0, metavar="SWEEPS",
                    help="profiling mode: one MB-VI solve of exactly SWEEPS sweeps (no bench line)")
    ap.add_argument("--workload", default="csr",
                    choices=["csr", "dense500", "dense16k", "batched", "adjoint", "maze", "select"],
                    help="csr: the headline line (default); the others measure the remaining workloads")
    ap.add_argument("--full", action="store_true", help="dense16k: also time full gamma=0.999 solves at n=16384")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "fp8"],
                    help="dense16k --profile-case: storage type of P")
    ap.add_argument("--profile-batch", default="512",
                    help="maze --profile-case: the batch size, 'n' (one batch) or 'async' (asynchronous sweeps)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload != "csr":
        return run_workload(args, world, rank, local)

    import torch
    import paper_2110_02901_b300 as rmb
    from paper_2110_02901_b300 import build as rbuild
    rbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    n = 1 << args.n_log2
    mdp = mdpgen.config2(n=n)
    dm = rmb.DeviceMDP.from_host(mdp, device=dev)
    b = min(args.b, n)
    launches0 = rmb.rmb_kernel_launches()
    assert rmb.rmb_validate(dm) == rmb.RMB_OK
    opts = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
    ws = rmb.workspace(dm, opts, device=dev)
    V = torch.zeros(n, dtype=torch.float32, device=dev)
    pi = torch.empty(n, dtype=torch.int32, device=dev)
    gap = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    if args.profile_case:
        po = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=args.profile_case, validate=False)
        st = rmb.rmb_vi(dm, po, V, pi, gap, ws=rmb.workspace(dm, po, device=dev), stream=stream)
        gb = (st["sweeps"] + 1) * sweep_bytes(n, M_ACTIONS, K_SUCC) / 1e9
        print(json.dumps({"profile_case": True, "n": n, "b": b, "sweeps": st["sweeps"], "ms": st["ms"],
                          "p_stream_gb": gb, "gbs": gb / (st["ms"] / 1e3), "path": st["path"],
                          "grid_ctas": st["grid_ctas"]}), flush=True)
        return 0

    def solve():
        V.zero_()
        st = rmb.rmb_vi(dm, opts, V, pi, gap, ws=ws, stream=stream)
        assert st["status"] == rmb.RMB_OK, st
        return st

    for _ in range(args.warmup):
        solve()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    l0 = rmb.rmb_kernel_launches()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            stats.append(solve())
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = rmb.rmb_kernel_launches() - l0
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    sweeps = sum(s["sweeps"] for s in stats)
    kernel_ms = sum(s["ms"] for s in stats)   # CUDA events around each launch, on its stream
    backups = n * sweeps
    total_backups = sum_over_ranks(backups, world)
    value = total_backups / (ms_max / 1e3)
    clocks = clk.summary()

    hbm, peak_kind = peaks()
    per_launch_bytes = [(s["sweeps"] + 1) * sweep_bytes(n, M_ACTIONS, K_SUCC) for s in stats]
    achieved = sum(per_launch_bytes) / (kernel_ms / 1e3) / 1e9
    # DRAM bytes per state and pass from one ncu capture of this kernel (n = 2^18, b = 65536, 20 sweeps
    # + the greedy pass: 11.178 GB); the values stay in L2, so traffic scales with states x passes
    traffic = statistics.mean((s["sweeps"] + 1) * n * CSR_DRAM_BYTES_PER_STATE_PASS for s in stats)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "traffic_note": "ncu capture at n=2^18 scaled by states x passes",
                "kernel": "rmb_csr_vec_kernel", "peak_kind": peak_kind,
                "bytes_per_launch": statistics.mean(per_launch_bytes),
                "note": "P stream (prob+col+cost) per sweep x (sweeps + 1 greedy pass) / launch time"}

    # the measured ceiling of the real bound: random 4-byte gathers from a table the size of the values
    g_idx = torch.randint(0, n, (1 << 27,), dtype=torch.int32, device=dev,
                          generator=torch.Generator(device=dev).manual_seed(7))
    g_src = torch.rand(n, dtype=torch.float32, device=dev)
    rmb.rmb_diag_gather_probe(g_src, g_idx, reps=1, stream=stream)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    rmb.rmb_diag_gather_probe(g_src, g_idx, reps=4, stream=stream)
    pe1.record(stream)
    torch.cuda.synchronize()
    ceiling = 4 * g_idx.numel() / (pe0.elapsed_time(pe1) / 1e3)
    # the same gathers issued by the tensor-memory-access unit (tile::gather4 of 16-byte rows)
    rmb.rmb_diag_gather_probe_tma(g_src, g_idx, reps=1, stream=stream)
    pe0.record(stream)
    tma_out = rmb.rmb_diag_gather_probe_tma(g_src, g_idx, reps=4, stream=stream)
    pe1.record(stream)
    torch.cuda.synchronize()
    tma_rate = 4 * g_idx.numel() / (pe0.elapsed_time(pe1) / 1e3) if bool(torch.isfinite(tma_out).all()) else None
    del g_idx, g_src, tma_out
    gathers = sum((st["sweeps"] + 1) * n * M_ACTIONS * K_SUCC for st in stats)
    roofline["gather_bound"] = {"rate_per_s": gathers / (kernel_ms / 1e3), "ceiling_per_s": ceiling,
                                "frac": gathers / (kernel_ms / 1e3) / ceiling,
                                "tma_gather4_per_s": tma_rate,
                                "note": "random successor gathers (one 32-byte L2 sector each) vs the measured rate "
                                        "of random 4-byte gathers from a 4 MB table (rmb_diag_gather_probe); "
                                        "tma_gather4_per_s: the same gathers as tile::gather4 copies "
                                        "(rmb_diag_gather_probe_tma)"}

    # end to end through the public API: pinned host inputs copied in, V and pi copied out, every step
    e2e = None
    if rank == 0 or world > 1:
        h = {k: torch.from_numpy(getattr(mdp, k)).pin_memory() for k in ("cost", "row_ptr", "col", "prob")}
        V0h = torch.zeros(n, dtype=torch.float32).pin_memory()
        Vh = torch.empty(n, dtype=torch.float32).pin_memory()
        pih = torch.empty(n, dtype=torch.int32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in h.values()) + V0h.numel() * 4
        d2h = n * 4 + n * 4

        def e2e_step():
            for k_, t in h.items():
                getattr(dm, k_).copy_(t, non_blocking=True)
            V.copy_(V0h, non_blocking=True)
            st = rmb.rmb_vi(dm, opts, V, pi, gap, ws=ws, stream=stream)
            Vh.copy_(V, non_blocking=True)
            pih.copy_(pi, non_blocking=True)
            torch.cuda.synchronize()
            return st

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        esw = 0
        for _ in range(args.steps):
            esw += e2e_step()["sweeps"]
        et = time.perf_counter() - t0
        e2e = {"value": n * esw / et, "unit": "Bellman backups/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * et / args.steps}

    # b-sweep side table (one warm + one timed solve per entry, outside the headline timing)
    bsweep = []
    if not args.no_sweep and rank == 0:
        for bb in B_SWEEP + ["auto", "async"]:
            # "auto": b chosen by the library's time model (opts.batch = 0); "async": asynchronous
            # sweeps (no barrier between batches, in-place writes)
            label = bb
            flags = rmb.RMB_FLAG_ASYNC if bb == "async" else 0
            bb = n if bb == "async" else (0 if bb == "auto" else min(bb, n))
            for scheme in ("vi", "mpi"):
                o = rmb.Opts(batch=bb, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000 if scheme == "vi" else 20000,
                             eval_sweeps=MPI_K, validate=False, flags=flags)
                w = rmb.workspace(dm, o, device=dev)
                res = None
                for _ in range(2):
                    V.zero_()
                    if scheme == "vi":
                        res = rmb.rmb_vi(dm, o, V, pi, gap, ws=w, stream=stream)
                    else:
                        res = rmb.rmb_mpi(dm, o, V, pi, gap, ws=w, stream=stream)
                passes = (res["sweeps"] + 1) if scheme == "vi" else (res["iters"] + res["sweeps"] / M_ACTIONS)
                gbs = passes * sweep_bytes(n, M_ACTIONS, K_SUCC) / (res["ms"] / 1e3) / 1e9
                bsweep.append({"b": label if isinstance(label, str) else bb, "b_used": res["batch"], "scheme": scheme,
                               "time_to_eps_ms": res["ms"], "sweeps": res["sweeps"],
                               "improvements": res["iters"], "backups_per_s": n * res["sweeps"] / (res["ms"] / 1e3),
                               "p_stream_gbs": gbs, "hbm_frac": gbs / hbm, "residual": res["residual"],
                               "barriers": res["barriers"]})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(mdp, b)

    # the other four workloads (outside the headline's timed region)
    cfgs = None
    if rank == 0 and not args.no_configs:
        del dm, ws
        torch.cuda.empty_cache()
        try:
            cfgs = configs_summary(args, rmb, torch, stream, hbm, peak_kind)
        except Exception as e:   # the headline line is printed whatever happens to the other workloads
            cfgs = {"error": f"{type(e).__name__}: {e}"[:400]}
            try:
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            except Exception:
                pass

    total_launches = rmb.rmb_kernel_launches() - launches0
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Bellman backups/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(b), "n": n, "m": M_ACTIONS, "k": K_SUCC, "gamma": GAMMA,
                       "batch": b, "eps": EPS, "sweeps_per_step": sweeps / args.steps,
                       "sa_backups_per_s": value * M_ACTIONS, "nnz_per_s": value * M_ACTIONS * K_SUCC,
                       "time_to_eps_ms": ms_max / args.steps, "parallelism": f"replicas x{world}",
                       "l2": "inputs (2.2 GB of P per sweep) exceed the 126 MB L2; no flush needed",
                       "validate": "once before timing", "path": stats[-1]["path"],
                       "grid_ctas": stats[-1]["grid_ctas"]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "b_sweep": bsweep, "kernel_launches_total": total_launches,
            "configs": cfgs,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------------
# The other four workloads, measured after the headline's timed region and reported in its line
# ("configs"): each with its time, throughput and roofline fraction.  Oracle work (the dense
# certificate, the n=500 oracle solve) runs only in the CPU-baseline leg (skipped with --no-cpu).
# ------------------------------------------------------------------------------------------------
def _ev_ms(fn, stream, reps=1):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, out = None, None
    for _ in range(reps):
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best, out


def configs_summary(args, rmb, torch, stream, hbm, peak_kind):
    out = {}
    # dense n=500, m=4, b=50 (latency-bound: 10 batches per sweep, P = 4 MB in L2)
    mdp = mdpgen.config1()
    dm = rmb.DeviceMDP.from_host(mdp)
    o = rmb.Opts(batch=50, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=100000, validate=False)
    ws = rmb.workspace(dm, o)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")

    def s1():
        V.zero_()
        return rmb.rmb_vi(dm, o, V, None, None, ws=ws, stream=stream)

    for _ in range(3):
        s1()
    ms, st = _ev_ms(s1, stream, reps=5)
    ach = (st["sweeps"] + 1) * mdp.n * mdp.m * mdp.n * 4 / (st["ms"] / 1e3) / 1e9
    e = {"workload": "dense n=500 m=4 dirichlet(1) c~U[0,1] gamma=0.95, MB-VI b=50 from V=0 to 1e-6",
         "time_to_eps_ms": ms, "sweeps": st["sweeps"], "backups_per_s": mdp.n * st["sweeps"] / (ms / 1e3),
         "barriers": st["barriers"], "us_per_barrier": 1e3 * st["ms"] / max(1, st["barriers"]), "path": st["path"],
         "roofline": {"bound": "latency", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                      "peak_kind": peak_kind,
                      "kernel": "rmb_small_kernel" if st["path"] == "cluster" else "rmb_dense_kernel<f32>",
                      "note": "P (4 MB) stays in L2; each of the 10 batches per sweep costs one barrier (a "
                              "hardware cluster barrier on the one-cluster path) plus the exchange of the "
                              "batch's values"}}
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.mbvi(mdp, 50, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=100000)
        ct = time.perf_counter() - t0
        e["max_abs_err_vs_oracle"] = float(np.abs(V.cpu().numpy() - ref["V"]).max())
        e["cpu_baseline"] = {"value": ct * 1e3, "unit": "ms to 1e-6", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"full FP64 solve, {ref['sweeps']} sweeps"}
    out["dense500"] = e
    del dm, ws, V

    # 256 uneven CSR MDPs: one graph-captured launch vs one rmb_vi launch per MDP (same b)
    mdps = mdpgen.config3()
    dms = [rmb.DeviceMDP.from_host(x) for x in mdps]
    tot_n = sum(x.n for x in mdps)
    Vall = torch.zeros(tot_n, dtype=torch.float32, device="cuda")
    Vs, off = [], 0
    for x in mdps:
        Vs.append(Vall[off:off + x.n])
        off += x.n
    o = rmb.Opts(batch=1, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
    s = torch.cuda.Stream()
    B = rmb.Batch(dms, Vs, o, stream=s)
    B.capture(s)

    def s3():
        with torch.cuda.stream(s):
            Vall.zero_()
        B.replay(s)

    for _ in range(2):
        s3()
    ms, _ = _ev_ms(s3, s, reps=3)
    res = B.results(stream=s)
    plan = B.plan_table()
    seq = 0.0
    for x, d, p_ in zip(mdps, dms, plan):
        oo = rmb.Opts(batch=p_["batch"], seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
        Vx = torch.zeros(x.n, dtype=torch.float32, device="cuda")
        seq += rmb.rmb_vi(d, oo, Vx)["ms"]
    nnz_passes = sum((r["sweeps"] + 1) * x.nnz * 8 for x, r in zip(mdps, res))
    ach = nnz_passes / (ms / 1e3) / 1e9
    out["batched256"] = {
        "workload": "256 csr-mdps n~logU[256,65536] m~U{2..16} k=16 dirichlet(1) gamma~U[0.9,0.99], MB-VI to 1e-6, "
                    "autotuned b, one CUDA-graph launch",
        "time_to_eps_ms": ms, "per_mdp_launches_ms": seq, "speedup_vs_per_mdp_launches": seq / ms,
        "backups_per_s": sum(x.n * r["sweeps"] for x, r in zip(mdps, res)) / (ms / 1e3),
        "all_converged": all(r["status"] == rmb.RMB_OK for r in res),
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "peak_kind": peak_kind, "kernel": "rmb_batched_kernel",
                     "note": "algorithmic bytes: (sweeps + 1) x nnz x 8 per MDP"}}
    del B, dms, Vs, Vall
    torch.cuda.empty_cache()

    # dense n=16384, m=16, gamma=0.999, b=4096: time to 1e-6 per storage type, errors vs the certified J*
    n, m, b = 16384, 16, 4096
    P, cost = mdpgen.dense_dirichlet_device(n, m, 0.1, 0.999, seed=3)
    d32 = rmb.DeviceMDP(n, m, 0.999, "dense", cost, P=P.reshape(-1), name="dense16k")
    o = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
    ws = rmb.workspace(d32, o)
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    rows = {}
    vals = {}
    for name in ("f32", "bf16", "fp8"):
        form = d32 if name == "f32" else rmb.dense_lowp(d32, rmb.RMB_P_BF16 if name == "bf16" else rmb.RMB_P_FP8E4M3)
        eb = {"f32": 4, "bf16": 2, "fp8": 1}[name]
        wo = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=20, validate=False)
        rmb.rmb_vi(form, wo, V, ws=ws, stream=stream)                        # warm-up (20 sweeps)
        V.zero_()
        if name == "f32":
            t, st = _ev_ms(lambda: rmb.rmb_vi(d32, o, V, ws=ws, stream=stream), stream)
            sw_low, sw_ref = st["sweeps"], 0
        else:
            t, (sa, sb) = _ev_ms(lambda: rmb.rmb_vi_refined(form, d32, o, EPS, V, ws=ws, stream=stream), stream)
            sw_low, sw_ref = sa["sweeps"], sb["sweeps"]
        pbytes = sw_low * n * m * n * eb + sw_ref * n * m * n * 4
        ach = pbytes / (t / 1e3) / 1e9
        rows[name if name == "f32" else name + "+f32 refinement"] = {
            "time_to_eps_ms": t, "sweeps": sw_low, "refinement_sweeps": sw_ref,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "peak_kind": peak_kind, "kernel": f"rmb_dense_tma_kernel<{name}>",
                         "note": "P bytes streamed by all sweeps (codes, then float32 rows) / solve time"}}
        vals[name] = V.cpu().numpy().astype(np.float64)
        if form is not d32:
            del form
    e = {"workload": "dense n=16384 m=16 dirichlet(0.1) c~N(0,1) gamma=0.999, MB-VI b=4096 from V=0 to 1e-6; "
                     "P stored f32 / bf16 codes / fp8-e4m3 codes (+ float32 refinement sweeps)",
         "solves": rows}
    f32_ms = rows["f32"]["time_to_eps_ms"]
    e["speedup_vs_f32"] = {k: f32_ms / r["time_to_eps_ms"] for k, r in rows.items() if k != "f32"}
    if not args.no_cpu:
        # CPU-baseline leg: the FP64 oracle solves the same MDP exactly (policy iteration, dense LU per
        # policy, Bellman passes over the rows streamed from the device); T J = J certifies J = J*
        from oracle import exact
        Pr = P.reshape(n * m, n)
        t0 = time.perf_counter()
        cert = exact.dense_policy_iteration(lambda r0, r1: Pr[r0:r1].cpu().numpy(),
                                            lambda idx: Pr[torch.from_numpy(np.asarray(idx)).cuda()].cpu().numpy(),
                                            cost.cpu().numpy(), 0.999, n, m, chunk_states=256)
        ct = time.perf_counter() - t0
        J = cert["J"]
        sc = float(np.abs(J).max())
        for name, key in (("f32", "f32"), ("bf16", "bf16+f32 refinement"), ("fp8", "fp8+f32 refinement")):
            rows[key]["rel_err_vs_certified_optimum"] = float(np.abs(vals[name] - J).max()) / sc
        e["certificate"] = {"policy_iterations": cert["iters"], "bellman_residual": cert["resid"],
                            "error_bound": cert["resid"] / (1 - 0.999)}
        import oracle
        e["cpu_baseline"] = {"value": ct * 1e3, "unit": "ms (exact FP64 solve)", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"policy iteration, {cert['iters']} dense LU solves at n=16384"}
    out["dense16k"] = e
    del d32, P, cost, ws, V
    torch.cuda.empty_cache()

    # differentiable fixed point n=65536: forward MB-VI + adjoint gradient (b = 16384)
    mdp = mdpgen.config5()
    dm = rmb.DeviceMDP.from_host(mdp)
    z = torch.from_numpy(mdp.logits).cuda()
    w = torch.from_numpy(mdpgen.random_values(mdp.n, seed=13)).cuda()
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    fo = rmb.Opts(batch=16384, seed=mdpgen.PERM_SEED, eps=1e-7, max_sweeps=100000, validate=False)
    go = rmb.Opts(batch=16384, seed=5, eps=1e-7, max_sweeps=100000, validate=False)
    fws = rmb.workspace(dm, fo)

    def s5():
        rmb.rmb_softmax_rows(dm, z, dm.prob)
        V.zero_()
        a = rmb.rmb_vi(dm, fo, V, pi, None, ws=fws, stream=stream)
        g = rmb.rmb_fixed_point_grad(dm, pi, V, w, go)
        return a, g[3]

    for _ in range(3):
        s5()
    ms, (a, g) = _ev_ms(s5, stream, reps=5)
    nk = mdp.n * mdp.uniform_k()
    byt = (a["sweeps"] + 1) * (mdp.nnz * 8 + mdp.n * mdp.m * 4) + g["sweeps"] * (nk * 8 + mdp.n * 8) + nk * 8
    ach = byt / ((a["ms"] + g["ms"]) / 1e3) / 1e9
    out["adjoint65536"] = {
        "workload": "csr n=65536 m=8 k=16 P=softmax(N(0,1) logits) gamma=0.95: forward MB-VI b=16384 to 1e-7 + "
                    "adjoint sweeps b=16384 to 1e-7, dL/dcost and dL/dlogits of w.V*",
        "ms_per_gradient": ms, "forward_sweeps": a["sweeps"], "adjoint_sweeps": g["sweeps"],
        "roofline": {"bound": "latency", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "peak_kind": peak_kind,
                     "note": "P (67 MB) fits in L2; 4 batches per sweep, each a grid barrier plus dependent loads"}}
    return out


# ------------------------------------------------------------------------------------------------
# The other workloads (one JSON line each; not the headline line).
# ------------------------------------------------------------------------------------------------
def _line(metric, value, unit, ms, args, world, config, **kw):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
         "data": "synthetic", "config": config}
    d.update(kw)
    return d


def _timed(fn, steps, stream):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, outs


def run_workload(args, world, rank, local):
    import torch
    import paper_2110_02901_b300 as rmb
    from paper_2110_02901_b300 import build as rbuild
    rbuild.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    l0 = rmb.rmb_kernel_launches()
    with ClockSampler(local) as clk:
        line = {"dense500": _dense500, "dense16k": _dense16k, "batched": _batched, "adjoint": _adjoint,
                "maze": _maze, "select": _select}[
            args.workload](args, world, rmb, torch, stream, hbm, peak_kind)
    line["clocks"] = clk.summary()
    line["gpu_launches_total"] = rmb.rmb_kernel_launches() - l0
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _dense500(args, world, rmb, torch, stream, hbm, peak_kind):
    """Dense n=500, m=4, Dirichlet(1), gamma=0.95, b=50: MB-VI to 1e-6 (latency-bound: P is 4 MB)."""
    mdp = mdpgen.config1()
    dm = rmb.DeviceMDP.from_host(mdp)
    o = rmb.Opts(batch=50, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=100000, validate=False)
    ws = rmb.workspace(dm, o)
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")

    def step():
        V.zero_()
        return rmb.rmb_vi(dm, o, V, pi, None, ws=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    ms, outs = _timed(step, args.steps, stream)
    sw = outs[-1]["sweeps"]
    path = outs[-1]["path"]
    err, cpu = None, None
    if not args.no_cpu:   # CPU-baseline leg: the FP64 oracle's full solve, timed, and the GPU error against it
        import oracle
        t0 = time.perf_counter()
        ref = oracle.mbvi(mdp, 50, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=100000)
        ct = time.perf_counter() - t0
        err = float(np.abs(V.cpu().numpy() - ref["V"]).max())
        cpu = {"value": mdp.n * ref["sweeps"] / ct, "unit": "Bellman backups/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"full solve, {ref['sweeps']} sweeps, {ct:.2f} s"}
    bytes_launch = (sw + 1) * mdp.n * mdp.m * mdp.n * 4
    ach = bytes_launch / (outs[-1]["ms"] / 1e3) / 1e9
    return _line(METRIC, mdp.n * sw / (ms / 1e3), "Bellman backups/s", ms, args, world,
                 {"workload": "dense-mdp n=500 m=4 dirichlet(1) c~U[0,1] gamma=0.95; MB-VI b=50 from V=0 to 1e-6",
                  "sweeps": sw, "barriers_per_solve": outs[-1]["barriers"], "time_to_eps_ms": ms, "path": path,
                  "max_abs_err_vs_oracle": err, "l2": "P is 4 MB: L2-resident by design (latency-bound workload)"},
                 roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "peak_kind": peak_kind,
                           "kernel": "rmb_small_kernel" if path == "cluster" else "rmb_dense_kernel<f32>",
                           "note": "P is L2-resident; the bound is the per-batch barrier latency (10 batches/sweep)"},
                 cpu_baseline=cpu)


def _dense16k(args, world, rmb, torch, stream, hbm, peak_kind):
    """Dense n=16384, m=16, Dirichlet(0.1), c~N(0,1), gamma=0.999: sweep throughput per storage type and
    b; converged error per storage type on the same recipe at n=2048 against the exact optimum."""
    if args.profile_case:
        # profiling mode: one solve of exactly profile_case sweeps at n = 2^n_log2 (default 2^20 is
        # reduced to 2^12 here), b = n/4, storage --storage
        n = 1 << (args.n_log2 if args.n_log2 != 20 else 12)
        P, cost = mdpgen.dense_dirichlet_device(n, 16, 0.1, 0.999, seed=3)
        dm = rmb.DeviceMDP(n, 16, 0.999, "dense", cost, P=P.reshape(-1))
        if args.storage != "f32":
            dm = rmb.dense_lowp(dm, rmb.RMB_P_BF16 if args.storage == "bf16" else rmb.RMB_P_FP8E4M3)
        V = torch.zeros(n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, rmb.Opts(batch=n // 4, eps=0.0, max_sweeps=args.profile_case, validate=False), V)
        eb = {"f32": 4, "bf16": 2, "fp8": 1}[args.storage]
        gb = st["sweeps"] * n * 16 * n * eb / 1e9
        return {"profile_case": True, "n": n, "storage": args.storage, "sweeps": st["sweeps"], "ms": st["ms"],
                "gbs": gb / (st["ms"] / 1e3)}
    n, m = 16384, 16
    P, cost = mdpgen.dense_dirichlet_device(n, m, 0.1, 0.999, seed=3)
    d32 = rmb.DeviceMDP(n, m, 0.999, "dense", cost, P=P.reshape(-1), name="dense16k")
    forms = {"f32": d32, "bf16": rmb.dense_lowp(d32, rmb.RMB_P_BF16), "fp8": rmb.dense_lowp(d32, rmb.RMB_P_FP8E4M3)}
    ebytes = {"f32": 4, "bf16": 2, "fp8": 1}
    thr = []
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    for name, dm in forms.items():
        for b in (256, 4096):
            o = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=20, validate=False)
            ws = rmb.workspace(dm, o)
            st = None
            for _ in range(2):
                V.zero_()
                st = rmb.rmb_vi(dm, o, V, None, None, ws=ws, stream=stream)
            per = st["ms"] / st["sweeps"]
            gb = n * m * n * ebytes[name] / 1e9
            thr.append({"storage": name, "b": b, "ms_per_sweep": per, "p_stream_gbs": gb / (per / 1e3),
                        "hbm_frac": gb / (per / 1e3) / hbm, "backups_per_s": n / (per / 1e3)})
    full = {}
    if args.full:
        for name in ("f32", "fp8", "bf16"):
            o = rmb.Opts(batch=4096, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
            V.zero_()
            if name == "f32":
                st = rmb.rmb_vi(forms["f32"], o, V, stream=stream)
                full[name] = {"time_to_eps_ms": st["ms"], "sweeps": st["sweeps"]}
            else:
                s1, s2 = rmb.rmb_vi_refined(forms[name], forms["f32"], o, EPS, V)
                full[name + "+f32 refinement"] = {"time_to_eps_ms": s1["ms"] + s2["ms"],
                                                  "sweeps": [s1["sweeps"], s2["sweeps"]]}
    del forms, d32, P
    torch.cuda.empty_cache()
    # CPU-baseline leg (skipped with --no-cpu): the FP64 exact optimum of the same recipe at n = 2048
    # (policy iteration), and the error of each storage type's converged GPU solve against it
    errs = {}
    if not args.no_cpu:
        from oracle import exact
        sm = mdpgen.dense_dirichlet(2048, 16, alpha=0.1, gamma=0.999, seed=3, cost_dist="normal")
        jstar, _, _ = exact.policy_iteration(sm)
        dm = rmb.DeviceMDP.from_host(sm)
        for name, form in (("f32", dm), ("bf16", rmb.dense_lowp(dm, rmb.RMB_P_BF16)),
                           ("fp8", rmb.dense_lowp(dm, rmb.RMB_P_FP8E4M3))):
            o = rmb.Opts(batch=256, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=400000, validate=False)
            V2 = torch.zeros(2048, dtype=torch.float32, device="cuda")
            st = rmb.rmb_vi(form, o, V2, stream=stream)
            e = float(np.abs(V2.cpu().numpy() - jstar).max() / np.abs(jstar).max())
            rec = {"sweeps": st["sweeps"], "ms": st["ms"], "rel_err_vs_exact": e}
            if name != "f32":
                V3 = torch.zeros(2048, dtype=torch.float32, device="cuda")
                s1, s2 = rmb.rmb_vi_refined(form, dm, o, EPS, V3)
                rec["refined_rel_err"] = float(np.abs(V3.cpu().numpy() - jstar).max() / np.abs(jstar).max())
                rec["refined_sweeps"] = [s1["sweeps"], s2["sweeps"]]
                rec["refined_ms"] = s1["ms"] + s2["ms"]
            errs[name] = rec
    best = max(thr, key=lambda r: r["p_stream_gbs"] if r["storage"] == "f32" else -1)
    # the FP64 oracle on the host cores: MB-VI sweeps of the same recipe at n = 2048 (the n = 16384 P
    # is 17 GB); its P-stream rate, converted to backups/s at n = 16384 (m * n * 4 bytes per backup)
    cpu = None
    if not args.no_cpu:
        import oracle
        small = mdpgen.dense_dirichlet(2048, m, alpha=0.1, gamma=0.999, seed=3, cost_dist="normal")
        Vc = np.zeros(small.n)
        t0 = time.perf_counter()
        csw = 0
        while csw < 200 and time.perf_counter() - t0 < 10.0:
            Vc = oracle.mbvi(small, 4096, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=1, V0=Vc, start_sweep=csw)["V"]
            csw += 1
        ct = time.perf_counter() - t0
        cpu_gbs = csw * small.P.nbytes / ct / 1e9
        cpu = {"value": cpu_gbs * 1e9 / (m * n * 4), "unit": "Bellman backups/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"{csw} FP64 MB-VI sweeps of the same recipe at n=2048 ({ct:.1f} s, "
                                           f"{cpu_gbs:.2f} GB/s of P), converted to n=16384 by P bytes per backup"}
    return _line("dense sweep throughput per P storage type (and converged error vs the exact optimum)",
                 best["backups_per_s"], "Bellman backups/s", best["ms_per_sweep"], args, world,
                 {"workload": "dense-mdp n=16384 m=16 dirichlet(0.1) c~N(0,1) gamma=0.999; 20 MB-VI sweeps "
                              "per (storage, b); errors: same recipe at n=2048 solved to 1e-6",
                  "p_gb_per_sweep_f32": n * m * n * 4 / 1e9},
                 roofline={"bound": "hbm", "achieved": best["p_stream_gbs"], "peak": hbm, "unit": "GB/s",
                           "frac": best["p_stream_gbs"] / hbm,
                           # 20 sweeps of P per launch x DRAM bytes per P byte of one ncu capture of this
                           # kernel (n = 4096, 4 sweeps: 4.2922 GB for 4.2950 GB of P)
                           "traffic": 20 * n * m * n * 4 * DENSE_DRAM_BYTES_PER_P_BYTE,
                           "traffic_note": "ncu capture at n=4096 scaled by P bytes",
                           "kernel": "rmb_dense_tma_kernel<f32>", "peak_kind": peak_kind},
                 cpu_baseline=cpu, throughput=thr, full_solves=full, converged_errors_n2048=errs)


def _batched(args, world, rmb, torch, stream, hbm, peak_kind):
    """256 uneven CSR MDPs: one graph-captured persistent launch vs one rmb_vi launch per MDP."""
    mdps = mdpgen.config3()
    dms = [rmb.DeviceMDP.from_host(x) for x in mdps]
    tot_n = sum(x.n for x in mdps)
    Vall = torch.zeros(tot_n, dtype=torch.float32, device="cuda")
    Vs, off = [], 0
    for x in mdps:
        Vs.append(Vall[off:off + x.n])
        off += x.n
    if args.profile_case:
        # profiling mode: the same launch (same plan), every MDP capped at profile_case sweeps
        o = rmb.Opts(batch=1, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=args.profile_case, validate=False)
        s = torch.cuda.Stream()
        B = rmb.Batch(dms, Vs, o, stream=s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        B.run(s)
        e1.record(s)
        torch.cuda.synchronize()
        res = B.results(stream=s, check=False)
        return {"profile_case": True, "mdps": len(mdps), "ms": e0.elapsed_time(e1),
                "sweeps_total": sum(r["sweeps"] for r in res),
                "nnz_pass_bytes": sum((r["sweeps"] + 1) * x.nnz * 8 for x, r in zip(mdps, res))}
    o = rmb.Opts(batch=1, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
    s = torch.cuda.Stream()
    B = rmb.Batch(dms, Vs, o, stream=s)
    B.capture(s)

    def step():
        with torch.cuda.stream(s):
            Vall.zero_()
        B.replay(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    res = B.results(stream=s)
    backups = sum(x.n * r["sweeps"] for x, r in zip(mdps, res))
    nnz_passes = sum((r["sweeps"] + 1) * x.nnz * 8 for x, r in zip(mdps, res))
    # the plain form: one rmb_vi launch per MDP, same b, one after the other
    plan = B.plan_table()
    seq_ms = 0.0
    for x, dm, p in zip(mdps, dms, plan):
        oo = rmb.Opts(batch=p["batch"], seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000, validate=False)
        V = torch.zeros(x.n, dtype=torch.float32, device="cuda")
        st = rmb.rmb_vi(dm, oo, V)
        seq_ms += st["ms"]
    # CPU-baseline leg: the FP64 oracle on the host cores, whole solves of the MDPs in plan order until
    # ~15 s, and the sum over all MDPs extrapolated by their nnz x sweeps (the GPU's sweep counts)
    cpu = None
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        done_work = 0.0
        solved = 0
        for x, p_ in zip(mdps, plan):
            oracle.mbvi(x, p_["batch"], seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000)
            done_work += x.nnz * res[solved]["sweeps"]
            solved += 1
            if time.perf_counter() - t0 > 15.0:
                break
        ct = time.perf_counter() - t0
        all_work = sum(x.nnz * r["sweeps"] for x, r in zip(mdps, res))
        cpu_total_s = ct * all_work / done_work
        cpu = {"value": backups / cpu_total_s, "unit": "Bellman backups/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"{solved} of {len(mdps)} MDPs solved to 1e-6 in FP64 ({ct:.1f} s); "
                                           f"all 256 extrapolated by nnz x sweeps: {cpu_total_s:.0f} s"}
    return _line("batched time-to-1e-6 (all 256 MDPs) and Bellman backups/s", backups / (ms / 1e3),
                 "Bellman backups/s", ms, args, world,
                 {"workload": "256 csr-mdps n~logU[256,65536] m~U{2..16} k=16 dirichlet(1) c~U[0,1] "
                              "gamma~U[0.9,0.99]; MB-VI to 1e-6, autotuned b, one graph-captured launch",
                  "mdps": len(mdps), "total_states": tot_n, "total_nnz": sum(x.nnz for x in mdps),
                  "time_to_eps_ms": ms, "plan_makespan_est_ms": B.handle.est_ms,
                  "sequential_single_mdp_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms,
                  "groups": sorted({p["group_ctas"] for p in plan}),
                  "max_sweeps": max(r["sweeps"] for r in res)},
                 roofline={"bound": "hbm", "achieved": nnz_passes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": nnz_passes / (ms / 1e3) / 1e9 / hbm,
                           "traffic": BATCHED_DRAM_PER_ALGO_BYTE * nnz_passes,
                           "traffic_note": "ncu DRAM bytes / algorithmic bytes of the same launch capped at 20 "
                                           "sweeps per MDP (1.011), times this run's algorithmic bytes",
                           "kernel": "rmb_batched_kernel", "peak_kind": peak_kind},
                 cpu_baseline=cpu)


def _adjoint(args, world, rmb, torch, stream, hbm, peak_kind):
    """n=65536, m=8, k=16 softmax MDP: forward MB-VI (gamma=0.95) and the adjoint gradient of w.V*."""
    mdp = mdpgen.config5()
    dm = rmb.DeviceMDP.from_host(mdp)
    z = torch.from_numpy(mdp.logits).cuda()
    w = torch.from_numpy(mdpgen.random_values(mdp.n, seed=13)).cuda()
    V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    pi = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    # b = 16384: at n = 65536 the solves are latency-bound, and 4 batches per sweep beat 16 (b = 4096:
    # 38 ms per gradient, b = 16384: 24 ms, b = 65536: 24 ms)
    fo = rmb.Opts(batch=16384, seed=mdpgen.PERM_SEED, eps=1e-7, max_sweeps=100000, validate=False)
    go = rmb.Opts(batch=16384, seed=5, eps=1e-7, max_sweeps=100000)
    fws = rmb.workspace(dm, fo)

    def step():
        rmb.rmb_softmax_rows(dm, z, dm.prob)
        V.zero_()
        st1 = rmb.rmb_vi(dm, fo, V, pi, None, ws=fws, stream=stream)
        lam, gc, gz, st2 = rmb.rmb_fixed_point_grad(dm, pi, V, w, go)
        return st1, st2

    for _ in range(args.warmup):
        step()
    ms, outs = _timed(step, args.steps, stream)
    st1, st2 = outs[-1]
    nk = mdp.n * mdp.uniform_k()
    fwd_bytes = (st1["sweeps"] + 1) * (mdp.nnz * 8 + mdp.n * mdp.m * 4)
    adj_bytes = st2["sweeps"] * (nk * 8 + mdp.n * 8) + nk * 8
    ach = (fwd_bytes + adj_bytes) / ((st1["ms"] + st2["ms"]) / 1e3) / 1e9
    cpu = None
    if not args.no_cpu:   # CPU-baseline leg: the FP64 direct-solve gradient on the host
        from oracle import exact
        t0 = time.perf_counter()
        exact.fixed_point_gradient(mdp, w.cpu().numpy().astype(np.float64))
        ct = time.perf_counter() - t0
        cpu = {"value": 1.0 / ct, "unit": "gradients/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"direct-solve gradient (policy iteration + GMRES adjoint), {ct:.1f} s"}
    return _line("time of forward solve + adjoint gradient (w.V*, dcost and dlogits)", 1e3 / ms, "gradients/s", ms,
                 args, world,
                 {"workload": "csr-mdp n=65536 m=8 k=16 P=softmax(N(0,1) logits) c~U[0,1] gamma=0.95; forward MB-VI "
                              "b=16384 to 1e-7, adjoint mini-batch sweeps b=16384 to 1e-7",
                  "forward_ms": st1["ms"], "forward_sweeps": st1["sweeps"], "adjoint_ms": st2["ms"],
                  "adjoint_sweeps": st2["sweeps"]},
                 roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "kernel": "rmb_csr_vec_kernel (forward) + rmb_csr_gen_kernel (adjoint)",
                           "peak_kind": peak_kind,
                           "note": "algorithmic bytes: forward (sweeps + 1) x (nnz x 8 + n m 4), adjoint sweeps x "
                                   "(n k 8 + n 8), gradient pass n k 8, over the two solves' device time; P (67 MB) "
                                   "fits in the 126 MB L2 and each batch costs barrier and dependent-load latency, so "
                                   "the solves are latency-bound"},
                 cpu_baseline=cpu)


# speed-ups at 1e-4 of J* printed in Sec. IV-B (GTX 1650 Ti): context, not targets
PAPER_MAZE = {"maze80": {"vi": {512: {"over_VI": 1.41, "over_GS": 89.28}}},
              "maze100": {"vi": {512: {"over_VI": 3.04, "over_GS": 58.86}, 4853: {"over_VI": 2.57, "over_GS": 49.73}},
                          "mpi": {512: {"over_MPI": 1.31, "over_GS": 194.52}}}}


def _maze(args, world, rmb, torch, stream, hbm, peak_kind):
    """2D-maze stand-ins (N = 80: 6166 states, N = 100: 9706 states, 4 actions, gamma 0.95, V0 = 0):
    time for MB-VI (and MB-MPI, K = 50) to reach ||V - J*||_inf <= 1e-4 for each batch size, the
    measure of Sec. IV-B.  J* comes from a GPU MB-MPI solve to ||TV - V||_inf <= 1e-7 (error below
    1.9e-6 by the contraction bound).  The sweep count k*(b) is found by stepping one sweep (MPI: one
    improvement round) at a time; the timed run is a fresh solve from 0 capped at k*(b)."""
    if args.profile_case:
        # profiling mode: one MB-VI solve of exactly profile_case sweeps on the N = 100 maze at
        # b = --profile-batch (default 512)
        mdp = mdpgen.maze100()
        dm = rmb.DeviceMDP.from_host(mdp)
        V = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
        pb = args.profile_batch
        b = mdp.n if pb in ("n", "async") else int(pb)
        st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=args.profile_case,
                                     validate=False, flags=rmb.RMB_FLAG_ASYNC if pb == "async" else 0), V)
        return {"profile_case": True, "n": mdp.n, "b": pb, "sweeps": st["sweeps"], "ms": st["ms"],
                "barriers": st["barriers"], "us_per_batch": 1e3 * st["ms"] / st["barriers"], "path": st["path"]}
    TOL = 1e-4
    K = 50
    rows, lines = [], {}
    for mk in (mdpgen.maze80, mdpgen.maze100):
        mdp = mk()
        dm = rmb.DeviceMDP.from_host(mdp)
        n = mdp.n
        J = torch.zeros(n, dtype=torch.float32, device="cuda")
        pi = torch.empty(n, dtype=torch.int32, device="cuda")
        st = rmb.rmb_mpi(dm, rmb.Opts(batch=n, seed=1, eps=1e-7, max_sweeps=100000, eval_sweeps=K), J, pi)
        cert = st["residual"] * mdp.gamma / (1 - mdp.gamma)
        V = torch.zeros(n, dtype=torch.float32, device="cuda")

        def err():
            return float((V - J).abs().max())

        def solve(scheme, b, cap, flags=0, resume=None):
            o = rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=cap, eval_sweeps=K, validate=False,
                         flags=flags, start_sweep=0 if resume is None else resume)
            if scheme == "vi":
                return rmb.rmb_vi(dm, o, V, stream=stream)
            return rmb.rmb_mpi(dm, o, V, pi, stream=stream)

        cases = [("vi", b, 0) for b in (1, 32, 128, 512, 2048, n // 2, n)] + [("vi", n, rmb.RMB_FLAG_ASYNC)]
        if mdp.name == "maze100":
            cases += [("mpi", b, 0) for b in (1, 512, n)]
        res = {}
        for scheme, b, flags in cases:
            # k*: sweeps (MPI: improvement rounds) until the error is within TOL
            V.zero_()
            k = 0
            while err() > TOL and k < 20000:
                if scheme == "vi":
                    solve("vi", b, 1, flags, resume=k)
                else:
                    solve("mpi", b, 2, flags, resume=k * K)
                k += 1
            cap = k if scheme == "vi" else k + 1
            ts = []
            for _ in range(max(3, args.steps)):
                V.zero_()
                ts.append(solve(scheme, b, cap, flags)["ms"])
            e = err()
            label = "async" if flags else b
            res[(scheme, label)] = min(ts)
            rows.append({"mdp": mdp.name, "n": n, "scheme": scheme, "b": label, "sweeps" if scheme == "vi" else
                         "improvements": k, "ms": round(min(ts), 4), "err": e})
        for r in rows:
            if r["mdp"] != mdp.name:
                continue
            full = res[(r["scheme"], n)]
            gs = res[(r["scheme"], 1)]
            r["speedup_over_b_n"] = round(full / r["ms"], 3)
            r["speedup_over_b_1"] = round(gs / r["ms"], 3)
        lines[mdp.name] = {"J*_certified_err": cert, "J*_mpi_ms": st["ms"]}
    # CPU-baseline leg: the FP64 oracle's MB-VI on the N = 100 maze at b = 512 for the same sweep count
    m100 = mdpgen.maze100()
    k512 = next(r["sweeps"] for r in rows if r["mdp"] == "maze100" and r["scheme"] == "vi" and r["b"] == 512)
    cpu = None
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        oracle.mbvi(m100, 512, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=k512)
        ct = time.perf_counter() - t0
        cpu = {"value": 1.0 / ct, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"N=100 maze, b=512, {k512} sweeps, {ct:.2f} s"}
    best = next(r for r in rows if r["mdp"] == "maze100" and r["scheme"] == "vi" and r["b"] == 512)
    pbytes = m100.prob.nbytes + m100.col.nbytes + m100.row_ptr.nbytes + m100.cost.nbytes
    ach = best["sweeps"] * pbytes / (best["ms"] / 1e3) / 1e9
    return _line("2D-maze MB-VI time to ||V - J*||_inf <= 1e-4 (N=100, b=512)", 1e3 / best["ms"], "solves/s",
                 best["ms"], args, world,
                 {"workload": "2D-maze stand-ins N=80 (6166 states) and N=100 (9706 states), 4 actions, slip 0.2, "
                              "unit cost, absorbing goal, gamma=0.95, V0=0; MB-VI for b in {1,32,128,512,2048,n/2,n} "
                              "and asynchronous sweeps; MB-MPI K=50 for b in {1,512,n} (N=100)",
                  "table": rows, "reference_solutions": lines, "paper_speedups_gtx1650ti": PAPER_MAZE,
                  "l2": "P is < 3 MB: L2-resident (latency-bound workload)"},
                 roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "kernel": "rmb_small_kernel (b <= 512) / rmb_csr_gen_kernel", "peak_kind": peak_kind,
                           "note": "latency-bound: P (2.6 MB) is L2-resident; a batch costs a barrier plus a "
                                   "few dependent L2 round trips, so HBM is not the bound"},
                 cpu_baseline=cpu)


def _select(args, world, rmb, torch, stream, hbm, peak_kind):
    """Batch selection (the Sec. V extension): sigma (the paper's order) against uniform draws with
    replacement and draws by residual weights (refreshed every few sweeps).
    (1) CSR n = 2^20, m = 8, k = 32, gamma = 0.99, from V = 0 to 1e-6: time, sweeps and the full
        residual ||TV - V||_inf at the end (draws stop on it; sigma stops on the sweep change);
    (2) warm start on the N = 100 maze after the costs of a 10 x 10 block of cells rise from 1 to 3:
        time from the old J* to ||V - J*_new||_inf <= 1e-4 (k* found by stepping, as for the maze workload)."""
    rows = []
    mdp = mdpgen.config2()
    dm = rmb.DeviceMDP.from_host(mdp)
    n = mdp.n
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    TV = torch.empty_like(V)
    gws = rmb.workspace(dm, rmb.Opts(batch=n))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for b in (16384, 262144):
        for label in ("sigma", "uniform", "prioritized"):
            ts, st = [], None
            for _ in range(2):
                V.zero_()
                torch.cuda.synchronize()
                ev0.record(stream)
                if label == "prioritized":
                    st = rmb.prioritized_vi(dm, V, batch=b, eps=EPS, refresh=16, floor_frac=0.05, stream=stream)
                else:
                    st = rmb.rmb_vi(dm, rmb.Opts(batch=b, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000,
                                                 validate=False, select=0 if label == "sigma" else 1), V, stream=stream)
                ev1.record(stream)
                torch.cuda.synchronize()
                ts.append(ev0.elapsed_time(ev1))
            full = rmb.rmb_greedy(dm, V, TV, ws=gws)["residual"]
            rows.append({"mdp": "csr2e20", "b": b, "selection": label, "ms": round(min(ts), 2), "sweeps": st["sweeps"],
                         "ms_per_sweep": round(min(ts) / st["sweeps"], 4), "full_residual": full,
                         "status": st["status"]})
    # (2) maze warm start
    old = mdpgen.maze100()
    new = mdpgen.maze100()
    cells = new.meta["cells"]
    block = np.flatnonzero((cells[:, 0] >= 45) & (cells[:, 0] < 55) & (cells[:, 1] >= 45) & (cells[:, 1] < 55))
    block = block[block != new.meta["goal"]]
    cost = new.cost.reshape(new.n, 4).copy()
    cost[block] = 3.0
    new.cost = cost.reshape(-1).astype(np.float32)
    dold, dnew = rmb.DeviceMDP.from_host(old), rmb.DeviceMDP.from_host(new)
    n = new.n
    J0 = torch.zeros(n, dtype=torch.float32, device="cuda")
    pi = torch.empty(n, dtype=torch.int32, device="cuda")
    rmb.rmb_mpi(dold, rmb.Opts(batch=n, eps=1e-7, max_sweeps=100000, eval_sweeps=50), J0, pi)
    J1 = J0.clone()
    rmb.rmb_mpi(dnew, rmb.Opts(batch=n, eps=1e-7, max_sweeps=100000, eval_sweeps=50), J1, pi)
    V = torch.empty_like(J0)
    TOL = 1e-4

    def err():
        return float((V - J1).abs().max())

    init_err = float((J0 - J1).abs().max())
    for label, b, refresh in (("sigma", n, 0), ("sigma", 512, 0), ("uniform", 512, 0), ("prioritized", 512, 1),
                              ("prioritized", 512, 4), ("prioritized", 2048, 4)):
        def run(cap):
            if label == "prioritized":
                done = 0
                while done < cap:
                    w = rmb.rmb_residual_weights(dnew, V, 0.05, stream=stream)
                    k = min(refresh, cap - done)
                    rmb.rmb_vi(dnew, rmb.Opts(batch=b, seed=7, eps=0.0, max_sweeps=k, start_sweep=done, validate=False,
                                              select=2, weights=w), V, stream=stream, stats=False)
                    done += k
            else:
                rmb.rmb_vi(dnew, rmb.Opts(batch=b, seed=7, eps=0.0, max_sweeps=cap, validate=False,
                                          select=0 if label == "sigma" else 1), V, stream=stream, stats=False)
        # k*: smallest sweep count reaching TOL (doubling, then bisection; each trial from the old J*)
        lo, hi = 0, 1
        while True:
            V.copy_(J0)
            run(hi)
            torch.cuda.synchronize()
            if err() <= TOL or hi > 4096:
                break
            lo, hi = hi, hi * 2
        while hi - lo > 1:
            mid = (lo + hi) // 2
            V.copy_(J0)
            run(mid)
            torch.cuda.synchronize()
            lo, hi = (lo, mid) if err() <= TOL else (mid, hi)
        ts = []
        for _ in range(3):
            V.copy_(J0)
            torch.cuda.synchronize()
            ev0.record(stream)
            run(hi)
            ev1.record(stream)
            torch.cuda.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        rows.append({"mdp": "maze100 warm start", "b": b, "selection": label + (f" refresh={refresh}" if refresh else ""),
                     "ms": round(min(ts), 3), "sweeps": hi, "err": err()})
    best = next(r for r in rows if r["mdp"] == "csr2e20" and r["b"] == 262144 and r["selection"] == "uniform")
    # CPU-baseline leg: the FP64 oracle on the host cores, uniform-draw sweeps of the same MDP (bounded)
    cpu = None
    if not args.no_cpu:
        import oracle
        Vc = np.zeros(mdp.n)
        t0 = time.perf_counter()
        csw = 0
        while csw < 50 and time.perf_counter() - t0 < 10.0:
            Vc = oracle.mbvi(mdp, 262144, seed=mdpgen.PERM_SEED, eps=0.0, max_sweeps=1, V0=Vc, start_sweep=csw,
                             select=1)["V"]
            csw += 1
        ct = time.perf_counter() - t0
        cpu = {"value": mdp.n * csw / ct, "unit": "Bellman backups/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"{csw} uniform-draw MB-VI sweeps (b=262144) of the n=2^20 MDP "
                                           f"from V=0, FP64, {ct:.1f} s"}
    ach = best["sweeps"] * sweep_bytes(mdp.n, M_ACTIONS, K_SUCC) / (best["ms"] / 1e3) / 1e9
    return _line("batch selection with replacement: CSR n=2^20 MB-VI to 1e-6 with uniform draws (b=262144)",
                 mdp.n * best["sweeps"] / (best["ms"] / 1e3), "Bellman backups/s", best["ms"], args, world,
                 {"workload": "csr-mdp n=2^20 m=8 k=32 gamma=0.99 (sigma / uniform draws / residual-weighted draws, "
                              "b in {16384, 262144}); maze N=100 warm start after a 10x10 cost block rises 1 -> 3",
                  "table": rows, "maze_initial_err": init_err, "maze_block_states": int(len(block))},
                 roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "kernel": "rmb_csr_vec_kernel (draws)", "peak_kind": peak_kind,
                           "note": "P stream per sweep x sweeps / solve time; bound by random successor gathers "
                                   "as the sigma solve"},
                 cpu_baseline=cpu)


if __name__ == "__main__":
    sys.exit(main())

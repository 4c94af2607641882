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
    ap.add_argument("--ref-sweeps", type=int, default=3, help="reference arm: oracle sweeps per step")
    ap.add_argument("--n-log2", type=int, default=20, help="states = 2^n_log2 (profiling of smaller cases)")
    ap.add_argument("--profile-case", type=int, default=0, metavar="SWEEPS",
                    help="profiling mode: one MB-VI solve of exactly SWEEPS sweeps (no bench line)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

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
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": "rmb_csr_vec_kernel", "peak_kind": peak_kind,
                "bytes_per_launch": statistics.mean(per_launch_bytes),
                "note": "P stream (prob+col+cost) per sweep x (sweeps + 1 greedy pass) / launch time"}

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
        for bb in B_SWEEP:
            bb = min(bb, n)
            for scheme in ("vi", "mpi"):
                o = rmb.Opts(batch=bb, seed=mdpgen.PERM_SEED, eps=EPS, max_sweeps=200000 if scheme == "vi" else 20000,
                             eval_sweeps=MPI_K, validate=False)
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
                bsweep.append({"b": bb, "scheme": scheme, "time_to_eps_ms": res["ms"], "sweeps": res["sweeps"],
                               "improvements": res["iters"], "backups_per_s": n * res["sweeps"] / (res["ms"] / 1e3),
                               "p_stream_gbs": gbs, "hbm_frac": gbs / hbm, "residual": res["residual"],
                               "barriers": res["barriers"]})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(mdp, b)

    total_launches = rmb.rmb_kernel_launches() - launches0
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Bellman backups/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(b), "n": n, "m": M_ACTIONS, "k": K_SUCC, "gamma": GAMMA,
                       "batch": b, "eps": EPS, "sweeps_per_step": sweeps / args.steps,
                       "time_to_eps_ms": ms_max / args.steps, "parallelism": f"replicas x{world}",
                       "l2": "inputs (2.2 GB of P per sweep) exceed the 126 MB L2; no flush needed",
                       "validate": "once before timing", "path": stats[-1]["path"],
                       "grid_ctas": stats[-1]["grid_ctas"]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "b_sweep": bsweep, "kernel_launches_total": total_launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

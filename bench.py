#!/usr/bin/env python3
"""Benchmark: Metropolis moves per second of the batched treecode Monte Carlo.

Workload (default): 256 independent replicas of the colloid double layer
(macroion R = 10, Z = -60; N ions per replica uniform in [2000, 50000]; a point
image per ion, so 2N+1 charges per tree), theta = 0.5, p = 4.  One step = one
persistent, CUDA-graph-replayed launch doing `--moves` trial moves on every
replica (propose, reject tests, treecode dE at the old and new positions of the
ion and its image, Metropolis, local octree adjustment, running energy).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the reference arm), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC moves/sec at N=1e4..1e6 (batched vs plain, 1 GB300); dE rel err vs FP64 oracle"
UNIT = "moves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--reps", type=int, default=256)
    ap.add_argument("--moves", type=int, default=2000, help="trial moves per replica per step")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--C", type=int, default=16, help="leaf capacity (autotuned: profiles/autotune_colloid64.md)")
    ap.add_argument("--warps", type=int, default=8)
    ap.add_argument("--layout", default="aos", choices=["soa", "aos"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def traffic_record():
    """DRAM bytes per trial move of the batched kernel from the committed ncu
    capture, if the kernel sources are unchanged since that capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_batch_traffic.json")))
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_1305_1825_gb300", "csrc", f), "rb").read())
        if h.hexdigest() == rec["sources_sha256"]:
            return rec
    except Exception:
        pass
    return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "of measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(args, rank=0):
    from paper_1305_1825_gb300 import workloads as W
    sizes = W.batch_sizes(args.reps, seed=3)
    systems = W.batch(sizes=sizes, theta=args.theta, p=args.p, C=args.C)
    seeds = [1000 + r + 100000 * rank for r in range(args.reps)]
    return sizes, systems, seeds


def config(args, sizes, extra=None):
    c = {"workload": "colloid-%d-replicas" % args.reps, "replicas": args.reps,
         "N_range": [min(sizes), max(sizes)], "charges_per_replica": "2N+1 (ions, images, macroion)",
         "moves_per_replica_per_step": args.moves, "theta": args.theta, "p": args.p, "C": args.C,
         "warps_per_move": args.warps, "layout": args.layout, "step": 1.0,
         "l2": "inputs larger than L2: the replicas' trees total several GB"}
    if extra:
        c.update(extra)
    return c


def oracle_sample(systems, seeds, moves, budget_s):
    """Run the FP64 oracle chain on replicas until ~budget_s of CPU time; moves/s."""
    import oracle
    done, t_total, used = 0, 0.0, 0
    for r, wl in enumerate(systems):
        ref = oracle.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
        t = time.perf_counter()
        ref.mc_run(seeds[r], moves, replica=r)
        t_total += time.perf_counter() - t
        done += moves
        used += 1
        if t_total >= budget_s:
            break
    return done / t_total, "%d replicas x %d moves (FP64 oracle treecode chain, single thread)" % (used, moves)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    sizes, systems, seeds = workload(args)
    vals = []
    sample = ""
    for s in range(args.warmup + args.steps):
        v, sample = oracle_sample(systems, seeds, 400, 3.0)
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(args, sizes),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def algorithmic_bytes_per_move(bh, batch, systems, K, acc_rate, n_sample_reps=8, n_moves=24):
    """Average algorithmic bytes of one trial move from the interaction-list
    counters (equal to the oracle's): 32 B per visited (cluster, point) header,
    4K B of FP32 moments per multipole evaluation, 32 B per direct pair, and on
    acceptance (20K + 32) B per cluster on the four ancestor paths."""
    import numpy as np
    rng = np.random.default_rng(0)
    V = A = Pp = 0
    n = 0
    depth_sum, depth_n = 0.0, 0
    reps = np.linspace(0, len(systems) - 1, n_sample_reps).astype(int)
    for r in reps:
        ctx = batch.replica(int(r))
        q, x = ctx.charges()
        wl = systems[r]
        for _ in range(n_moves):
            i = int(rng.integers(0, wl["n_mobile"]))
            rc, dE, cnt = ctx.delta_energy(i, x[i] + rng.uniform(-0.5, 0.5, 3))
            if rc:
                continue
            V += cnt.visited
            A += cnt.accepted
            Pp += cnt.pairs
            n += 1
        tree = ctx.export_tree()
        for (d, k), (leaf, cnt_, mem) in tree.items():
            if leaf and cnt_:
                depth_sum += d * cnt_
                depth_n += cnt_
    V, A, Pp = V / n, A / n, Pp / n
    depth = depth_sum / max(depth_n, 1)
    commit = acc_rate * 4 * (depth + 1) * (20 * K + 32)
    b = 32 * V + 4 * K * A + 32 * Pp + commit
    flops = A * (10 * K) + Pp * 14
    return b, {"visited": V, "multipole": A, "direct_pairs": Pp, "leaf_depth": depth,
               "commit_bytes": commit, "fp32_flops": flops}


def plain_rate(bh, wl, warps, moves=400):
    import torch
    ctx = bh.Context(wl, warps=warps)
    ctx.step_mc(50, 1.0, seed=2, move0=0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.step_mc(moves, 1.0, seed=2, move0=50)
    torch.cuda.synchronize()
    r = moves / (time.perf_counter() - t)
    ctx.close()
    return r


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1825_gb300 import bhmc
    from paper_1305_1825_gb300 import workloads as W

    sizes, systems, seeds = workload(args, rank)
    layout = bhmc.LAYOUT_AOS if args.layout == "aos" else bhmc.LAYOUT_SOA
    stream = torch.cuda.current_stream()
    batch = bhmc.Batch(systems, warps=args.warps, layout=layout)
    K = (args.p + 1) * (args.p + 2) * (args.p + 3) // 6
    move0 = 0
    stats = None
    for _ in range(args.warmup):
        stats = batch.step_mc(args.moves, 1.0, seeds, move0=move0)
        move0 += args.moves
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc = tot = 0
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            stats = batch.step_mc(args.moves, 1.0, seeds, move0=move0)
            move0 += args.moves
            acc += sum(s["accepted"] for s in stats)
            tot += sum(s["moves"] for s in stats)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    moves_total = args.reps * args.moves * args.steps * world
    value = moves_total / (ms / 1e3)
    acc_rate = acc / max(tot, 1)

    # end to end through the public call (host clock): seeds up, stats down, every step
    barrier()
    t = time.perf_counter()
    for _ in range(2):
        batch.step_mc(args.moves, 1.0, seeds, move0=move0)
        move0 += args.moves
    e2e_s = (time.perf_counter() - t) / 2
    e2e = {"value": args.reps * args.moves * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * args.reps + 32, "d2h_bytes_per_step": 64 * args.reps,
           "call": "bhmc_batch_step_mc (host buffers; state stays device-resident)"}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    pk, pk_src = peaks()
    bpm, detail = algorithmic_bytes_per_move(bhmc, batch, systems, K, acc_rate)
    launch_ms = ms / args.steps
    achieved = bpm * args.reps * args.moves / (launch_ms / 1e3) / 1e9
    trec = traffic_record()
    traffic = trec["dram_bytes_per_move"] * args.reps * args.moves if trec else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "peak_source": pk_src,
            "traffic_note": ("ncu dram bytes per move of a 96-replica capture x moves per launch"
                             if trec else "kernel changed since the last ncu capture"),
            "kernel": "k_batch (persistent, one replica per block)",
            "bytes_per_move": bpm, "per_move": detail}
    extra = {}
    if not args.no_plain:
        wl1 = W.colloid(n=10000, seed=2, theta=args.theta, p=args.p, C=args.C)
        pr = plain_rate(bhmc, wl1, args.warps)
        extra = {"plain_moves_per_s_colloid_N1e4": pr, "batched_per_replica_moves_per_s": value / args.reps / world,
                 "batched_over_plain": value / pr, "acceptance": acc_rate}
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        v, sample = oracle_sample(systems, seeds, 500, 15.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config(args, sizes, {"parallelism": "replicas" if world == 1 else "replicas x %d ranks" % world}),
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
           "clocks": clk.summary(), **extra}
    print(json.dumps(out), flush=True)
    batch.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

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


def parse(argv=None):
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
    ap.add_argument("--suite", action="store_true",
                    help="one JSON line per workload family instead of the headline line")
    ap.add_argument("--suite-large", action="store_true", help="include the 1e6-ion items in --suite")
    ap.add_argument("--sections", default="plain,grid,edl,single,psweep,n0,fig6,naxis,mala,field,large",
                    help="comma-separated --suite sections")
    return ap.parse_args(argv)


def parse_args(argv):
    return parse(argv)


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
        # raw samples: BHMC_CLOCKS_CSV if set, else a file in the temporary directory
        import tempfile
        self.path = os.environ.get("BHMC_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "bhmc_clocks_%d.csv" % os.getpid())

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


def max_over_ranks(ms, dist, device):
    """The timed region's length: the maximum over ranks (every rank's replicas
    must finish)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(reps, moves, steps, world, ms):
    """Whole-job moves/s: every rank runs its own replicas (weak scaling)."""
    return reps * moves * steps * world / (ms / 1e3)


def workload(args, rank=0):
    from paper_1305_1825_gb300 import workloads as W
    sizes = W.batch_sizes(args.reps, seed=3)
    systems = W.batch(sizes=sizes, theta=args.theta, p=args.p, C=args.C)
    seeds = [1000 + r + 100000 * rank for r in range(args.reps)]
    return sizes, systems, seeds


def config(args, sizes, extra=None):
    c = {"workload": "colloid-%d-replicas" % args.reps, "replicas": args.reps,
         "N_range": [min(sizes), max(sizes)],
         "charges_per_replica": "2N in the tree (ions and images) + the macroion, whose interactions are exact",
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


def _oracle_worker(task):
    """One host core: the FP64 oracle chains of a list of replicas; returns
    (moves, seconds spent in the chains)."""
    import oracle
    work, moves = task
    done, t_total = 0, 0.0
    for (r, seed, wl) in work:
        ref = oracle.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
        t = time.perf_counter()
        ref.mc_run(seed, moves, replica=r)
        t_total += time.perf_counter() - t
        done += moves
    return done, t_total


def oracle_sample_parallel(systems, seeds, moves, per_core):
    """The oracle's replica chains spread over every host core (a spawned
    process per core, `per_core` replicas each); moves/s = all moves over the
    busiest core's chain time.  Returns (moves/s, cores, sample text)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = min(len(systems), cores * per_core)
    tasks = [([(r, seeds[r], systems[r]) for r in range(c, n, cores)], moves) for c in range(cores)]
    tasks = [t for t in tasks if t[0]]
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        res = pool.map(_oracle_worker, tasks)
    total = sum(m for m, _ in res)
    busiest = max(t for _, t in res)
    return total / busiest, len(tasks), ("%d replicas x %d moves over %d host processes (FP64 oracle treecode "
                                         "chains, replica-parallel)" % (n, moves, len(tasks)))


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    sizes, systems, seeds = workload(args)
    vals = []
    sample, cores = "", 1
    for s in range(args.warmup + args.steps):
        v, cores, sample = oracle_sample_parallel(systems, seeds, 150, 1)
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(args, sizes, {"parallelism": "replicas" if args.gpus == 1 else
                                          "replicas x %d ranks" % args.gpus}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def algorithmic_bytes_per_move(bh, batch, systems, K, acc_rate, n_sample_reps=8, n_moves=24):
    """Algorithmic bytes of one trial move from the interaction-list counters
    (equal to the oracle's): 16 B per visited (cluster, point) pair, 4K B of
    moments per multipole evaluation, 16 B per direct pair, and on acceptance
    2 d K 16 B (FP64 moments read and written) + 8 K d B (FP32 mirror) on the
    path of each moved charge (the ion and its image; d = mean leaf depth).
    `layout` counts the bytes of this build's records instead: 32 B cluster
    headers, 32 B leaf slots and (20K + 32) B per cluster on the four ancestor
    paths of an accepted move."""
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
    moved = 2 if systems[0]["params"].get("image") else 1
    commit = acc_rate * moved * (2 * depth * K * 16 + 8 * K * depth)
    b = 16 * V + 4 * K * A + 16 * Pp + commit
    layout = 32 * V + 4 * K * A + 32 * Pp + acc_rate * 4 * (depth + 1) * (20 * K + 32)
    flops = A * (10 * K) + Pp * 14
    return b, {"visited": V, "multipole": A, "direct_pairs": Pp, "leaf_depth": depth,
               "moved_charges": moved, "commit_bytes": commit, "layout_bytes": layout, "fp32_flops": flops}


def de_error_sample(bh, wl, n, seed, warps, layout):
    """dE of the FP32 traversal against the FP64 traversal at the same theta and
    p (the FP64 mode equals the FP64 oracle within 1e-12 of the interaction
    sums, a parity-tested bar) on n random moves of one replica."""
    import numpy as np
    c32 = bh.Context(wl, warps=warps, layout=layout)
    c64 = bh.Context(wl, precision=bh.PREC_F64, warps=warps)
    rng = np.random.default_rng(seed)
    rel = []
    for _ in range(n):
        i = int(rng.integers(0, wl["n_mobile"]))
        b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
        rc, d32, _ = c32.delta_energy(i, b)
        rc2, d64, _ = c64.delta_energy(i, b)
        if rc or rc2:
            continue
        rel.append(abs(d32 - d64) / max(abs(d64), 1e-300))
    c32.close()
    c64.close()
    rel = np.array(rel)
    return {"vs": "FP64 traversal (= FP64 oracle within 1e-12 of the interaction sums, tested)",
            "samples": int(len(rel)), "median": float(np.median(rel)), "p99": float(np.quantile(rel, 0.99)),
            "max": float(rel.max())}


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
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    value = weak_value(args.reps, args.moves, args.steps, world, ms)
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
    moves_per_launch = args.reps * args.moves
    achieved = bpm * moves_per_launch / (launch_ms / 1e3) / 1e9
    trec = traffic_record()
    traffic = trec["dram_bytes_per_move"] * moves_per_launch if trec else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "peak_source": pk_src,
            "traffic_note": ("ncu dram bytes per move of a 96-replica capture x moves per launch"
                             if trec else "kernel changed since the last ncu capture"),
            "kernel": "k_batch (persistent, one replica per block)",
            "bytes_per_move": bpm, "bytes_per_move_layout": detail["layout_bytes"],
            "frac_layout_bytes": detail["layout_bytes"] * moves_per_launch / (launch_ms / 1e3) / 1e9 / pk["hbm_gbs"],
            "dram_frac": (traffic / (launch_ms / 1e3) / 1e9 / pk["hbm_gbs"]) if traffic else None,
            "per_move": detail}
    extra = {}
    if not args.no_plain:
        wl1 = W.colloid(n=10000, seed=2, theta=args.theta, p=args.p, C=args.C)
        pr = plain_rate(bhmc, wl1, args.warps)
        extra = {"plain_moves_per_s_colloid_N1e4": pr, "batched_per_replica_moves_per_s": value / args.reps / world,
                 "batched_over_plain": value / pr, "acceptance": acc_rate}
    extra["dE_error"] = de_error_sample(bhmc, systems[0], 200, 17, args.warps, layout)
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        v1, sample1 = oracle_sample(systems, seeds, 300, 5.0)
        v, cores, sample = oracle_sample_parallel(systems, seeds, 300, 1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": v1, "cores": 1, "sample": sample1}}
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


# ------------------------------------------------------------------ suite
def _ev_time(fn):
    """Device time (ms) of fn() on torch's current stream (the library's stream)."""
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    out = fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _de_errors(bh, wl, n, seed, warps, layout):
    """FP32-traversal dE against the FP64 GPU traversal at the same theta and p
    (the FP64 mode equals the oracle to ~1e-16 of the interaction sums), and
    against the exact dE (theta = 0, FP64)."""
    import copy
    import numpy as np
    tree = bh.Context(wl, warps=warps, layout=layout)
    f64 = bh.Context(wl, precision=bh.PREC_F64, warps=warps)
    ex_wl = copy.deepcopy(wl)
    ex_wl["params"]["theta"] = 0.0
    exact = bh.Context(ex_wl, precision=bh.PREC_F64, warps=8)
    rng = np.random.default_rng(seed)
    rel32, rel_tree, num, den = [], [], 0.0, 0.0
    for _ in range(n):
        i = int(rng.integers(0, wl["n_mobile"]))
        b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
        rc, d32, _ = tree.delta_energy(i, b)
        rc2, d64, _ = f64.delta_energy(i, b)
        rc3, dex, _ = exact.delta_energy(i, b)
        if rc or rc2 or rc3:
            continue
        rel32.append(abs(d32 - d64) / max(abs(d64), 1e-300))
        rel_tree.append(abs(d64 - dex) / max(abs(dex), 1e-300))
        num += (d64 - dex) ** 2
        den += dex ** 2
    for c in (tree, f64, exact):
        c.close()
    rel32, rel_tree = np.array(rel32), np.array(rel_tree)
    q = lambda a, v: float(np.quantile(a, v))
    return {"samples": int(len(rel32)),
            "f32_vs_f64_treecode_rel": {"median": q(rel32, 0.5), "p99": q(rel32, 0.99), "max": float(rel32.max())},
            "treecode_vs_direct_rel": {"median": q(rel_tree, 0.5), "p99": q(rel_tree, 0.99)},
            "E_eq4_1": float(np.sqrt(num / den))}


def _plain_moves(bh, wl, warps, layout, moves, precision=0):
    import torch
    ctx = bh.Context(wl, warps=warps, layout=layout, precision=precision)
    step = wl.get("step", 1.0)
    ctx.step_mc(20, step, seed=wl.get("seed", 1), move0=0)
    ms, _ = _ev_time(lambda: ctx.step_mc(moves, step, seed=wl.get("seed", 1), move0=20))
    ctx.close()
    torch.cuda.synchronize()
    return moves / (ms / 1e3)


def _spec_moves(bh, wl, warps, layout, moves, proposals):
    """One chain in one launch of a cluster of `proposals` CTAs (speculative trials)."""
    import torch
    ctx = bh.Context(wl, warps=warps, layout=layout)
    step = wl.get("step", 1.0)
    ctx.step_mc_spec(200, step, seed=wl.get("seed", 1), move0=0, proposals=proposals)
    ms, out = _ev_time(lambda: ctx.step_mc_spec(moves, step, seed=wl.get("seed", 1), move0=200,
                                                proposals=proposals))
    acc = out[0].accepted / max(out[0].moves, 1)
    ctx.close()
    torch.cuda.synchronize()
    return moves / (ms / 1e3), acc


def _batched_moves(bh, systems, seeds, warps, layout, moves):
    b = bh.Batch(systems, warps=warps, layout=layout)
    step = systems[0].get("step", 1.0)
    b.step_mc(moves // 4, step, seeds)
    ms, st = _ev_time(lambda: b.step_mc(moves, step, seeds, move0=moves // 4))
    acc = sum(s["accepted"] for s in st) / max(sum(s["moves"] for s in st), 1)
    b.close()
    return len(systems) * moves / (ms / 1e3), acc


def _spec_batched_moves(bh, systems, seeds, warps, layout, moves, proposals):
    b = bh.Batch(systems, warps=warps, layout=layout)
    step = systems[0].get("step", 1.0)
    b.step_mc_spec(moves // 4, step, seeds, proposals=proposals)
    ms, _ = _ev_time(lambda: b.step_mc_spec(moves, step, seeds, move0=moves // 4, proposals=proposals))
    b.close()
    return len(systems) * moves / (ms / 1e3)


def _oracle_moves(wl, seed, moves, budget_s):
    import oracle
    ref = oracle.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        ref.mc_run(seed, moves, step=wl.get("step", 1.0), m0=done)
        done += moves
    return done / (time.perf_counter() - t0)


def _direct_forces(q, x, idx, lB):
    """dE/dr_i = -l_B q_i sum_j q_j (r_i - r_j)/|r_i - r_j|^3 (FP64 direct sum)."""
    import numpy as np
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        d = x[i] - x
        r2 = np.einsum("ij,ij->i", d, d)
        r2[i] = np.inf
        out[k] = -lB * q[i] * ((q / r2 ** 1.5)[:, None] * d).sum(axis=0)
    return out


def _field_item(bh, name, wl, reps=3):
    """Full treecode energy and adjoint forces: targets/s, and forces against
    the FP64 direct sum on 64 sampled charges."""
    import numpy as np
    import torch
    ctx = bh.Context(wl, warps=8, layout=bh.LAYOUT_AOS)
    q, x = ctx.charges()
    n = len(q)
    _, cnt = ctx.energy_counters()
    ms_e = min(_ev_time(ctx.energy)[0] for _ in range(reps))
    p = wl["params"]["p"]
    K = (p + 1) * (p + 2) * (p + 3) // 6
    # algorithmic bytes (16 B per visited cluster and per direct pair, 4K B per
    # multipole evaluation) and this build's record bytes (32 B headers and slots)
    bytes_e = 16 * cnt.visited + 4 * K * cnt.accepted + 16 * cnt.pairs
    bytes_layout = 32 * cnt.visited + 4 * K * cnt.accepted + 32 * cnt.pairs
    pk, pk_src = peaks()
    dEdr = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    dEdq = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.forces(dEdr, dEdq)
    ms_f = min(_ev_time(lambda: ctx.forces(dEdr, dEdq))[0] for _ in range(reps))
    g = dEdr.cpu().numpy()
    idx = np.random.default_rng(4).choice(len(q), 64, replace=False)
    want = _direct_forces(q, x, idx, wl["params"].get("lB", 1.0))
    err = np.linalg.norm(g[idx] - want, axis=1) / np.linalg.norm(want, axis=1)
    ctx.close()
    achieved = bytes_e / (ms_e / 1e3) / 1e9
    return {"suite": name, "charges": int(len(q)), "energy_ms": ms_e, "energy_targets_per_s": len(q) / (ms_e / 1e3),
            "energy_roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                "frac": achieved / pk["hbm_gbs"], "peak_source": pk_src,
                                "bytes_per_target": bytes_e / len(q),
                                "frac_layout_bytes": bytes_layout / (ms_e / 1e3) / 1e9 / pk["hbm_gbs"],
                                "per_target": {"visited": cnt.visited / len(q), "multipole": cnt.accepted / len(q),
                                               "direct_pairs": cnt.pairs / len(q)}},
            "forces_ms": ms_f, "forces_targets_per_s": len(q) / (ms_f / 1e3),
            "forces_vs_direct_rel": {"median": float(np.median(err)), "max": float(err.max())},
            "theta": wl["params"]["theta"], "p": wl["params"]["p"]}


def _eq4_1(bh, wl, warps):
    """Eq. (4.1), E = (sum_i |V_i - Vt_i|^2 / sum_i |V_i|^2)^(1/2) over the N
    counterions i = 1..N (the mobile ions), V_i = l_B q_i phi_i with V exact
    (theta = 0, FP64) and Vt the treecode under wl's reading of the macroion
    (fixed_direct); also E of the FP64 traversal and E over every charge."""
    import numpy as np
    n, nt = wl["n_mobile"], wl["n_mobile"] + wl["n_fixed"]
    q = np.asarray(wl["q"][:nt])
    ex = bh.Context(dict(wl, params=dict(wl["params"], theta=0.0)), precision=bh.PREC_F64, warps=8)
    v = ex.potentials()[:nt] * q
    ex.close()
    tr = bh.Context(wl, warps=warps, layout=bh.LAYOUT_AOS)
    vt = tr.potentials()[:nt] * q
    tr.close()
    t64 = bh.Context(wl, precision=bh.PREC_F64, warps=8)
    v64 = t64.potentials()[:nt] * q
    t64.close()
    rel = lambda a, b: float(np.sqrt(np.sum((a - b) ** 2) / np.sum(a ** 2)))
    return {"E_ions": rel(v[:n], vt[:n]), "E_ions_f64_traversal": rel(v[:n], v64[:n]),
            "E_all_charges": rel(v, vt)}


def _equilibrated(bh, wl, moves, warps):
    """Positions of a configuration after `moves` trial moves of the workload's
    own chain (one replica, persistent kernel): the paper measures Eq. (4.1) on
    a snapshot of an equilibrated double layer."""
    b = bh.Batch([wl], warps=warps, layout=bh.LAYOUT_AOS)
    b.step_mc(moves, wl["step"], [wl["seed"]])
    snap = b.replica(0).charges()[1][: wl["n_mobile"] + wl["n_fixed"]].copy()
    b.close()
    return snap


def run_suite(args):
    """One JSON line per workload and setting, in sections (--sections):

    plain   the 2000-charge system, one launch per move, FP32 and FP64
    grid    the 1e4 colloid over theta x p, plain and 152 batched replicas
    edl     the paper's hard-core double layer (Sec. 4) at N = 800 and 1e4 on
            the adaptive and the fixed-level tree
    single  one chain: one launch per move against a cluster of K CTAs
    psweep  Eq. (4.1) over the counterions and moves/s against p = 0..10 at
            theta 0.5 and 0.3 (Figs. 5 and 7), both readings of the macroion
    n0      N_0(p) chosen by timing (Sec. 4)
    fig6    RDF g(r) and ICDF Q(r) sampled inside the chains (Fig. 6):
            treecode at p = 0, 1, 2, 4 against theta = 0 (direct)
    naxis   Eq. (4.1) and moves/s against N = 100..1e4 (Figs. 5 and 7)
    mala    Langevin moves
    field   full energy and adjoint forces at 1e5 charges (1e6 with
            --suite-large)
    large   the 1e6-ion colloid (with --suite-large)

    Moves per second are CUDA-event times on the library's stream; dE errors
    are measured on the GPU against its FP64 mode and the theta = 0 sum."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1825_gb300 import autotune
    from paper_1305_1825_gb300 import bhmc as bh
    from paper_1305_1825_gb300 import workloads as W
    torch.cuda.set_device(0)
    lines = []
    sections = set(args.sections.split(","))
    AOS = bh.LAYOUT_AOS

    def emit(d):
        lines.append(d)
        print(json.dumps(d), flush=True)

    if "plain" in sections:
        wl = W.plain(n=2000)
        emit({"suite": "plain-N2000", "theta": 0.5, "p": 4, "C": 8,
              "gpu_plain_f32_moves_per_s": _plain_moves(bh, wl, 8, AOS, 1000),
              "gpu_plain_f64_moves_per_s": _plain_moves(bh, wl, 8, AOS, 1000, precision=bh.PREC_F64),
              "oracle_moves_per_s": None if args.no_cpu_baseline else _oracle_moves(wl, 1, 200, 3.0),
              "dE_error": _de_errors(bh, wl, 200, 11, 8, AOS)})

    if "grid" in sections:
        for theta in (0.3, 0.5, 0.7):
            for p in (2, 4, 6):
                wl = W.colloid(n=10000, seed=2, theta=theta, p=p, C=args.C)
                systems = [W.colloid(n=10000, seed=2000 + r, theta=theta, p=p, C=args.C) for r in range(152)]
                rate_b, acc = _batched_moves(bh, systems, [2000 + r for r in range(152)], args.warps, AOS, 400)
                rate_p = _plain_moves(bh, wl, args.warps, AOS, 400)
                emit({"suite": "colloid-N1e4", "theta": theta, "p": p, "C": args.C,
                      "gpu_plain_moves_per_s": rate_p, "gpu_batched_152_replicas_moves_per_s": rate_b,
                      "batched_over_plain": rate_b / rate_p, "acceptance": acc,
                      "oracle_moves_per_s": None if args.no_cpu_baseline else _oracle_moves(wl, 2, 100, 2.0),
                      "dE_error": _de_errors(bh, wl, 40, 100 + p, args.warps, AOS)})
                del systems

    if "edl" in sections:
        # the paper's double layer with hard cores (Sec. 4, Eq. 2.1), on the
        # adaptive tree and on the fixed-level tree of Sec. 3.2 (L_max = 6:
        # leaves of side tau)
        for n, reps in ((800, 152), (10000, 16)):
            for Lmax in (0, 6):
                wl = W.edl_hard(n=n, seed=8, Lmax=Lmax)
                rate_p = _plain_moves(bh, wl, args.warps, AOS, 400 if n > 1000 else 1000)
                systems = [W.edl_hard(n=n, seed=8000 + r, Lmax=Lmax) for r in range(reps)]
                rate_b, acc = _batched_moves(bh, systems, [8000 + r for r in range(reps)], args.warps, AOS,
                                             1000 if n <= 1000 else 400)
                spec = {}
                if reps * 8 <= 152:  # few replicas: a cluster of K CTAs per replica
                    for k in (4, 8):
                        spec["gpu_batched_%d_replicas_clusters_of_%d_moves_per_s" % (reps, k)] = \
                            _spec_batched_moves(bh, systems, [8000 + r for r in range(reps)], args.warps, AOS, 4000, k)
                del systems
                emit({"suite": "edl-hard-N%d" % n, "tree": "fixed L_max=%d" % Lmax if Lmax else "adaptive C=8",
                      **spec, "theta": 0.5, "p": 2, "C": 8, "tau": 4.0, "lB": 7.14,
                      "gpu_plain_moves_per_s": rate_p, "gpu_batched_%d_replicas_moves_per_s" % reps: rate_b,
                      "acceptance": acc,
                      "oracle_moves_per_s": None if args.no_cpu_baseline else _oracle_moves(wl, 8, 200, 2.0)})

    if "single" in sections:
        # one chain (the paper's setting): one launch per trial move against one
        # persistent launch of a cluster of K CTAs that evaluates K trials at once
        for wl in (W.edl_hard(n=800, seed=8), W.edl_hard(n=10000, seed=8), W.colloid(n=10000, seed=2, C=args.C)):
            line = {"suite": "single-chain-" + wl["name"], "theta": wl["params"]["theta"], "p": wl["params"]["p"],
                    "gpu_plain_moves_per_s": _plain_moves(bh, wl, args.warps, AOS, 1000)}
            for k in (1, 2, 4, 8):
                rate, acc = _spec_moves(bh, wl, args.warps, AOS, 20000, k)
                line["gpu_cluster_%d_proposals_moves_per_s" % k] = rate
                line["acceptance"] = acc
            emit(line)

    snap = None
    if sections & {"psweep", "n0"}:
        # a snapshot of an equilibrated chain of the N = 800 double layer
        snap = _equilibrated(bh, W.edl_hard(n=800, seed=8), 200000, args.warps)

    if "psweep" in sections:
        # error and speed against the multipole order (Figs. 5 and 7): E of
        # Eq. (4.1) over the 800 counterions with the macroion's interactions
        # exact (the reading adopted) and with the macroion as a tree charge,
        # and moves/s of the workload's own chains (plain and 152 replicas)
        for theta in (0.5, 0.3):
            for pp in range(0, 11):
                wl = W.edl_hard(n=800, seed=8, theta=theta, p=pp)
                wl["xyz"] = snap
                e = _eq4_1(bh, wl, args.warps)
                e_tree = _eq4_1(bh, W.edl_hard(n=800, seed=8, theta=theta, p=pp, fixed_direct=False) | {"xyz": snap},
                                args.warps)
                rate_p = _plain_moves(bh, wl, args.warps, AOS, 1000)
                systems = [W.edl_hard(n=800, seed=8000 + r, theta=theta, p=pp) for r in range(152)]
                rate_b, _ = _batched_moves(bh, systems, [8000 + r for r in range(152)], args.warps, AOS, 1000)
                del systems
                emit({"suite": "p-sweep-edl-N800", "theta": theta, "p": pp,
                      "E_eq4_1_counterions": e["E_ions"], "E_eq4_1_counterions_f64_traversal": e["E_ions_f64_traversal"],
                      "E_eq4_1_all_charges": e["E_all_charges"],
                      "E_eq4_1_counterions_macroion_in_tree": e_tree["E_ions"],
                      "E_eq4_1_all_charges_macroion_in_tree": e_tree["E_all_charges"],
                      "gpu_plain_moves_per_s": rate_p, "gpu_batched_152_replicas_moves_per_s": rate_b})

    if "n0" in sections:
        # N_0(p) by timing (Sec. 4: N_0 chosen from measured times for each p)
        systems = [W.edl_hard(n=800, seed=8000 + r) for r in range(152)]
        seeds = [8000 + r for r in range(152)]
        res = autotune.tune_n0(systems, seeds, warps=args.warps, layout=AOS, moves=1000)
        del systems
        for pp, d in sorted(res.items()):
            wl = W.edl_hard(n=800, seed=8, theta=0.5, p=pp)
            wl["xyz"] = snap
            wl["params"]["N0"] = d["chosen"]
            e = _eq4_1(bh, wl, args.warps)
            emit({"suite": "N0-by-timing-edl-N800", "theta": 0.5, "p": pp, "N0_chosen": d["chosen"],
                  "gpu_batched_152_replicas_moves_per_s": {str(k): v for k, v in d["rates"].items()},
                  "E_eq4_1_counterions_at_chosen_N0": e["E_ions"]})

    if "fig6" in sections:
        # Fig. 6: g(r) and Q(r) of the N = 800 double layer averaged over the
        # chains (sampled inside the persistent kernel every 100 moves after a
        # burn-in), the treecode at theta = 0.5 and p = 0, 1, 2, 4 against
        # theta = 0 (every interaction direct)
        nb, lo, hi, reps = 46, 32.0, 78.0, 152
        qm = -1600.0

        def profiles(theta, pp, burn=20000, moves=100000):
            systems = [W.edl_hard(n=800, seed=8000 + r, theta=theta, p=pp) for r in range(reps)]
            seeds = [8000 + r for r in range(reps)]
            b = bh.Batch(systems, warps=args.warps, layout=AOS)
            b.step_mc(burn, 2.0, seeds)
            b.set_radial_sampling(nb, lo, hi, 100)
            t0 = time.perf_counter()
            b.step_mc(moves, 2.0, seeds, move0=burn)
            dt = time.perf_counter() - t0
            c, q, ns = b.radial_samples()
            b.close()
            halves = []
            for part in (slice(0, reps // 2), slice(reps // 2, reps)):
                halves.append(bh.radial_profiles(c[part].sum(0), q[part].sum(0), lo, hi, int(ns[part].sum()), q_fixed=qm))
            full = bh.radial_profiles(c.sum(0), q.sum(0), lo, hi, int(ns.sum()), q_fixed=qm)
            return full, halves, reps * moves / dt

        (ref, ref_h, rate0) = profiles(0.0, 0)
        noise_g = float(np.abs(ref_h[0][1] - ref_h[1][1]).max())
        noise_Q = float(np.abs(ref_h[0][3] - ref_h[1][3]).max())
        for pp in (0, 1, 2, 4):
            full, _, rate = profiles(0.5, pp)
            emit({"suite": "fig6-rdf-icdf-edl-N800", "theta": 0.5, "p": pp, "bins": nb, "r_range": [lo, hi],
                  "samples_per_replica": 1000, "replicas": reps,
                  "max_abs_dg_vs_direct": float(np.abs(full[1] - ref[1]).max()),
                  "max_abs_dQ_vs_direct": float(np.abs(full[3] - ref[3]).max()),
                  "direct_half_vs_half_max_abs_dg": noise_g, "direct_half_vs_half_max_abs_dQ": noise_Q,
                  "g_first_bins": [float(v) for v in full[1][:6]], "g_direct_first_bins": [float(v) for v in ref[1][:6]],
                  "Q_at_a_plus_4": float(full[3][3]), "Q_direct_at_a_plus_4": float(ref[3][3]),
                  "moves_per_s_with_sampling": rate, "moves_per_s_direct_with_sampling": rate0})

    if "naxis" in sections:
        # Eq. (4.1) over the counterions and moves/s against N (Figs. 5 and 7)
        for n in (100, 300, 1000, 3000, 10000):
            base = W.edl_hard(n=n, seed=8)
            sn = _equilibrated(bh, base, 100000, args.warps)
            line = {"suite": "N-axis-edl", "N": n, "p": 2}
            for theta in (0.5, 0.3):
                wl = W.edl_hard(n=n, seed=8, theta=theta, p=2)
                wl["xyz"] = sn
                line["E_eq4_1_counterions_theta%.1f" % theta] = _eq4_1(bh, wl, args.warps)["E_ions"]
            reps = 152 if n <= 3000 else 16
            systems = [W.edl_hard(n=n, seed=8000 + r) for r in range(reps)]
            line["gpu_batched_%d_replicas_moves_per_s" % reps], line["acceptance"] = _batched_moves(
                bh, systems, [8000 + r for r in range(reps)], args.warps, AOS, 1000 if n <= 3000 else 400)
            del systems
            line["gpu_plain_moves_per_s"] = _plain_moves(bh, base, args.warps, AOS, 400)
            if not args.no_cpu_baseline:
                line["oracle_moves_per_s"] = _oracle_moves(base, 8, 100, 1.0)
            emit(line)

    if "mala" in sections:
        wl = W.colloid(n=10000, seed=2)
        ctx = bh.Context(wl, warps=args.warps, layout=AOS)
        ctx.step_mala(20, 0.05, seed=3)
        ms, (st, _) = _ev_time(lambda: ctx.step_mala(400, 0.05, seed=3, move0=20))
        emit({"suite": "mala-colloid-N1e4", "tau": 0.05, "gpu_moves_per_s": 400 / (ms / 1e3),
              "acceptance": st.accepted / max(st.moves, 1)})
        ctx.close()

    if "field" in sections:
        emit(_field_item(bh, "field-uniform-N1e5", W.uniform(n=100000)))
        emit(_field_item(bh, "field-colloid-scaled-N1e5", W.colloid_scaled(n=100000)))
        if args.suite_large:
            emit(_field_item(bh, "field-large-N1e6", W.large(), reps=2))

    if "large" in sections and args.suite_large:
        wl = W.large()
        ctx = bh.Context(wl, warps=args.warps, layout=AOS)
        ctx.step_mc(20, 1.0, seed=9)
        ms, st = _ev_time(lambda: ctx.step_mc(500, 1.0, seed=9, move0=20))
        ctx.close()
        b = bh.Batch([wl], warps=args.warps, layout=AOS)
        b.step_mc(100, 1.0, [9])
        ms_b, _ = _ev_time(lambda: b.step_mc(4000, 1.0, [9], move0=100))
        b.close()
        rate4, acc4 = _spec_moves(bh, wl, args.warps, AOS, 4000, 4)
        emit({"suite": "large-N1e6", "theta": 0.5, "p": 6, "C": 8, "charges_in_tree": 2000000,
              "gpu_plain_moves_per_s": 500 / (ms / 1e3),
              "gpu_persistent_1_replica_moves_per_s": 4000 / (ms_b / 1e3),
              "gpu_cluster_4_proposals_moves_per_s": rate4, "acceptance": acc4})
    return lines


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.suite:
        run_suite(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

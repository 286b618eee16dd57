"""Autotuner of the batched treecode Monte Carlo: leaf capacity C, warps per
move and the FP32 moment layout (AoS/SoA); and the minimum expansion number
N_0 as a function of the order p (Sec. 3.2: clusters with fewer than N_0
charges are summed directly; Sec. 4 chooses N_0(p) from measured times).

Every candidate runs short persistent batched launches on a subset of the
replicas (CUDA-event timing).  Because C changes the tree and therefore the
interaction lists, each C is also scored for accuracy: the treecode dE of
sampled trial moves against the exact dE from an all-direct FP64 context
(theta = 0) of the same replica, both on the GPU.  The choice is the fastest
candidate whose accuracy is within `acc_factor` of the reference capacity's.
"""
from __future__ import annotations

import copy
import time

import numpy as np

from . import bhmc


def _with_C(systems, C):
    out = []
    for wl in systems:
        w = dict(wl)
        w["params"] = dict(wl["params"], C=C)
        out.append(w)
    return out


def accuracy(systems, n_moves=40, seed=0, reps=4):
    """Median and 99th percentile of |dE_tree - dE_exact| / |dE_exact| over
    sampled trial moves, and the Eq. (4.1)-style ratio
    sqrt(sum |dE_tree - dE_exact|^2 / sum |dE_exact|^2)."""
    rng = np.random.default_rng(seed)
    rel, num, den = [], 0.0, 0.0
    for wl in systems[:reps]:
        tree = bhmc.Context(wl, warps=8, layout=bhmc.LAYOUT_AOS)
        exact_wl = copy.deepcopy(wl)
        exact_wl["params"]["theta"] = 0.0
        exact = bhmc.Context(exact_wl, precision=bhmc.PREC_F64, warps=8)
        for _ in range(n_moves):
            i = int(rng.integers(0, wl["n_mobile"]))
            b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
            rc, d_tree, _ = tree.delta_energy(i, b)
            rc2, d_exact, _ = exact.delta_energy(i, b)
            if rc or rc2:
                continue
            num += (d_tree - d_exact) ** 2
            den += d_exact ** 2
            rel.append(abs(d_tree - d_exact) / max(abs(d_exact), 1e-300))
        tree.close()
        exact.close()
    rel = np.array(rel)
    return {"median_rel": float(np.median(rel)), "p99_rel": float(np.quantile(rel, 0.99)),
            "E": float(np.sqrt(num / den)), "samples": int(len(rel))}


def time_batch(systems, seeds, warps, layout, moves=200, launches=3):
    import torch
    batch = bhmc.Batch(systems, warps=warps, layout=layout)
    step = systems[0].get("step", 1.0)
    batch.step_mc(moves // 4, step, seeds)  # warm-up
    move0 = moves // 4
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(launches):
        batch.step_mc(moves, step, seeds, move0=move0)
        move0 += moves
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    batch.close()
    return len(systems) * moves * launches / (ms / 1e3)


def autotune(systems, seeds, C_values=(4, 8, 16, 32), warps_values=(1, 2, 4, 8),
             layouts=(bhmc.LAYOUT_AOS, bhmc.LAYOUT_SOA), ref_C=8, acc_factor=1.5, moves=200,
             verbose=False):
    """Returns {"best": {...}, "results": [...], "accuracy": {C: {...}}}."""
    results, acc = [], {}
    for C in C_values:
        sysC = _with_C(systems, C)
        acc[C] = accuracy(sysC)
        for warps in warps_values:
            for layout in layouts:
                t = time.time()
                rate = time_batch(sysC, seeds, warps, layout, moves=moves)
                r = {"C": C, "warps": warps, "layout": "aos" if layout == bhmc.LAYOUT_AOS else "soa",
                     "moves_per_s": rate}
                results.append(r)
                if verbose:
                    print(r, "E=%.3g" % acc[C]["E"], "(%.1fs)" % (time.time() - t), flush=True)
    bound = acc_factor * acc[ref_C]["E"] if ref_C in acc else float("inf")
    ok = [r for r in results if acc[r["C"]]["E"] <= bound]
    best = max(ok or results, key=lambda r: r["moves_per_s"])
    return {"best": best, "results": results, "accuracy": acc, "accuracy_bound_E": bound}


def _with(systems, **kw):
    out = []
    for wl in systems:
        w = dict(wl)
        w["params"] = dict(wl["params"], **kw)
        out.append(w)
    return out


def tune_n0(systems, seeds, p_values=tuple(range(11)), n0_values=(0, 2, 4, 8, 16, 32), warps=8,
            layout=bhmc.LAYOUT_AOS, moves=400, tol=0.02, verbose=False):
    """N_0(p) by timing: for each order p the batched moves/s of every N_0, and
    the chosen N_0, the smallest whose rate is within `tol` of the fastest
    (a larger N_0 only adds direct terms, so it never costs accuracy).
    Returns {p: {"chosen": N_0, "rates": {N_0: moves/s}}}."""
    out = {}
    for p in p_values:
        rates = {}
        for n0 in n0_values:
            rates[n0] = time_batch(_with(systems, p=p, N0=n0), seeds, warps, layout, moves=moves)
            if verbose:
                print({"p": p, "N0": n0, "moves_per_s": rates[n0]}, flush=True)
        top = max(rates.values())
        chosen = min(n0 for n0, r in rates.items() if r >= (1.0 - tol) * top)
        out[p] = {"chosen": chosen, "rates": rates}
    return out


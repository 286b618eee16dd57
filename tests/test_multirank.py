"""The replicas-only multi-GPU path, exercised on CPU: two gloo ranks.

Each rank runs its own replicas (seeds offset by rank, no exchange on the data
path); the timed region is the maximum over ranks and the whole-job rate is
the moves of all ranks over it.  The reference arm under torchrun prints one
line from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse_args(["--reps", "3"])
    r, w, _ = bench.dist_env()
    _, _, seeds = bench.workload(args, r)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    out.put((r, w, ms, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, ms0, s0), (r1, w1, ms1, s1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert ms0 == ms1 == 20.0  # every rank times the slowest rank
    assert not set(s0) & set(s1)  # independent chains on every rank
    sys.path.insert(0, ROOT)
    import bench
    assert bench.weak_value(3, 100, 2, 2, 20.0) == pytest.approx(3 * 100 * 2 * 2 / 0.02)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--reps", "4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

"""The N>1 launch path on CPU (gloo, world size 2): replicas only.

Each rank renders its own frame (cameras rotated per rank, no data-path collective); the timed
region is closed by a barrier and the step time is the maximum over ranks, the work the sum."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = bench.load_workload("c1", rank, world)
    eye = [float(x) for x in wl["cams"][0]["eye"]]
    mx = bench.max_over_ranks(dist, float(rank + 1))
    sm = bench.sum_over_ranks(dist, float(10 * (rank + 1)))
    bench.barrier(dist)
    q.put((rank, eye, mx, sm))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, eye0, mx0, sm0), (r1, eye1, mx1, sm1) = res
    assert eye0 != eye1                    # each rank renders its own view
    assert mx0 == mx1 == 2.0               # max over ranks
    assert sm0 == sm1 == 30.0              # total work over ranks


def test_torchrun_reference_arm_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "c1", "--gpus", "2", "--steps", "2", "--warmup", "3",
           "--ref-frac", "0.02"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

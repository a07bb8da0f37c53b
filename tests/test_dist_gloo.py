"""The benchmark's replica path across ranks, on CPU with the gloo backend (world size 2):
the timing aggregates (maximum of the per-rank step time, sum of the per-rank plan counts)
and the reference arm, where rank 0 alone prints the result line."""
import argparse
import json
import os
import socket
import subprocess
import sys

import pytest

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    w, r, _, dist = bench.dist_setup(argparse.Namespace(impl="reference"))
    bench.barrier(dist, torch)
    mx = bench.max_over_ranks(dist, torch, 1.5 + r)
    sm = bench.sum_over_ranks(dist, torch, 10.0 * (r + 1))
    q.put((r, w, mx, sm))
    bench.barrier(dist, torch)
    dist.destroy_process_group()


def test_rank_aggregates_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, w, mx, sm in out:
        assert w == 2 and mx == 2.5 and sm == 30.0


def test_reference_arm_two_ranks():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--workload", "prostate-2k-8plans",
           "--cpu-sample", "2", "--steps", "1", "--warmup", "0", "--max-iters", "30"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "plans/s" and d["value"] >= 0.0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0

"""Several ranks, no GPU: the host side of the multi-process benchmark.

Invocations are independent of one another, so ranks are independent
replicas (weak scaling): every rank holds the same problem, schedules its
own shard of invocations, and the only cross-rank traffic is the timing
reduction.  These tests run two ``gloo`` ranks on the CPU.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, inv = bench.make_workload("medium", rank)
        # the problem is the same on every rank; the invocations are the rank's own
        sig = torch.tensor([int(p.lat_us.astype(np.int64).sum()), int(p.cost_nd.sum() % (1 << 50)),
                            int(inv.dag.astype(np.int64) @ np.arange(inv.n) % (1 << 50))],
                           dtype=torch.int64)
        sigs = [torch.zeros_like(sig) for _ in range(world)]
        dist.all_gather(sigs, sig)
        # each replica's own decisions on a slice of its shard (the oracle stands in
        # for the GPU here: this checks the sharding, not the kernels)
        d, rc = oracle.schedule(p, inv.subset(np.arange(64)))
        # made-up step times: rank r took 1 + r seconds in total
        slowest = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
        value = bench.job_throughput(world, inv.n, 10, slowest)
        q.put((rank, [s.tolist() for s in sigs], int(rc), int(d["flags"].sum()), slowest, value, inv.n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_are_replicas():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, sigs, rc, flags, slowest, value, n in res:
        assert sigs[0][:2] == sigs[1][:2], "ranks must hold the same problem"
        assert sigs[0][2] != sigs[1][2], "ranks must schedule different invocations"
        assert rc == 0 and flags > 0
        assert slowest == 2.0  # the job's time is its slowest rank's
        assert value == pytest.approx(world * n * 10 / 2.0)


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--workload", "tiny"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"

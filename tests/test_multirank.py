"""The N > 1 path of the benchmark, on CPU with two gloo ranks.

Stripes are independent, so N ranks run N replicas of the step with no
collective on the data path: each rank draws its own stripe, and the only
communication is the reduction of the step time to the slowest rank's, from
which the whole-job throughput is computed.  These tests run that host logic
(bench.rank_seed, bench.ranks_max, bench.whole_job_gbps) in two processes
over gloo, which is the same code the NCCL run executes.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_1412_3022_gb300 import inputs  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's stripe comes from its own seed
        X = inputs.blocks(8, 64, seed=bench.rank_seed(7, rank))
        digest = int(np.frombuffer(X.tobytes(), dtype=np.uint8).astype(np.int64).sum())
        # a rank-dependent step time: the job takes the slowest rank's
        my_ms = 1.5 + rank
        slowest = bench.ranks_max(dist, my_ms, "cpu")
        gbps = bench.whole_job_gbps(56 << 20, world, slowest)
        dist.barrier()
        out.put((rank, digest, slowest, gbps))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_use_distinct_stripes():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    slowest = [g[2] for g in got]
    assert slowest == [2.5, 2.5]                      # max over ranks, seen by every rank
    expect = (56 << 20) * world / (2.5e-3) / 1e9     # all ranks' bytes over the slowest time
    assert all(abs(g[3] - expect) < 1e-9 for g in got)
    assert got[0][1] != got[1][1]                     # independent stripes per rank


def test_single_rank_needs_no_process_group():
    assert bench.ranks_max(None, 3.25, "cpu") == 3.25
    assert bench.whole_job_gbps(10**9, 1, 1000.0) == pytest.approx(1.0)
    assert bench.rank_seed(5, 0) != bench.rank_seed(5, 1)

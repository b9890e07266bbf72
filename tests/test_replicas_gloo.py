"""The multi-GPU path runs independent replicas (no data-path collective): two
gloo ranks on the CPU check the benchmark's host logic -- distinct Philox keys
per rank, the job time as the maximum over ranks, whole-job throughput -- and
that the ranks' streams differ (oracle Philox)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.replica_seed(rank)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")  # rank 1 is the slower one
    rate = bench.job_rate(1000.0, world, t)
    draws = [oracle.draw_m(seed, 0, 0, 0, i) for i in range(8)]
    q.put((rank, seed, t, rate, draws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0, d0), (r1, s1, t1, v1, d1) = out
    assert s0 != s1                       # independent streams per replica
    assert t0 == t1 == 15.0               # job time = the slowest rank
    assert v0 == v1 == 2 * 1000.0 / 15.0  # units of both ranks over that time
    assert np.all(np.array(d0) != np.array(d1))

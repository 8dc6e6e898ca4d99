"""The N > 1 bench path on CPU: ranks are independent replicas (no data
exchange); the only collective is the max over ranks of the timed region,
and the whole-job rate counts every rank's node-steps. world_size 2, gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    e2e = 0.2 + 0.1 * rank
    out = bench.aggregate_over_ranks(ms, e2e, world, nodes=1000, steps=10, dist=dist, device="cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_rate_uses_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        value, e2e, ms_max = res[r]
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150 / 1e9)
        assert e2e == pytest.approx(2 * 1000 * 10 / 0.3 / 1e9)


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    value, e2e, ms = bench.aggregate_over_ranks(200.0, 0.5, 1, nodes=500, steps=4)
    assert ms == 200.0 and value == pytest.approx(500 * 4 / 0.2 / 1e9)

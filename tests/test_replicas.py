"""Multi-rank bench logic on CPU: two gloo ranks, slowest-rank time, whole-job throughput.

The path does not shard (replicas only), so the only multi-rank logic is the
timing aggregation; it is exercised here without a GPU.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    worst = bench.max_over_ranks(ms, dist)
    q.put((rank, worst, bench.job_throughput(ws, 20, worst)))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, worst, thr in out:
        assert worst == pytest.approx(150.0)
        assert thr == pytest.approx(2 * 20 / 0.150)

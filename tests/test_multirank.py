"""The N > 1 host path of the benchmark on CPU: two gloo ranks, each with
its own timing, agree on the whole-job time (the slowest rank) and count
both ranks' frames; no data-path collective is involved."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [400.0, 520.0][rank]           # rank 1 is the slow one
    ms, value, w = bench.aggregate_ranks(total_ms, 640000, 10, dist, "cpu")
    q.put((rank, ms, value, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, w in out:
        assert w == 2
        assert ms == pytest.approx(52.0)
        assert value == pytest.approx(2 * 640000 / 0.052)


def test_single_rank_aggregation():
    import bench
    ms, value, w = bench.aggregate_ranks(400.0, 640000, 10)
    assert (w, ms) == (1, 40.0) and value == pytest.approx(640000 / 0.04)

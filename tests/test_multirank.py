"""World-size-2 CPU test (gloo) of the multi-rank bench path: the match does not shard
within one query, so each rank runs an independent replica; the bench takes the slowest
rank's time and reports every rank's templates over it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        my_ms = [120.0, 150.0][rank]
        tmax = bench.max_over_ranks(my_ms, dist, "cpu")
        value = bench.whole_job_value(ws, 32768 * 10, tmax)
        q.put((rank, tmax, value))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, value in res:
        assert tmax == 150.0
        assert abs(value - 2 * 32768 * 10 / 0.150) < 1e-6


def test_single_process_value():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_value(1, 32768, 10.0) == 32768 / 0.010

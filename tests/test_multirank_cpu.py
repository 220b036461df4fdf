"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its own timing; the
whole-job value uses the slowest rank's time (weak scaling, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el_ms = [100.0, 250.0][rank]
    value, mx = bench.aggregate(el_ms, steps=10, world=world)
    q.put((rank, value, mx))
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for rank, value, mx in out:
        assert mx == 250.0
        assert abs(value - 2 * 10 / 0.25) < 1e-9

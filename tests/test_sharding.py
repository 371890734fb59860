"""Multi-rank path on CPU: world size 2 over gloo (127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1905_00473_gb300 import sharding


def test_slice_ranges_cover_every_slice_once():
    for N in (1, 7, 32, 64, 65):
        for world in (1, 2, 3, 8):
            ranges = [sharding.slice_range(N, world, r) for r in range(world)]
            flat = [n for b, e in ranges for n in range(b, e)]
            assert flat == list(range(N))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.slice_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, N, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranges = sharding.gather_ranges(N)
        t = sharding.max_over_ranks(10.0 + rank)
        q.put((rank, ranges, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 9, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ranges, t in res:
        assert ranges == [(0, 5), (5, 9)]
        assert t == 11.0

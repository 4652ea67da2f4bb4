"""Sharding host logic on 2 CPU ranks (gloo): disjoint, complete shards and the
max/sum timing reduction the benchmark uses."""
import os
import socket

import pytest

from paper_2310_15183_gb300 import sharding, workloads as W


def test_pixel_ranges_partition_the_image():
    for n in (1, 7, 1000, 10 ** 6 + 3):
        for world in (1, 2, 3, 8):
            seen = 0
            for r in range(world):
                first, count = sharding.pixel_range(n, r, world)
                assert first == seen
                seen += count
            assert seen == n
    with pytest.raises(ValueError):
        sharding.pixel_range(10, 2, 2)


def test_sweep_cameras_are_distinct():
    cams = [sharding.sweep_camera(W.MN_1000, r, 4) for r in range(4)]
    assert len({c.theta0 for c in cams}) == 4
    assert cams[0] == W.MN_1000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = sharding.pixel_range(1000, rank, world)
        t, u = sharding.reduce_timing(dist, 1.0 + rank, float(count))
        q.put((rank, first, count, t, u))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1:3] for r in res] == [(0, 500), (500, 500)]
    for r in res:
        assert r[3] == 2.0 and r[4] == 1000.0

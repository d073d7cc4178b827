"""The multi-GPU form's host logic on CPU: two `gloo` ranks on 127.0.0.1 (no GPU)."""
import os
import socket

import pytest

from paper_2510_21100_gb300 import shard


def test_shard_range_covers_every_image_once():
    for n in (0, 1, 7, 512):
        for world in (1, 2, 3, 8):
            seen = []
            lens = []
            for r in range(world):
                lo, hi = shard.shard_range(n, r, world)
                seen.extend(range(lo, hi))
                lens.append(hi - lo)
            assert seen == list(range(n))
            assert max(lens) - min(lens) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(4, 2, 2)


def test_rank_seeds_are_distinct_across_ranks():
    a = shard.rank_image_seeds(0, 3)
    b = shard.rank_image_seeds(1, 3)
    assert len(set(a + b)) == 6
    assert a == shard.rank_image_seeds(0, 3)


def test_job_throughput_is_all_ranks_over_the_slowest():
    assert shard.job_throughput(2, 33.1776, 250.0) == pytest.approx(2 * 33.1776 / 0.25)
    with pytest.raises(ValueError):
        shard.job_throughput(1, 1.0, 0.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [1.25, 2.5][rank]
        dist.barrier()
        ms = shard.max_over_ranks(local_ms, dist)
        lo, hi = shard.shard_range(10, rank, world)
        q.put((rank, ms, shard.job_throughput(world, 33.1776, ms), lo, hi))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.5, 2.5]
    assert res[0][2] == pytest.approx(2 * 33.1776 / 0.0025)
    assert (res[0][3], res[0][4], res[1][3], res[1][4]) == (0, 5, 5, 10)

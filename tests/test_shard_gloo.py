"""The multi-rank path of bench.py on CPU: two gloo ranks, no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2201_10473_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = shard.world_info()
        rng = shard.shard_range(r, w, 4096)
        shard.barrier()
        # the slowest rank decides: rank r pretends to take 1 + r seconds
        slowest = shard.max_over_ranks(1.0 + r)
        rate = shard.whole_job_rate(len(rng), w, slowest)
        q.put((r, rng.start, rng.stop, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, s0, v0), (r1, a1, b1, s1, v1) = res
    assert (a0, b0, a1, b1) == (0, 4096, 4096, 8192)        # disjoint, contiguous, weak scaling
    assert s0 == s1 == 2.0                                  # max over ranks
    assert v0 == v1 == 2 * 4096 / 2.0


def test_split_range_covers_exactly():
    for total in (0, 1, 7, 4096, 4099):
        for world in (1, 2, 3, 8):
            got = [shard.split_range(r, world, total) for r in range(world)]
            flat = [i for g in got for i in g]
            assert flat == list(range(total))
            assert max(map(len, got)) - min(map(len, got)) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(2, 2, 10)

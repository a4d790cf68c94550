"""The multi-rank measurement path on CPU: two gloo ranks aggregate their work and time as the benchmark does
on N GPUs (whole-job work over the slowest rank's time), and query shards cover a frame exactly."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_16121_b300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.rank_env() == (rank, world, rank)
        replicas.barrier()
        units, ms = replicas.aggregate(1000.0 * (rank + 1), 2.0 + rank)
        out.put((rank, units, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_work_and_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, units, ms in res:
        assert units == 3000.0 and ms == 3.0  # 1000 + 2000 queries over the slower rank's 3 ms


@pytest.mark.parametrize("n,world", [(8294400, 1), (8294400, 8), (10, 3), (2, 4)])
def test_shards_cover_the_frame(n, world):
    ranges = [replicas.shard(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_aggregate_is_identity():
    assert replicas.aggregate(5.0, 7.0) == (5.0, 7.0)

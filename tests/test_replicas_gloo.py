"""Host logic of replica-parallel runs, with world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest

from paper_2406_06344_gb300 import replicas as R


def test_shard_covers_every_unit_once():
    for total in (0, 1, 7, 1024, 1000003):
        for world in (1, 2, 3, 8):
            spans = [R.shard(total, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.shard(10, 2, 2)


def test_seeds_and_rank_info():
    assert R.replica_seed(1, 0) == 1 and R.replica_seed(1, 3) == 1 + 3 * R.SEED_STRIDE
    info = R.rank_info({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "0"})
    assert (info.rank, info.world, info.local) == (1, 2, 0)
    assert R.rank_info({}) == R.RankInfo(0, 1, 0)


def test_single_process_aggregate_is_identity():
    assert R.aggregate(5, [1.5, 2.0]) == (5.0, [1.5, 2.0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = R.shard(1024, world, rank)
        units, ms = R.aggregate(hi - lo, [10.0 + rank, 3.0 - rank])
        q.put((rank, lo, hi, units, ms))
    finally:
        dist.destroy_process_group()


def test_aggregate_sums_units_and_takes_max_time_over_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1:3] for o in out] == [(0, 512), (512, 1024)]
    for _, _, _, units, ms in out:
        assert units == 1024.0 and ms == [11.0, 3.0]

"""The multi-process aggregation of bench.py on CPU: two gloo ranks time their
own replica; every rank reports the slowest rank's time and the whole-job
throughput counts the steps of both ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # the ranks' own timings
        slowest = bench.max_over_ranks(ms, tdist, "cpu")
        out[rank] = (slowest, bench.job_throughput(world, 200, slowest))
    finally:
        tdist.destroy_process_group()


def test_two_rank_max_and_job_throughput():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        slowest, value = res[rank]
        assert slowest == 150.0
        assert value == pytest.approx(2 * 200 / 0.150)


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_throughput(1, 100, 250.0) == pytest.approx(400.0)


def test_batch_shards_cover_every_simulation_once():
    import bench

    items = list(range(512))
    for world in (1, 2, 3, 8):
        shards = [bench.shard_batch(items, r, world) for r in range(world)]
        assert sorted(x for sh in shards for x in sh) == items
        assert max(map(len, shards)) - min(map(len, shards)) <= 1

"""Host logic of the multi-GPU bench path, on CPU with two gloo ranks.

Each GPU rank computes its own replica (single scene) or its own share of a
batch (scenes dealt longest-first by pixel count); the only collectives are
the timing barrier and the max-over-ranks reduction. These tests run those
pieces in two processes over gloo, with fake per-rank timings.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, weights, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, slowest, bench.shard_lpt(weights, world, rank),
           bench.whole_job_rate(1000.0, world, slowest)))
    dist.destroy_process_group()


def _run(world, weights):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, weights, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_ranks_max_time_and_rate():
    weights = [1.0] * 8
    out = _run(2, weights)
    for rank, slowest, _, rate in out:
        assert slowest == 15.0  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 15.0)


def test_two_ranks_lpt_sharding_partitions_the_batch():
    import bench
    sides = [128, 256, 512, 1024]
    weights = [float(sides[(7 * i) % 4] ** 2) for i in range(40)]
    out = _run(2, weights)
    shards = [s for _, _, s, _ in out]
    got = sorted(shards[0] + shards[1])
    assert got == list(range(len(weights)))  # every scene on exactly one rank
    loads = [sum(weights[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(weights)  # longest-first keeps ranks within one item
    # the same deal as the single-process function
    assert shards == [bench.shard_lpt(weights, 2, r) for r in range(2)]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.shard_lpt([3.0, 1.0, 2.0], 1, 0) == [0, 1, 2]
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_row_slabs_partition_the_grid():
    import paper_1805_08500_gb300 as spm
    for grid_h, tile, world in [(4096, 32, 2), (4096, 32, 3), (1000, 16, 4), (17, 16, 2), (8, 16, 3)]:
        slabs = spm.row_slabs(grid_h, tile, world)
        assert len(slabs) == world
        assert slabs[0][0] == 0 and slabs[-1][1] == grid_h
        for (a0, a1), (b0, b1) in zip(slabs, slabs[1:]):
            assert a1 == b0 and a0 <= a1
        for r0, r1 in slabs:
            assert r0 % tile == 0 and (r1 % tile == 0 or r1 == grid_h)

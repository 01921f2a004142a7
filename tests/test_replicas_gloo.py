"""Replica runs (one independent propagation per GPU, no data-path
collective): the whole-job numbers that bench.py prints under torchrun,
checked with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_info()
        assert (r, w, loc) == (rank, world, rank)
        reduce = bench.make_reduce(dist, torch, "cpu")
        ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
        e2e = 900.0 - 100.0 * rank
        calls = []
        dist.barrier()
        ms_max, value, e2e_total = bench.combine_ranks(ms, e2e, 20, world, reduce)
        calls.append((ms_max, value, e2e_total))
        out[rank] = calls[0]
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    import bench
    want_ms = 150.0
    for rank in (0, 1):
        ms_max, value, e2e_total = res[rank]
        assert ms_max == want_ms                                      # slowest rank
        assert value == pytest.approx(20 * bench.SPLIT * 2 / (want_ms / 1000.0))
        assert e2e_total == pytest.approx(800.0 * 2)                  # slowest rate x ranks


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    reduce = bench.make_reduce(None, torch, "cpu")
    ms_max, value, e2e_total = bench.combine_ranks(120.0, 700.0, 20, 1, reduce)
    assert ms_max == 120.0 and e2e_total == 700.0
    assert value == pytest.approx(20 * bench.SPLIT / 0.120)

"""Host logic of the multi-rank benchmark, on CPU: the size-balanced share of
the batch's trees per rank, and the reduction of time (max) and work (sum)
over two gloo ranks."""
import os
import socket
import tempfile

import pytest

import bench


def test_shard_by_size_covers_every_tree_once_and_balances():
    sizes = [int(64 * 4 ** (2 + (7 * i) % 5)) for i in range(32)]   # uneven, like the star batch
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_by_size(sizes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than one tree
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert bench.shard_by_size([5, 5, 5], 2) == [[0, 2], [1]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.reduce_over_ranks(1.5 + rank, 100 * (rank + 1), "cpu", world)
        with open(os.path.join(out_dir, "r%d" % rank), "w") as fh:
            fh.write("%r %r" % (ms, units))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        for r in range(2):
            ms, units = open(os.path.join(d, "r%d" % r)).read().split()
            assert float(ms) == 2.5 and float(units) == 300.0


def test_reduce_on_one_rank_is_identity():
    assert bench.reduce_over_ranks(3.0, 7, "cpu", 1) == (3.0, 7.0)

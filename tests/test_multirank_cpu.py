"""The N > 1 path of the benchmark on CPU with two gloo ranks: the (q, J) pairs are sharded
round-robin with no overlap and nothing left out, and the whole-job numbers are the maximum of the
ranks' times and the sum of their work (weak scaling, no collective on the data path)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pairs = [(iq, J) for J in (0, 1, 2, 3) for iq in range(8)]
    mine = bench.shard_pairs(pairs, rank, world)
    # each rank reports its own time and the work it did (one unit per pair)
    elapsed = 1.0 + rank
    t, units = bench.reduce_over_ranks(elapsed, len(mine), dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(repr((t, units, gathered, pairs)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_reduction(tmp_path):
    out = tmp_path / "result.txt"
    mp.spawn(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    t, units, shards, pairs = eval(out.read_text())
    assert t == 2.0                      # slowest rank
    assert units == len(pairs)           # every pair counted once
    flat = [p for s in shards for p in s]
    assert sorted(flat) == sorted(pairs) and len(set(flat)) == len(flat)
    assert abs(len(shards[0]) - len(shards[1])) <= 1

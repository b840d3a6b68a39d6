"""The N > 1 path of bench.py on the CPU: world_size-2 `gloo` ranks.

Queries are independent units, so the multi-GPU form shards the batch across ranks with
no collective on the data path and takes the maximum of the per-rank times. These tests
run that host logic (bench.shard, bench.max_over_ranks) in two gloo processes, each
answering its shard with the FP64 oracle, and check that the union of the ranks' answers
is the single-process answer.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def test_shard_partitions_the_batch():
    for total in (0, 1, 7, 10_000, 10_001):
        for ws in (1, 2, 3, 8):
            ranges = [bench.shard(total, ws, r) for r in range(ws)]
            assert ranges[0][0] == 0 and ranges[-1][1] == total
            for (a, b), (c, _) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import taco_oracle as O
    from synth import make_workload

    w, data, queries = make_workload("tiny20k", n=3000, nq=10)
    oix = O.create_index(data, 4, 32, 8, kmeans_iters=4, seed=5)
    lo, hi = bench.shard(len(queries), ws, rank)
    ids, dists, _ = O.search(oix, data, queries[lo:hi], 5, 200, 40)
    # each rank reports a different time; every rank must see the maximum
    t = bench.max_over_ranks([1.0 + rank, 5.0 - rank], ws)
    got = [None] * ws
    dist.all_gather_object(got, (lo, hi, ids, dists))
    if rank == 0:
        np.save(os.path.join(out_dir, "times.npy"), np.array(t))
        all_ids = np.concatenate([g[2] for g in sorted(got, key=lambda g: g[0])])
        all_d = np.concatenate([g[3] for g in sorted(got, key=lambda g: g[0])])
        np.save(os.path.join(out_dir, "ids.npy"), all_ids)
        np.save(os.path.join(out_dir, "dists.npy"), all_d)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    from oracle import taco_oracle as O
    from synth import make_workload

    w, data, queries = make_workload("tiny20k", n=3000, nq=10)
    oix = O.create_index(data, 4, 32, 8, kmeans_iters=4, seed=5)
    ids, dists, _ = O.search(oix, data, queries, 5, 200, 40)
    assert np.array_equal(np.load(tmp_path / "ids.npy"), ids)
    assert np.array_equal(np.load(tmp_path / "dists.npy"), dists)
    assert list(np.load(tmp_path / "times.npy")) == [2.0, 5.0]

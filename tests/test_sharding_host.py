"""Id-range shards on the CPU: the host combine of paper_2603_24919_gb300.sharding and the
exchange protocol of taco_shard_count / taco_shard_select, run with the FP64 oracle.

Two `gloo` ranks each hold one id range of the points. Every rank probes the same cells
(the global cell sizes), counts the collisions of its own ids (Def. 6), and reports its level
counts; after the all-reduce every rank finds the one-index Alg. 5 threshold, re-ranks its own
candidates, and the all-gather + merge by (distance, id) must give the one-index answer of
the oracle's search, ids and distances."""
import os
import socket

import numpy as np
import pytest

from paper_2603_24919_gb300 import sharding

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_merge_orders_by_distance_then_id_and_pads():
    a = (np.array([[5, 3, -1], [7, -1, -1]]), np.array([[1.0, 2.0, np.inf], [0.5, np.inf, np.inf]], np.float32))
    b = (np.array([[2, 9, 4], [8, 1, -1]]), np.array([[1.0, 2.0, 3.0], [0.5, 0.25, np.inf]], np.float32))
    ids, d = sharding.merge_topk([a, b], 3)
    assert ids.tolist() == [[2, 5, 3], [1, 7, 8]]             # ties at 1.0 and 0.5 by id
    assert d.tolist() == [[1.0, 1.0, 2.0], [0.25, 0.5, 0.5]]
    ids, d = sharding.merge_topk([a, b], 3, ks=[1, 2])          # per-query k
    assert ids.tolist() == [[2, -1, -1], [1, 7, -1]]
    assert np.isinf(d[0, 1:]).all() and np.isinf(d[1, 2])
    e = (np.full((2, 3), -1), np.full((2, 3), np.inf, np.float32))
    ids, d = sharding.merge_topk([e, e], 3)                     # no candidates anywhere
    assert (ids == -1).all() and np.isinf(d).all()


def test_reduce_counts_sums_shards():
    h = [np.array([[10, 4, 1]]), np.array([[7, 2, 0]]), np.array([[3, 3, 3]])]
    assert sharding.reduce_counts(h).tolist() == [[20, 9, 4]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_answer(oix, data, q, k, budget, target, lo, hi, group=None):
    """One rank's side of the protocol for one query, with the oracle's steps."""
    from oracle import taco_oracle as O
    Ns = oix.n_subspaces
    q_t = O.transform(np.asarray(q, np.float64)[None, :], oix.o_bar, oix.B)[0]
    probed = []
    for i in range(Ns):
        d1, d2 = O.half_distances(oix, q_t, i)
        kept, _, _ = O.probe_by_definition(d1, d2, oix.cell_sizes(i), budget)   # global sizes
        probed.append(np.asarray(kept, dtype=np.int64))
    sc = O.collision_counts(oix, probed)[lo:hi]            # this shard's ids only
    hist = np.array([[hi - lo] + [int((sc >= j).sum()) for j in range(1, Ns + 1)]], dtype=np.int64)
    g = sharding.allreduce_counts(hist, group)[0]           # [N_s + 1]: ids with SC >= j, all shards
    level = np.append(g, 0)
    counts = level[:-1] - level[1:]                          # ids with SC == j
    fake = np.repeat(np.arange(Ns + 1), counts)              # same level histogram as the whole index
    _, _, last, _ = O.candidate_selection(fake, Ns, target)
    C = lo + np.nonzero(sc >= last)[0]
    ids, dists, _ = O.rerank(data, q, C, k)
    return ids[None, :], dists[None, :].astype(np.float32), last


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import taco_oracle as O
    from synth import make_workload

    w, data, queries = make_workload("tiny20k", n=3000, nq=6)
    oix = O.create_index(data, 4, 32, 8, kmeans_iters=4, seed=5)
    bounds = [0, 1700, 3000]                               # uneven id ranges
    lo, hi = bounds[rank], bounds[rank + 1]
    rows = []
    for qi, (budget, target) in enumerate([(200, 40), (400, 60), (80, 2500)] * 2):   # last 2 reach level <= 1
        ids, dists, last = _shard_answer(oix, data, queries[qi], 5, budget, target, lo, hi)
        mids, md = sharding.allgather_merge(ids, dists, 5)
        rows.append((mids[0], md[0], last))
    if rank == 0:
        np.save(os.path.join(out_dir, "ids.npy"), np.stack([r[0] for r in rows]))
        np.save(os.path.join(out_dir, "dists.npy"), np.stack([r[1] for r in rows]))
        np.save(os.path.join(out_dir, "last.npy"), np.array([r[2] for r in rows]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_id_range_shards_equal_one_index(tmp_path):
    from oracle import taco_oracle as O
    from synth import make_workload

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    ids = np.load(tmp_path / "ids.npy")
    dists = np.load(tmp_path / "dists.npy")
    last = np.load(tmp_path / "last.npy")
    w, data, queries = make_workload("tiny20k", n=3000, nq=6)
    oix = O.create_index(data, 4, 32, 8, kmeans_iters=4, seed=5)
    for qi, (budget, target) in enumerate([(200, 40), (400, 60), (80, 2500)] * 2):
        t = O.search_one(oix, data, queries[qi], 5, budget, target)
        assert last[qi] == t.last_collision
        np.testing.assert_array_equal(ids[qi], t.ids)
        np.testing.assert_allclose(dists[qi], t.dists, rtol=1e-6)
    assert (last[[2, 5]] <= 1).all()   # the cases below level 2 (the codes fallback's) are covered


def test_shard_select_checks_its_arguments_before_the_library():
    import ctypes as C

    from paper_2603_24919_gb300.taco import ShardSearch

    class _Index:   # stands in for TacoIndex: only what the checks read
        def __init__(self, h):
            self._h = h

        def info(self):
            return {"n_subspaces": 6}

    # stand-in handles are never freed: each object's handle is cleared before it goes away
    g = np.zeros((4, 7), dtype=np.int64)
    with pytest.raises(ValueError, match="handle is closed"):
        ShardSearch(C.c_void_p(0), 4, 10, _Index(C.c_void_p(1))).select(g)
    sh = ShardSearch(C.c_void_p(1), 4, 10, _Index(None))
    try:
        with pytest.raises(ValueError, match="index is closed"):
            sh.select(g)
    finally:
        sh.handle = None
    sh = ShardSearch(C.c_void_p(1), 4, 10, _Index(C.c_void_p(1)))
    try:
        for bad in (np.zeros((4, 6), np.int64), np.zeros((3, 7), np.int64), np.zeros(28, np.int64)):
            with pytest.raises(ValueError, match="global_hist must be"):
                sh.select(bad)
    finally:
        sh.handle = None

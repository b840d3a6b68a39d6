"""Combining the outputs of id-range shards (taco_shard_count / taco_shard_select).

A search split over the points needs two exchanges per batch: the level counts of Alg. 5
summed over the shards (every shard then finds the same threshold), and the shards' k
nearest merged by (distance, id). In one process the shards' outputs are NumPy arrays and
`reduce_counts` / `merge_topk` combine them; across processes (one shard per rank)
`allreduce_counts` / `allgather_merge` do the same with torch.distributed collectives on
[nq][N_s + 1] int64 counts and [nq][k] results.
"""
from __future__ import annotations

import numpy as np

_NO_ID = np.int64(-1)


def reduce_counts(hists):
    """Sum of the shards' level counts ([S] arrays of [nq, N_s + 1] int64)."""
    return np.sum(np.stack([np.asarray(h, dtype=np.int64) for h in hists]), axis=0)


def _order_keys(ids, dists):
    """64-bit keys that order (distance, id) pairs: the FP32 bit pattern of a non-negative
    distance (or +inf) in the high word, the id in the low word; missing entries (-1) last."""
    bits = np.ascontiguousarray(dists, dtype=np.float32).view(np.uint32).astype(np.uint64)
    idw = np.where(ids < 0, np.uint64(0xFFFFFFFF), ids.astype(np.uint64))
    return (bits << np.uint64(32)) | idw


def merge_topk(parts, k_stride, ks=None):
    """The k nearest of the shards' results. parts: [(ids [nq, k_stride] int64, dists
    [nq, k_stride] float32), ...] with -1 / +inf past a shard's candidates; ks: each query's k
    (None: k_stride). Returns (ids, dists) [nq, k_stride], -1 / +inf past the query's k."""
    ids = np.concatenate([np.asarray(p[0], dtype=np.int64) for p in parts], axis=1)
    dists = np.concatenate([np.asarray(p[1], dtype=np.float32) for p in parts], axis=1)
    order = np.argsort(_order_keys(ids, dists), axis=1, kind="stable")[:, :k_stride]
    out_ids = np.take_along_axis(ids, order, axis=1)
    out_d = np.take_along_axis(dists, order, axis=1)
    if ks is not None:
        past = np.arange(k_stride)[None, :] >= np.asarray(ks, dtype=np.int64)[:, None]
        out_ids[past] = _NO_ID
        out_d[past] = np.float32(np.inf)
    return out_ids, out_d


def allreduce_counts(hist, group=None):
    """reduce_counts across the ranks of a process group (one shard per rank)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(hist, dtype=np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


def allgather_merge(ids, dists, k_stride, ks=None, group=None):
    """merge_topk across the ranks of a process group (one shard per rank)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    ti = torch.from_numpy(np.ascontiguousarray(ids, dtype=np.int64))
    td = torch.from_numpy(np.ascontiguousarray(dists, dtype=np.float32))
    gi = [torch.empty_like(ti) for _ in range(ws)]
    gd = [torch.empty_like(td) for _ in range(ws)]
    dist.all_gather(gi, ti, group=group)
    dist.all_gather(gd, td, group=group)
    return merge_topk([(a.numpy(), b.numpy()) for a, b in zip(gi, gd)], k_stride, ks)

"""bench.py's CPU baseline on the host cores: the FP64 oracle's query routine in spawned
processes over one index, queries dealt round-robin, clocks started at a common barrier.

The pool must answer queries and report the processes it used; procs = 1 times the
routine in this process.
"""
import numpy as np

import bench
from oracle import taco_oracle as O
from synth import make_workload


def _parts():
    w, data, queries = make_workload("tiny20k", nq=12)
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=3, seed=1)
    parts = {"o_bar": oix.o_bar, "B": oix.B, "centroids": oix.centroids,
             "codes": oix.codes.astype(np.uint16)}
    return w, data, queries, parts


def test_pool_uses_every_process():
    w, data, queries, parts = _parts()
    op = {"alpha": 0.05, "beta": 0.01}
    r = bench.cpu_baseline_parts(parts, data, queries, (w.n_subspaces, w.sub_dim, w.sqrt_k), op,
                                 seconds=1.0, procs=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0
    assert "2 processes" in r["sample"]


def test_single_process_fallback():
    w, data, queries, parts = _parts()
    op = {"alpha": 0.05, "beta": 0.01}
    r = bench.cpu_baseline_parts(parts, data, queries, (w.n_subspaces, w.sub_dim, w.sqrt_k), op,
                                 seconds=0.5, procs=1)
    assert r["cores"] == 1 and r["value"] > 0 and "single process" in r["sample"]


def test_pool_failure_falls_back_to_one_process(monkeypatch):
    """A pool that fails (here: a process that raises at start-up) leaves the baseline to
    this process alone instead of losing the bench line."""
    w, data, queries, parts = _parts()

    class Broken:
        def __init__(self, *a, **k):
            raise ValueError("injected start-up failure")

    monkeypatch.setattr(bench, "OraclePool", Broken)
    r = bench.cpu_baseline_parts(parts, data, queries, (w.n_subspaces, w.sub_dim, w.sqrt_k),
                                 {"alpha": 0.05, "beta": 0.01}, seconds=0.5, procs=4)
    assert r["cores"] == 1 and r["value"] > 0 and "single process" in r["sample"]

"""bench.py's host-side measurement helpers on the CPU.

- The exact k-NN used as recall ground truth (FP32 candidate pool, FP64 re-check ordered by
  distance then id) equals the oracle's FP64 brute force, also on integer data with exact
  distance ties and with data blocks smaller than n (the running top-k merge).
- recall@k and the per-query-k recall on hand-made cases.
- The clock sampler's parsing of nvidia-smi records: median SM clock, maximum, and the
  throttle reasons that make a run invalid.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from oracle import taco_oracle as O  # noqa: E402


def _data(seed, n, d, integer):
    rng = np.random.default_rng(seed)
    if integer:   # small integer coordinates: many exactly equal distances
        data = rng.integers(0, 4, size=(n, d)).astype(np.float32)
        queries = rng.integers(0, 4, size=(40, d)).astype(np.float32)
    else:
        data = rng.standard_normal((n, d)).astype(np.float32)
        queries = rng.standard_normal((40, d)).astype(np.float32)
    return data, queries


@pytest.mark.parametrize("integer", [False, True])
def test_exact_knn_equals_oracle_brute_force(integer):
    data, queries = _data(3, 5000, 12, integer)
    want, _ = O.brute_force_knn(data, queries, 10)
    dt, qt = torch.from_numpy(data), torch.from_numpy(queries)
    got = bench.exact_knn_gpu(torch, dt, qt, data, queries, 10, extra=200, chunk=16)
    blk = bench.exact_knn_blocked(torch, dt, qt, data, queries, 10, extra=200, qchunk=16,
                                  dchunk=777)
    if integer:
        # FP32 pools may differ among exact ties beyond the pool; the FP64 distances of the
        # returned lists must match the oracle's
        def dists(ids):
            return np.sort(((data[ids].astype(np.float64) - queries[:, None, :]) ** 2).sum(-1), 1)
        np.testing.assert_array_equal(dists(got), dists(want))
        np.testing.assert_array_equal(dists(blk), dists(want))
    else:
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(blk, want)


def test_recall_helpers():
    truth = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    ids = np.array([[4, 3, 9, 9], [5, 0, 0, 0]])
    assert bench.recall_at(ids, truth, 2) == pytest.approx((0 + 0.5) / 2)
    assert bench.recall_at(ids, truth, 4) == pytest.approx((2 / 4 + 1 / 4) / 2)
    assert bench.recall_per_query_k(ids, truth, [4, 1]) == pytest.approx((2 / 4 + 1.0) / 2)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parsing():
    s = bench.ClockSampler(0)
    s.f = open(s.path, "w")
    s.proc = _Done()
    s.f.write("1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "2070, 2070, 1210.5, 0x4, Not Active, Not Active, Not Active, Active\n"
              "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "2070, 2070, 1250.0, 0x8, Active, Not Active, Not Active, Not Active\n")
    s.f.flush()
    r = s.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_algorithmic_bytes_formulas():
    """Per-launch algorithmic bytes on a hand-counted batch: 2 queries, 1,000 retrieved ids,
    30 probed cells, 50 candidates, 20 level-list entries, d = 128, k = 10, shortlist 2k."""
    a = bench.algorithmic_bytes(2, 1000, 30, 50, 20, d=128, d_pad=128, k=10, mult=2, n_ranges=3,
                                n_subspaces=8, sqrt_k=64)
    io = 2 * (128 * 4 + 10 * 12)
    assert a["count_lists"] == 4000 + 240 + 80 + 2 * 3 * 72
    assert a["select_rerank"] == 50 * 256 + 2 * 20 * 512 + 80 + 2 * 3 * 72 + io
    assert a["probe_cells"] == 2 * 8 * 4096 * 4 + 60
    assert a["path"] == 4000 + 120 + 50 * 256 + 2 * 20 * 512 + io
    # the shortlist is capped at 512 rows
    b = bench.algorithmic_bytes(1, 0, 0, 0, 0, d=8, d_pad=8, k=100, mult=8, n_ranges=1,
                                n_subspaces=1, sqrt_k=1)
    assert b["path"] == 512 * 8 * 4 + 8 * 4 + 100 * 12


def test_ncu_figures_follow_the_kernel_source(monkeypatch):
    """Traffic and limiter come from the committed summary only while its source hash is
    the current one."""
    import json
    import os
    j = json.load(open(os.path.join(bench.ROOT, "profiles", "count_lists_deep10m.json")))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: j["bf16"]["source_hash"])
    assert bench.ncu_traffic("count_lists", "bf16", "deep10m") == j["bf16"]["dram_bytes_per_launch_full_batch"]
    if j.get("limiter", {}).get("source_hash") == j["bf16"]["source_hash"]:
        assert bench.ncu_limiter("count_lists", "deep10m")["issue_active_pct"] > 0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("count_lists", "bf16", "deep10m") is None
    assert bench.ncu_limiter("count_lists", "deep10m") is None
    assert bench.ncu_traffic("no_such_kernel", "bf16", "deep10m") is None
    assert bench.ncu_traffic("count_lists", "bf16", "no_such_workload") is None

"""taco_autotune: it times searches of a sample over counter layouts, counting CTA sizes and
walk depths, lanes per row and probe strategies, keeps the fastest, and the searches that
follow still match the FP64 oracle under the parity rule (the layout is exact integer work;
only the FP32 summation order of a distance may change). reps <= 0 restores the default
layout. Every counting variant, forced through taco_index_set_option, matches the oracle,
with 4-bit counters (up to 12 slabs per range) and 3-bit counters (13-15 slabs, N_s <= 7)."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import budget_from_alpha, target_from_beta
from tests.parity_util import ParityReport, check_exclusions, compare_query, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoIndex, build_lib  # noqa: E402

build_lib.build()


@pytest.fixture(scope="module")
def multislab():
    rng = np.random.default_rng(91)
    n, d = 300_001, 32
    centres = rng.uniform(0, 60, size=(200, d))
    data = (centres[rng.integers(0, 200, n)] + 5 * rng.standard_normal((n, d))).astype(np.float32)
    queries = (centres[rng.integers(0, 200, 40)] + 5 * rng.standard_normal((40, d))).astype(np.float32)
    oix = O.create_index(data, 4, 8, 32, kmeans_iters=6, seed=9)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              4, 8, 32, keep_bf16=True)
    yield data, queries, oix, ix
    ix.close()


def _parity(ix, oix, data, queries, k, b, t):
    q = torch.from_numpy(queries).cuda()
    dbg = to_numpy(ix.search_debug(q, k, b, t))
    rep = ParityReport()
    for j, qq in enumerate(queries):
        compare_query(rep, O.search_one(oix, data, qq, k, b, t), dbg, j, k, oix.n)
    check_exclusions(rep, f"autotune k={k} b={b} t={t}")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_autotune_keeps_parity(multislab, precision):
    data, queries, oix, ix = multislab
    b, t = budget_from_alpha(0.05, oix.n), target_from_beta(0.01, oix.n)
    q = torch.from_numpy(queries).cuda()
    before_ids, _ = ix.search(q, 10, b, t, precision=precision, shortlist_mult=2)
    r = ix.autotune(q, 10, b, t, precision=precision, shortlist_mult=2, reps=2)
    assert r["trials"] >= 5 and 0 < r["ms_after"] <= r["ms_before"]
    assert r["slabs_per_range"] in (1, 2, 4, 5, 8, 10) and r["n_ranges"] * r["slabs_per_range"] >= 10
    assert r["lanes_per_row"] in (0, 4, 8, 16, 32) and r["probe_walk"] in (-1, 0)
    assert r["count_warps"] in (8, 16, 32) and r["walk_unroll"] in (2, 4, 8)
    _parity(ix, oix, data, queries, 10, b, t)
    after_ids, _ = ix.search(q, 10, b, t, precision=precision, shortlist_mult=2)
    same = (before_ids == after_ids).all(dim=1).float().mean().item()
    assert same >= 0.9   # only near-ties of FP32 distances may reorder
    d = ix.autotune(None, 10, b, t, reps=0)
    assert d["slabs_per_range"] * d["n_ranges"] >= 10 and d["lanes_per_row"] == 0
    assert d["count_warps"] == 16 and d["walk_unroll"] == 4
    assert ix.device_status() == 0


def test_every_counter_layout_matches_oracle(multislab):
    """Force each counter layout through the tuner's reset-and-trial path by tuning on
    different samples, and check parity after each."""
    data, queries, oix, ix = multislab
    b, t = budget_from_alpha(0.02, oix.n), target_from_beta(0.005, oix.n)
    q = torch.from_numpy(queries).cuda()
    for sample in (q[:8], q[8:24], q):
        ix.autotune(sample, 10, b, t, reps=1)
        _parity(ix, oix, data, queries[:16], 10, b, t)
    ix.autotune(None, 10, b, t, reps=0)


@pytest.mark.parametrize("spc,warps,unroll", [(4, 16, 4), (4, 32, 4), (4, 16, 8), (12, 16, 8),
                                              (1, 16, 8), (8, 32, 2), (5, 16, 4), (5, 8, 2),
                                              (3, 8, 4), (12, 16, 2)])
def test_forced_count_variants_match_oracle(multislab, spc, warps, unroll):
    """Each (slabs per range, warps, walk depth) variant of the counting pass, including
    one-slab ranges and a range wider than the index (12 > 10 slabs)."""
    data, queries, oix, ix = multislab
    b, t = budget_from_alpha(0.03, oix.n), target_from_beta(0.005, oix.n)
    ix.set_count_layout(slabs_per_range=spc, count_warps=warps, walk_unroll=unroll)
    try:
        _parity(ix, oix, data, queries[:20], 10, b, t)
        assert ix.device_status() == 0
    finally:
        ix.autotune(None, 10, b, t, reps=0)


@pytest.mark.parametrize("spc,warps,unroll", [(4, 8, 2), (5, 8, 4), (12, 16, 4), (4, 32, 2)])
def test_count_variants_with_more_cells_than_one_staging_batch(multislab, spc, warps, unroll):
    """alpha = 0.3 probes about 300 cells in each of the 4 subspaces, more than one staging
    batch holds (512): the counting pass stages and walks the cells in batches of one cell per
    thread (256 with 8 warps), and every variant still matches the oracle."""
    data, queries, oix, ix = multislab
    b, t = budget_from_alpha(0.3, oix.n), target_from_beta(0.01, oix.n)
    ix.set_count_layout(slabs_per_range=spc, count_warps=warps, walk_unroll=unroll)
    try:
        _parity(ix, oix, data, queries[:12], 10, b, t)
        dbg = to_numpy(ix.search_debug(torch.from_numpy(queries[:12]).cuda(), 10, b, t, want_sc=False))
        assert (dbg["probed"].reshape(12, -1).sum(axis=1) > 512).all()
        assert ix.device_status() == 0
    finally:
        ix.autotune(None, 10, b, t, reps=0)


def test_count_layout_rejects_bad_values(multislab):
    from paper_2603_24919_gb300 import TacoError
    data, queries, oix, ix = multislab
    for kw in (dict(slabs_per_range=0), dict(slabs_per_range=16), dict(count_warps=4),
               dict(walk_unroll=12)):
        with pytest.raises(TacoError) as err:
            ix.set_count_layout(**kw)
        assert err.value.code == -1


@pytest.fixture(scope="module")
def wide():
    """16 slabs (500,003 points, N_s = 4): a 15-slab range and a ragged one-slab range."""
    rng = np.random.default_rng(93)
    n, d = 500_003, 32
    centres = rng.uniform(0, 60, size=(200, d))
    data = (centres[rng.integers(0, 200, n)] + 5 * rng.standard_normal((n, d))).astype(np.float32)
    queries = (centres[rng.integers(0, 200, 24)] + 5 * rng.standard_normal((24, d))).astype(np.float32)
    oix = O.create_index(data, 4, 8, 32, kmeans_iters=6, seed=9)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              4, 8, 32, keep_bf16=True)
    yield data, queries, oix, ix
    ix.close()


@pytest.mark.parametrize("spc,warps,unroll", [(15, 16, 4), (15, 8, 2), (15, 32, 4), (13, 16, 8),
                                              (14, 16, 2), (12, 16, 4)])
def test_three_bit_counters_match_oracle(wide, spc, warps, unroll):
    """13-15 slabs per range count in 3-bit counters (10 a word); SC-scores, level counts,
    last_collision and results match the oracle bit-exactly as with 4-bit counters."""
    data, queries, oix, ix = wide
    assert ix.info()["n_slabs"] == 16
    b, t = budget_from_alpha(0.03, oix.n), target_from_beta(0.004, oix.n)
    ix.set_count_layout(slabs_per_range=spc, count_warps=warps, walk_unroll=unroll)
    try:
        _parity(ix, oix, data, queries, 10, b, t)
        assert ix.device_status() == 0
    finally:
        ix.autotune(None, 10, b, t, reps=0)


def test_three_bit_counters_refused_above_seven_subspaces():
    from paper_2603_24919_gb300 import TacoError
    rng = np.random.default_rng(5)
    data = rng.standard_normal((40_000, 64)).astype(np.float32)
    ix = TacoIndex.build(data, 8, 8, 16, kmeans_iters=2, seed=1)
    try:
        with pytest.raises(TacoError) as err:
            ix.set_count_layout(slabs_per_range=13)
        assert err.value.code == -1
        ix.set_count_layout(slabs_per_range=12)
    finally:
        ix.close()

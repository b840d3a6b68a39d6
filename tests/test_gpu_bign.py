"""The codes fallback for the queries the two-pass search cannot finish (Alg. 5 threshold
below 2, or a level list past its slot): SC-scores recomputed from the cell codes of the
probed points (Def. 6) instead of the cluster kernel's shared-memory counters.

Forced on the 20k x 128 workload and a multi-slab index, every intermediate and result must
match the FP64 oracle under the parity rule for budgets and targets that reach each case
(threshold 0 = all points, threshold 1, overflowing lists). An index with more points than
any cluster's shared memory holds (6.4M > 16 x 11 x 2^15) uses it always: sampled queries
match the oracle on the exported index, and the entry points that need a cluster refuse."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import budget_from_alpha, make_workload, target_from_beta
from tests.parity_util import ParityReport, check_exclusions, compare_query, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoError, TacoIndex, build_lib  # noqa: E402

build_lib.build()


def _check(ix, oix, data, queries, k, b, t, **kw):
    q = torch.from_numpy(queries).cuda()
    dbg = to_numpy(ix.search_debug(q, k, b, t, **kw))
    rep = ParityReport()
    for j, qq in enumerate(queries):
        compare_query(rep, O.search_one(oix, data, qq, k, b, t), dbg, j, k, oix.n)
    check_exclusions(rep, f"codes fallback k={k} b={b} t={t}")
    assert ix.device_status() == 0
    return dbg


@pytest.fixture(scope="module")
def tiny():
    w, data, queries = make_workload("tiny20k", nq=40)
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=10, seed=1)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              w.n_subspaces, w.sub_dim, w.sqrt_k, keep_bf16=True)
    ix.set_codes_fallback(True)
    yield w, data, queries, oix, ix
    ix.close()


@pytest.mark.parametrize("budget,target", [(1000, 200), (200, 5000), (50, 19_000), (20_000, 400),
                                           (3000, 10 ** 9)])
def test_codes_fallback_parity(tiny, budget, target):
    w, data, queries, oix, ix = tiny
    dbg = _check(ix, oix, data, queries, 10, budget, target)
    if target >= 10 ** 9:
        assert np.all(dbg["candidate_num"] == oix.n)   # threshold 0: every point


def test_codes_fallback_bf16_and_k(tiny):
    w, data, queries, oix, ix = tiny
    _check(ix, oix, data, queries, 100, 300, 3000, precision="bf16", shortlist_mult=4)


@pytest.fixture(scope="module")
def big():
    rng = np.random.default_rng(123)
    n, d = 6_400_000, 16
    centres = rng.uniform(0, 100, size=(512, d)).astype(np.float32)
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, 1 << 20):
        m = min(n, a + (1 << 20)) - a
        data[a:a + m] = centres[rng.integers(0, 512, m)] + 3 * rng.standard_normal((m, d), dtype=np.float32)
    queries = (centres[rng.integers(0, 512, 6)] + 3 * rng.standard_normal((6, d))).astype(np.float32)
    ix = TacoIndex.build(data, 2, 8, 32, kmeans_iters=4, seed=7, keep_bf16=True)
    ex = ix.export()
    oix = O.index_from_parts(ex["o_bar"], ex["B"], ex["centroids"], ex["codes"], 2, 8, 32)
    yield data, queries, oix, ix
    ix.close()


def test_big_index_parity(big):
    data, queries, oix, ix = big
    info = ix.info()
    assert info["n_slabs"] > 16 * 12 and info["cluster_size"] == 0
    b, t = budget_from_alpha(0.001, oix.n), target_from_beta(0.0005, oix.n)
    _check(ix, oix, data, queries, 10, b, t)
    # the autotuner's reset restores the index's own two-pass layout (no cluster layout here)
    dflt = ix.autotune(None, 10, b, t, reps=0)
    assert dflt["slabs_per_range"] == 15 and dflt["slabs_per_range"] * dflt["n_ranges"] >= info["n_slabs"]
    _check(ix, oix, data, queries, 10, b, t)


def test_big_index_refuses_cluster_paths(big):
    data, queries, oix, ix = big
    with pytest.raises(TacoError) as err:
        ix.set_codes_fallback(False)
    assert err.value.code == -5
    q = torch.from_numpy(queries).cuda()
    ids = torch.empty((len(queries), 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((len(queries), 10), dtype=torch.float32, device="cuda")
    with pytest.raises(TacoError) as err:
        ix.search_noalloc(q, ids, dists, 10, 1000, 100)
    assert err.value.code == -5


def test_cluster_layout_fits_shared_memory():
    """89 slabs (2.9M points): 8 CTAs of 12 slabs would need more shared memory than a CTA
    can opt into, so the layout takes 15 CTAs of 6 slabs; queries whose threshold falls
    below 2 are answered by the cluster kernel in that layout and match the oracle."""
    rng = np.random.default_rng(321)
    n, d = 2_900_000, 16
    centres = rng.uniform(0, 100, size=(256, d)).astype(np.float32)
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, 1 << 20):
        m = min(n, a + (1 << 20)) - a
        data[a:a + m] = centres[rng.integers(0, 256, m)] + 3 * rng.standard_normal((m, d), dtype=np.float32)
    queries = (centres[rng.integers(0, 256, 5)] + 3 * rng.standard_normal((5, d))).astype(np.float32)
    ix = TacoIndex.build(data, 2, 8, 32, kmeans_iters=4, seed=7, keep_bf16=True)
    try:
        info = ix.info()
        assert info["n_slabs"] == 89 and 8 < info["cluster_size"] <= 16
        ex = ix.export()
        oix = O.index_from_parts(ex["o_bar"], ex["B"], ex["centroids"], ex["codes"], 2, 8, 32)
        # a target far above the ids with SC >= 2: threshold 1, every query flagged
        dbg = _check(ix, oix, data, queries, 10, budget_from_alpha(0.001, n), target_from_beta(0.01, n))
        assert np.all(dbg["last_collision"] <= 1)
    finally:
        ix.close()

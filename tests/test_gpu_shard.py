"""Id-range shards of one index through the C ABI (taco_shard_count / taco_shard_select), run
in one process on one device with the host combine of paper_2603_24919_gb300.sharding.

With FP32 rows the merged result of S shards is the one-index result, ids and distances
bit for bit (the same candidates, the same distance arithmetic; flagged queries take the
codes fallback in both): checked for S = 1 .. the index's ranges, at budgets that keep every
query above level 2, at targets that take queries to level 1 or 0 (the codes fallback over
each shard's ids), with per-query k and budgets, and with 3-bit and 4-bit counters. The shards' level counts sum to the one-index histogram of
the oracle (Def. 6), and BF16 rows (each shard re-ranks its own shortlist exactly) return
exact FP32 distances and at least the one-index recall."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import budget_from_alpha, target_from_beta

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoError, TacoIndex, build_lib, sharding  # noqa: E402

build_lib.build()


@pytest.fixture(scope="module")
def index():
    rng = np.random.default_rng(71)
    n, d = 400_003, 32
    centres = rng.uniform(0, 60, size=(200, d))
    data = (centres[rng.integers(0, 200, n)] + 5 * rng.standard_normal((n, d))).astype(np.float32)
    queries = (centres[rng.integers(0, 200, 24)] + 5 * rng.standard_normal((24, d))).astype(np.float32)
    oix = O.create_index(data, 4, 8, 32, kmeans_iters=6, seed=9)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              4, 8, 32, keep_bf16=True)
    ix.set_count_layout(slabs_per_range=2)   # 13 slabs: 7 ranges, so up to 7 shards
    # flagged queries take the codes fallback in the one-index search too (a shard always
    # does), so that both compute every candidate's distance in the same kernel
    ix.set_codes_fallback(True)
    yield data, queries, oix, ix
    ix.close()


def _one(ix, q, **kw):
    ids, d = ix.search(q, **kw)
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("alpha,beta", [(0.02, 0.003), (0.005, 0.2), (0.0005, 0.9)])
def test_fp32_shards_equal_one_index(index, alpha, beta):
    data, queries, oix, ix = index
    q = torch.from_numpy(queries).cuda()
    n = oix.n
    kw = dict(k=10, budget=budget_from_alpha(alpha, n), rerank_target=target_from_beta(beta, n))
    ref_ids, ref_d = _one(ix, q, **kw)
    for S in (1, 2, 3, 7):
        ids, d = ix.search_sharded(q, n_shards=S, **kw)
        np.testing.assert_array_equal(ids, ref_ids, err_msg=f"S={S}")
        np.testing.assert_array_equal(d, ref_d, err_msg=f"S={S}")
    assert ix.device_status() == 0


def test_shard_counts_sum_to_the_one_index_histogram(index):
    data, queries, oix, ix = index
    n = oix.n
    b, t = budget_from_alpha(0.02, n), target_from_beta(0.003, n)
    hists = []
    handles = []
    for s in range(3):
        h, hist = ix.shard_count(s, 3, queries[:6], 10, b, t)
        handles.append(h)
        hists.append(hist)
    for h in handles:
        h.close()
    g = sharding.reduce_counts(hists)
    for j in range(6):
        tr = O.search_one(oix, data, queries[j], 10, b, t)
        level = np.cumsum(tr.collision_num[::-1])[::-1]          # ids with SC >= j
        assert g[j, 0] == n
        np.testing.assert_array_equal(g[j, 1:], level[1:])


def test_per_query_parameters_and_counter_widths(index):
    data, queries, oix, ix = index
    q = torch.from_numpy(queries).cuda()
    n = oix.n
    rng = np.random.default_rng(5)
    pq = [dict(k=int(rng.choice([1, 10, 40])), budget=budget_from_alpha(float(rng.choice([0.002, 0.02])), n),
               rerank_target=target_from_beta(float(rng.choice([0.001, 0.3])), n)) for _ in range(len(queries))]
    for spc in (2, 13):   # 4-bit counters, 7 ranges; 3-bit counters (13 slabs), 1 range
        ix.set_count_layout(slabs_per_range=spc)
        try:
            ref_ids, ref_d = _one(ix, q, k=10, budget=1, rerank_target=0, per_query=pq, k_stride=40)
            S = 3 if spc == 2 else 1
            ids, d = ix.search_sharded(q, 10, 1, 0, S, per_query=pq, k_stride=40)
            np.testing.assert_array_equal(ids, ref_ids)
            np.testing.assert_array_equal(d, ref_d)
        finally:
            ix.set_count_layout(slabs_per_range=2)


def test_bf16_shards_keep_exact_distances(index):
    data, queries, oix, ix = index
    q = torch.from_numpy(queries).cuda()
    n = oix.n
    kw = dict(k=10, budget=budget_from_alpha(0.02, n), rerank_target=target_from_beta(0.003, n),
              precision="bf16", shortlist_mult=1)
    one_ids, _ = _one(ix, q, **kw)
    ids, d = ix.search_sharded(q, n_shards=4, **kw)
    truth = O.brute_force_knn(data, queries, 10)[0]
    rec = lambda r: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(r, truth)])
    assert rec(ids) >= rec(one_ids) - 1e-9
    exact = np.sqrt(((data[ids].astype(np.float64) - queries[:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(d, exact, rtol=1e-5)


def test_shard_arguments_are_checked(index):
    data, queries, oix, ix = index
    for s, S in ((0, 0), (3, 3), (0, 8), (-1, 2)):
        with pytest.raises(TacoError) as err:
            ix.shard_count(s, S, queries[:2], 10, 100, 10)
        assert err.value.code == -1

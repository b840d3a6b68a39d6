"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same index.

The index is built by the oracle (Alg. 1-3 in FP64) and imported into the library with
taco_index_create, so probed cells, SC-scores, Alg. 5 thresholds and results depend only
on query-time arithmetic. Inputs are seeded synthetic workloads (synth/)."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import budget_from_alpha, make_workload, target_from_beta
from tests.parity_util import ParityReport, check_exclusions, compare_query, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoIndex, build_lib  # noqa: E402

build_lib.build()


def _import(oix, data, keep_bf16=True):
    return TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids,
                                oix.codes.astype(np.uint16), oix.n_subspaces, oix.sub_dim,
                                oix.sqrt_k, keep_bf16=keep_bf16)


def _run(ix, oix, data, queries, k, budget, target, rule="literal", per_query=None,
         precision="fp32", want_sc=True):
    q = torch.from_numpy(queries).cuda()
    dbg = ix.search_debug(q, k, budget, target, select_rule=rule, per_query=per_query,
                          precision=precision, want_sc=want_sc)
    torch.cuda.synchronize()
    return to_numpy(dbg)


def _check_all(oix, data, queries, gpu, k, budget, target, name, rule="literal"):
    rep = ParityReport()
    for j, q in enumerate(queries):
        t = O.search_one(oix, data, q, k, budget, target, rule)
        compare_query(rep, t, gpu, j, k, oix.n)
    return check_exclusions(rep, name)


# ------------------------------------------------------------------ tiny workload (20k x 128)
@pytest.fixture(scope="module")
def tiny():
    w, data, queries = make_workload("tiny20k")
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1)
    ix = _import(oix, data)
    yield w, data, queries, oix, ix
    ix.close()


def test_tiny_parity_all_intermediates(tiny):
    w, data, queries, oix, ix = tiny
    gpu = _run(ix, oix, data, queries, w.k, w.budget, w.rerank_target)
    # transformed query agrees with the FP64 transform
    qt = O.transform(queries, oix.o_bar, oix.B)
    scale = np.abs(qt).max()
    assert np.abs(gpu["query_t"] - qt).max() <= 1e-5 * scale
    _check_all(oix, data, queries, gpu, w.k, w.budget, w.rerank_target, "tiny all intermediates")


@pytest.mark.parametrize("rule", ["literal", "prose"])
@pytest.mark.parametrize("alpha,beta", [(0.01, 0.002), (0.05, 0.01), (0.1, 0.05), (0.5, 0.4)])
def test_tiny_parity_budget_grid(tiny, rule, alpha, beta):
    w, data, queries, oix, ix = tiny
    b, t = budget_from_alpha(alpha, oix.n), target_from_beta(beta, oix.n)
    gpu = _run(ix, oix, data, queries[:40], 10, b, t, rule=rule)
    rep = ParityReport()
    big = 0
    for j, q in enumerate(queries[:40]):
        tr = O.search_one(oix, data, q, 10, b, t, rule)
        big += tr.n_candidates > 4096
        compare_query(rep, tr, gpu, j, 10, oix.n)
    check_exclusions(rep, f"tiny grid {rule} alpha={alpha} beta={beta}")
    if alpha == 0.5:
        assert big > 0   # exercises the path for more candidates than one buffer holds


@pytest.mark.parametrize("k", [1, 33, 100, 300])
def test_tiny_parity_k(tiny, k):
    w, data, queries, oix, ix = tiny
    gpu = _run(ix, oix, data, queries[:20], k, w.budget, 2000, want_sc=False)
    rep = ParityReport()
    for j, q in enumerate(queries[:20]):
        compare_query(rep, O.search_one(oix, data, q, k, w.budget, 2000), gpu, j, k, oix.n,
                      check_sc=False)
    check_exclusions(rep, f"tiny k={k}")


def test_full_budget_is_exact_knn(tiny):
    """budget > n probes every cell, every SC = N_s, C = all points: exact k-NN."""
    w, data, queries, oix, ix = tiny
    q = torch.from_numpy(queries[:30]).cuda()
    ids, dists = ix.search(q, 10, oix.n + 1, 5)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    t_ids, t_d = O.brute_force_knn(data, queries[:30], 11)
    for j in range(30):
        margin = (t_d[j, 10] ** 2 - t_d[j, 9] ** 2) / t_d[j, 10] ** 2
        assert np.allclose(dists[j], t_d[j, :10], rtol=1e-5)
        if margin >= 1e-5:
            assert set(ids[j]) == set(t_ids[j, :10])


def test_everything_selected_when_target_is_huge(tiny):
    """R >= 2n: Alg. 5 never stops (last_collision = -1), C = all n points."""
    w, data, queries, oix, ix = tiny
    gpu = _run(ix, oix, data, queries[:5], 10, w.budget, 10 * oix.n, want_sc=False)
    assert np.all(gpu["last_collision"] == -1)
    assert np.all(gpu["candidate_num"] == oix.n)
    t_ids, t_d = O.brute_force_knn(data, queries[:5], 10)
    assert np.allclose(gpu["dists"], t_d, rtol=1e-5)


def test_per_query_uneven_batch(tiny):
    """Per-query k, budget and target in one batch give each query's own answer."""
    w, data, queries, oix, ix = tiny
    rng = np.random.default_rng(0)
    pq = []
    for j in range(24):
        pq.append(dict(k=int(rng.choice([1, 10, 50, 100])),
                       budget=int(rng.choice([200, 1000, 3000])),
                       rerank_target=int(rng.choice([50, 200, 1000]))))
    kmax = max(p["k"] for p in pq)
    q = torch.from_numpy(queries[:24]).cuda()
    gpu = to_numpy(ix.search_debug(q, 10, 1000, 200, per_query=pq, k_stride=kmax))
    ids = gpu["ids"]
    rep = ParityReport()
    for j, p in enumerate(pq):
        t = O.search_one(oix, data, queries[j], p["k"], p["budget"], p["rerank_target"])
        compare_query(rep, t, gpu, j, p["k"], oix.n)
        assert np.all(ids[j, p["k"]:] == -1)
        # the same query alone gives the same answer
        a_ids, _ = ix.search(q[j:j + 1], p["k"], p["budget"], p["rerank_target"])
        assert np.array_equal(a_ids.cpu().numpy()[0], ids[j, :p["k"]])
    check_exclusions(rep, "tiny uneven batch")


def test_per_query_uneven_bf16_batch_equals_alone(tiny):
    """BF16 rows with per-query k and shortlist: each query's shortlist is its own, so its
    answer in a mixed batch equals its answer alone."""
    w, data, queries, oix, ix = tiny
    rng = np.random.default_rng(1)
    pq = [dict(k=int(rng.choice([1, 10, 50])), budget=int(rng.choice([200, 1000, 3000])),
               rerank_target=int(rng.choice([50, 200, 1000])), precision="bf16",
               shortlist_mult=int(rng.choice([1, 2, 4]))) for _ in range(24)]
    kmax = max(p["k"] for p in pq)
    q = torch.from_numpy(queries[:24]).cuda()
    ids, dists = ix.search(q, 10, 1000, 200, precision="bf16", per_query=pq, k_stride=kmax)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    for j, p in enumerate(pq):
        a_ids, a_d = ix.search(q[j:j + 1], p["k"], p["budget"], p["rerank_target"],
                               precision="bf16", shortlist_mult=p["shortlist_mult"], k_stride=kmax)
        assert np.array_equal(a_ids.cpu().numpy()[0], ids[j]), j
        ok = np.isfinite(dists[j])
        np.testing.assert_allclose(a_d.cpu().numpy()[0][ok], dists[j][ok], rtol=1e-5)


def test_host_pointers_match_device(tiny):
    w, data, queries, oix, ix = tiny
    ids_h, d_h = ix.search(queries[:50], 10, w.budget, w.rerank_target)      # numpy in/out
    ids_d, d_d = ix.search(torch.from_numpy(queries[:50]).cuda(), 10, w.budget, w.rerank_target)
    assert isinstance(ids_h, np.ndarray)
    assert np.array_equal(ids_h, ids_d.cpu().numpy())
    assert np.array_equal(d_h, d_d.cpu().numpy())


def test_empty_batch(tiny):
    w, data, queries, oix, ix = tiny
    ids, dists = ix.search(torch.zeros((0, 128), device="cuda"), 10, 100, 10)
    assert ids.shape == (0, 10)


def test_bad_arguments_raise(tiny):
    from paper_2603_24919_gb300 import TacoError
    w, data, queries, oix, ix = tiny
    q = torch.from_numpy(queries[:2]).cuda()
    with pytest.raises(TacoError):
        ix.search(q, 0, 100, 10)
    with pytest.raises(TacoError):
        ix.search(q, 10, 0, 10)
    with pytest.raises(TacoError):
        ix.search(q, 600, 100, 10, k_stride=600)


def test_save_load_roundtrip(tiny, tmp_path):
    w, data, queries, oix, ix = tiny
    path = str(tmp_path / "tiny.taco")
    ix.save(path)
    ix2 = TacoIndex.load(path)
    q = torch.from_numpy(queries[:20]).cuda()
    a = ix.search(q, 10, w.budget, w.rerank_target)
    b = ix2.search(q, 10, w.budget, w.rerank_target)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    ex = ix2.export()
    assert np.array_equal(ex["codes"], oix.codes.astype(np.uint16))
    assert np.allclose(ex["B"], oix.B)
    ix2.close()


# ------------------------------------------------------- ragged geometry: odd s, d, sqrt_k, n
@pytest.fixture(scope="module")
def ragged():
    rng = np.random.default_rng(77)
    n, d = 20003, 100
    centres = rng.uniform(0, 50, size=(40, d))
    data = (centres[rng.integers(0, 40, n)] + 4 * rng.standard_normal((n, d))).astype(np.float32)
    queries = (centres[rng.integers(0, 40, 30)] + 4 * rng.standard_normal((30, d))).astype(np.float32)
    oix = O.create_index(data, 4, 5, 7, kmeans_iters=8, seed=5)
    ix = _import(oix, data)
    yield data, queries, oix, ix
    ix.close()


@pytest.mark.parametrize("budget,target,k", [(1, 0, 5), (400, 100, 10), (2500, 600, 64),
                                             (20003, 20003, 10)])
def test_ragged_parity(ragged, budget, target, k):
    data, queries, oix, ix = ragged
    gpu = _run(ix, oix, data, queries, k, budget, target)
    _check_all(oix, data, queries, gpu, k, budget, target, f"ragged budget={budget} target={target} k={k}")


# --------------------------------------------------- several slabs: a cluster of CTAs per query
@pytest.fixture(scope="module")
def multislab():
    rng = np.random.default_rng(91)
    n, d = 300_001, 32
    centres = rng.uniform(0, 60, size=(200, d))
    data = (centres[rng.integers(0, 200, n)] + 5 * rng.standard_normal((n, d))).astype(np.float32)
    queries = (centres[rng.integers(0, 200, 24)] + 5 * rng.standard_normal((24, d))).astype(np.float32)
    oix = O.create_index(data, 4, 8, 32, kmeans_iters=6, seed=9)
    ix = _import(oix, data)
    yield data, queries, oix, ix
    ix.close()


@pytest.mark.parametrize("k", [10, 100])
def test_multislab_parity(multislab, k):
    data, queries, oix, ix = multislab
    info = ix.info()
    assert info["cluster_size"] > 1 and info["n_slabs"] == 10
    b, t = budget_from_alpha(0.05, oix.n), target_from_beta(0.01, oix.n)
    gpu = _run(ix, oix, data, queries, k, b, t)
    _check_all(oix, data, queries, gpu, k, b, t, f"multislab k={k}")


def test_multislab_all_points(multislab):
    data, queries, oix, ix = multislab
    gpu = _run(ix, oix, data, queries[:4], 10, 1000, 10 * oix.n, want_sc=False)
    assert np.all(gpu["candidate_num"] == oix.n)
    t_ids, t_d = O.brute_force_knn(data, queries[:4], 10)
    assert np.allclose(gpu["dists"], t_d, rtol=1e-5)


# ------------------------------------------------------------------------- BF16 re-rank form
def test_bf16_integer_data_matches_oracle():
    """On integer data in [0, 255] the BF16 copy is exact, so the BF16 form returns the
    oracle's results under the same acceptance rule as the FP32 form."""
    w, data, queries = make_workload("sift1m", n=40_000, nq=40)
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, 16, kmeans_iters=6, seed=2)
    ix = _import(oix, data)
    b, t = budget_from_alpha(0.05, oix.n), target_from_beta(0.01, oix.n)
    q = torch.from_numpy(queries).cuda()
    gpu = to_numpy(ix.search_debug(q, 10, b, t, precision="bf16", shortlist_mult=4))
    rep = ParityReport()
    for j in range(len(queries)):
        compare_query(rep, O.search_one(oix, data, queries[j], 10, b, t), gpu, j, 10, oix.n)
    check_exclusions(rep, "bf16 on integer data")
    ix.close()


def test_bf16_recall_close_to_fp32(tiny):
    w, data, queries, oix, ix = tiny
    q = torch.from_numpy(queries).cuda()
    t_ids, _ = O.brute_force_knn(data, queries, 10)
    f_ids, _ = ix.search(q, 10, w.budget, w.rerank_target)
    b_ids, b_d = ix.search(q, 10, w.budget, w.rerank_target, precision="bf16", shortlist_mult=4)
    rf = O.recall(f_ids.cpu().numpy(), t_ids, 10)
    rb = O.recall(b_ids.cpu().numpy(), t_ids, 10)
    assert rb >= rf - 0.01, (rb, rf)
    # returned distances are exact FP32 distances of the returned ids
    bi = b_ids.cpu().numpy()
    exact = np.sqrt(((data[bi].astype(np.float64) - queries[:, None, :]) ** 2).sum(-1))
    assert np.allclose(b_d.cpu().numpy(), exact, rtol=1e-5)


# ------------------------------------------------------------------ FP8 rows (precision form)
@pytest.fixture(scope="module")
def tiny_fp8(tiny):
    w, data, queries, oix, _ = tiny
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              oix.n_subspaces, oix.sub_dim, oix.sqrt_k, keep_bf16=False,
                              keep_fp8=True)
    yield ix
    ix.close()


def test_fp8_shortlist_covering_the_candidates_matches_oracle(tiny, tiny_fp8):
    """When the shortlist holds every candidate, the exact FP32 re-rank sees all of C, so the
    FP8 form returns the oracle's result under the FP32 acceptance rule."""
    w, data, queries, oix, _ = tiny
    ix = tiny_fp8
    info = ix.info()
    assert info["has_fp8"] == 1 and info["fp8_pitch"] % 16 == 0 and info["has_bf16"] == 0
    b, t = w.budget, 100
    q = torch.from_numpy(queries).cuda()
    gpu = to_numpy(ix.search_debug(q, 10, b, t, precision="fp8", shortlist_mult=51))   # 510
    rep = ParityReport()
    used = 0
    for j in range(len(queries)):
        tr = O.search_one(oix, data, queries[j], 10, b, t)
        covered = tr.candidate_num <= 510   # the shortlist holds all of C
        used += covered
        compare_query(rep, tr, gpu, j, 10, oix.n, check_topk=covered)
    check_exclusions(rep, "fp8 shortlist covering C")
    assert used >= len(queries) // 2, used


def test_fp8_recall_close_to_fp32(tiny, tiny_fp8):
    """FP8-e4m3 rows with per-16-dimension scales and an exact FP32 re-rank of a 4k shortlist
    lose at most 0.02 of recall@10 against the FP32 form; distances are exact FP32 ones."""
    w, data, queries, oix, ix32 = tiny
    q = torch.from_numpy(queries).cuda()
    t_ids, _ = O.brute_force_knn(data, queries, 10)
    f_ids, _ = ix32.search(q, 10, w.budget, w.rerank_target)
    e_ids, e_d = tiny_fp8.search(q, 10, w.budget, w.rerank_target, precision="fp8",
                                 shortlist_mult=4)
    rf = O.recall(f_ids.cpu().numpy(), t_ids, 10)
    re = O.recall(e_ids.cpu().numpy(), t_ids, 10)
    assert re >= rf - 0.02, (re, rf)
    ei = e_ids.cpu().numpy()
    ok = ei >= 0
    exact = np.sqrt(((data[np.where(ok, ei, 0)].astype(np.float64) - queries[:, None, :]) ** 2).sum(-1))
    assert np.allclose(e_d.cpu().numpy()[ok], exact[ok], rtol=1e-5)


def test_fp8_outlier_queries_stay_finite(tiny, tiny_fp8):
    """Queries far outside the points' range (coordinates up to 10x theirs): the FP8 pass
    clamps their half-precision coordinates at 4x the block's largest point coordinate, so
    every candidate distance stays finite; the FP32 shortlist re-rank returns exact distances
    and the same results as the FP32 form when the shortlist covers the candidates."""
    w, data, queries, oix, ix32 = tiny
    centre = data.mean(0)
    far = (centre + 10.0 * (queries - centre)).astype(np.float32)
    q = torch.from_numpy(far).cuda()
    f_ids, f_d = ix32.search(q, 10, w.budget, w.rerank_target)
    e_ids, e_d = tiny_fp8.search(q, 10, w.budget, w.rerank_target, precision="fp8", shortlist_mult=50)
    ei, ed = e_ids.cpu().numpy(), e_d.cpu().numpy()
    assert (ei >= 0).all() and np.isfinite(ed).all()
    exact = np.sqrt(((data[ei].astype(np.float64) - far[:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(ed, exact, rtol=1e-5)
    cand = tiny_fp8.search_debug(q, 10, w.budget, w.rerank_target, want_sc=False)["candidate_num"].cpu().numpy()
    cover = cand <= 500   # (the two forms sum a row's FP32 distance over different lanes:
    assert cover.any()    # compare the distances, which are equal up to that order)
    np.testing.assert_allclose(ed[cover], f_d.cpu().numpy()[cover], rtol=1e-6)


def test_fp8_needs_fp8_rows(tiny):
    w, data, queries, oix, ix = tiny   # built with BF16 rows only
    q = torch.from_numpy(queries[:4]).cuda()
    with pytest.raises(Exception) as err:
        ix.search(q, 10, w.budget, w.rerank_target, precision="fp8")
    assert "FP8" in str(err.value)

"""Parity at full size: the 1M x 128 integer-GMM workload with its 10,000-query batch, run
through taco_search_batch in one call at the operating point the benchmark times on it
(alpha = 0.01, beta = 0.001; FP32 with shortlist 4k, BF16 with shortlist k), in the counting
layout of 31 slabs of 2^15 ids, 12 per id range (3 ranges), 16 warps and 8 chunk loads in
flight per lane.

The index is built by the library (Alg. 1-3 on the GPU) and exported; the FP64 oracle
answers sampled queries one by one on that same index (its transform, centroids and cell
codes), under the acceptance rule of tests/parity_util.py: for 256 queries the probed cells
of every subspace (settled by the row-merge walk, the kernel the search path runs),
retrieved_num, collision_num, last_collision, candidate_num and the top k; for 16 of them the
SC-score of every point as well. Properties that hold at any size are checked on the whole
batch: ids valid and distinct per query, distances ascending and equal to the exact
distances of the returned ids, and agreement with the single-pass path of
taco_search_batch_noalloc."""
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

ALPHA, BETA, K = 0.01, 0.001, 10
FORMS = [("fp32", 4), ("bf16", 1)]
LAYOUT = dict(slabs_per_range=12, count_warps=16, walk_unroll=8)
SAMPLE = np.linspace(0, 9999, 256).astype(np.int64)
SC_SAMPLE = SAMPLE[::16]


@pytest.fixture(scope="module")
def full():
    w, data, queries = make_workload("sift1m")
    assert data.shape == (1_000_000, 128) and queries.shape == (10_000, 128)
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1,
                         keep_bf16=True)
    ix.set_count_layout(**LAYOUT)
    parts = ix.export()
    oix = O.index_from_parts(parts["o_bar"], parts["B"], parts["centroids"], parts["codes"],
                             w.n_subspaces, w.sub_dim, w.sqrt_k)
    q = torch.from_numpy(queries).cuda()
    b, t = budget_from_alpha(ALPHA, w.n), target_from_beta(BETA, w.n)
    results = {}
    for prec, mult in FORMS:
        ids, dists = ix.search(q, K, b, t, precision=prec, shortlist_mult=mult)
        torch.cuda.synchronize()
        results[prec] = (ids, dists)
    yield w, data, queries, q, ix, oix, b, t, results
    ix.close()


def _debug(ix, q, b, t, want_sc, **form):
    """search_debug of a sub-batch with the probe kernels' launches counted."""
    ix.profile_read(reset=True)
    ix.profile(True)
    dbg = ix.search_debug(q, K, b, t, want_sc=want_sc, **form)
    torch.cuda.synchronize()
    ix.profile(False)
    kt = ix.profile_read(reset=True)
    return to_numpy(dbg), kt


@pytest.mark.parametrize("prec,mult", FORMS)
def test_full_size_intermediates_match_oracle(full, prec, mult):
    """Probed cells (row-merge walk), retrieved_num, Alg. 5 counts and threshold, |C| and the
    top k of 256 queries equal the oracle's at the benchmark's layout and operating point."""
    w, data, queries, q, ix, oix, b, t, results = full
    info = ix.info()
    assert info["n_slabs"] == 31
    sel = torch.from_numpy(SAMPLE).cuda()
    dbg, kt = _debug(ix, q[sel], b, t, False, precision=prec, shortlist_mult=mult)
    # the walk ran (two probe launches: the walk and the histogram kernel for what it flags)
    assert kt["probe_cells"]["launches"] == 2, kt["probe_cells"]
    rep = ParityReport()
    for j, qi in enumerate(SAMPLE):
        tr = O.search_one(oix, data, queries[qi], K, b, t)
        compare_query(rep, tr, dbg, j, K, oix.n, check_sc=False)
    check_exclusions(rep, f"1M x 128 {prec} 256 queries")
    # the debug run returns what the timed search returned for these queries
    ids, dists = (x[sel].cpu().numpy() for x in results[prec])
    assert np.array_equal(dbg["ids"], ids)
    assert np.array_equal(dbg["dists"], dists)


def test_full_size_sc_scores_match_oracle(full):
    """The SC-score of every one of the 1M points (Def. 6) for 16 queries."""
    w, data, queries, q, ix, oix, b, t, results = full
    sel = torch.from_numpy(SC_SAMPLE).cuda()
    dbg, _ = _debug(ix, q[sel], b, t, True)
    rep = ParityReport()
    for j, qi in enumerate(SC_SAMPLE):
        tr = O.search_one(oix, data, queries[qi], K, b, t)
        compare_query(rep, tr, dbg, j, K, oix.n, check_sc=True)
    check_exclusions(rep, "1M x 128 SC of every point, 16 queries")


@pytest.mark.parametrize("prec", [f[0] for f in FORMS])
def test_full_batch_properties(full, prec):
    w, data, queries, q, ix, oix, b, t, results = full
    ids, dists = results[prec]
    assert bool((ids >= 0).all()) and bool((ids < w.n).all())
    srt, _ = ids.sort(dim=1)
    assert not bool((srt[:, 1:] == srt[:, :-1]).any()), "duplicate id in a result row"
    assert bool((dists[:, 1:] >= dists[:, :-1]).all()), "distances not ascending"
    # returned distances are the exact distances of the returned ids (FP64 recomputation)
    rows = torch.arange(0, q.shape[0], 7, device=q.device)
    x = torch.from_numpy(data).cuda()[ids[rows]].double()
    exact = (x - q[rows, None, :].double()).pow(2).sum(-1).sqrt()
    assert torch.allclose(dists[rows].double(), exact, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("prec,mult", FORMS)
def test_full_batch_two_paths_agree(full, prec, mult):
    """The two-pass path (count lists, then select) and the single-pass cluster path
    return the same answers."""
    w, data, queries, q, ix, oix, b, t, results = full
    ids, dists = results[prec]
    n = 1600
    i1 = torch.empty((n, K), dtype=torch.int64, device=q.device)
    d1 = torch.empty((n, K), dtype=torch.float32, device=q.device)
    for s0 in range(0, n, 800):
        ix.search_noalloc(q[s0:s0 + 800], i1[s0:s0 + 800], d1[s0:s0 + 800], K, b, t,
                          precision=prec, shortlist_mult=mult)
    torch.cuda.synchronize()
    assert torch.equal(i1, ids[:n])
    assert torch.equal(d1, dists[:n])

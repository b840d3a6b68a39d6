"""Pins for the oracle's query side: Alg. 4 (probe), SC-scores (Def. 6), Alg. 5
(selection), the re-rank of Alg. 6, and end-to-end special cases. CPU only."""
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import taco_oracle as O
from synth import make_workload, budget_from_alpha, target_from_beta


# ----------------------------------------------------------------------------- Alg. 4
def _read_probe(golden_dir):
    vals, probes = {}, []
    for line in open(os.path.join(golden_dir, "alg4_probe_order.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("probe"):
            head, tail = line[len("probe"):].split(";")
            b, *cells = [int(t) for t in head.split()]
            probes.append((b, cells, int(tail)))
        else:
            k, *v = line.split()
            vals[k] = [float(t) for t in v]
    return vals, probes


def test_alg4_hand_example(golden_dir):
    vals, probes = _read_probe(golden_dir)
    d1, d2 = np.array(vals["d1"]), np.array(vals["d2"])
    sizes = np.array(vals["sizes"], dtype=np.int64)
    assert len(probes) == 9
    for budget, cells, num in probes:
        popped, got = O.scalable_dynamic_activation(d1, d2, sizes, budget)
        assert popped == cells and got == num, (budget, popped, got)
        kept, got2, _ = O.probe_by_definition(d1, d2, sizes, budget)
        assert list(kept) == cells and got2 == num
    # the full order
    kept, _, _ = O.probe_by_definition(d1, d2, sizes, 10 ** 9)
    assert list(kept) == [int(v) for v in vals["order"]]


@pytest.mark.parametrize("sk", [2, 3, 8, 16])
def test_alg4_heap_equals_sorted_prefix_random(sk):
    """The heap (Alg. 4) pops cells in ascending key order, so its output is the sorted
    prefix, including integer-valued distances with many ties and empty cells."""
    rng = np.random.default_rng(sk)
    for trial in range(40):
        if trial % 2:
            d1 = rng.integers(0, 4, sk).astype(float)
            d2 = rng.integers(0, 4, sk).astype(float)
        else:
            d1, d2 = rng.random(sk) * 10, rng.random(sk) * 10
        sizes = rng.integers(0, 6, sk * sk)
        total = int(sizes.sum())
        for budget in [1, 2, max(1, total // 3), total, total + 5]:
            popped, num = O.scalable_dynamic_activation(d1, d2, sizes, budget)
            kept, num2, _ = O.probe_by_definition(d1, d2, sizes, budget)
            assert popped == list(kept) and num == num2


def test_alg4_prefix_is_minimal():
    rng = np.random.default_rng(3)
    for _ in range(100):
        sk = 6
        d1, d2 = rng.random(sk), rng.random(sk)
        sizes = rng.integers(0, 9, sk * sk)
        budget = int(rng.integers(1, sizes.sum() + 1))
        kept, num, _ = O.probe_by_definition(d1, d2, sizes, budget)
        assert num == sizes[kept].sum()
        assert num >= budget
        assert num - sizes[kept[-1]] < budget
        # no un-kept cell has a smaller key than a kept one
        keys = (d1[:, None] + d2[None, :]).ravel()
        rest = np.setdiff1d(np.arange(sk * sk), kept)
        if rest.size:
            assert keys[kept].max() <= keys[rest].min()


def test_alg4_brute_force_over_orders_tiny():
    """Brute force: among all key-sorted orders of a 2x2 grid, the probed set is the
    smallest prefix reaching the budget."""
    d1, d2 = np.array([0.0, 2.0]), np.array([0.0, 1.0])   # keys 0, 1, 2, 3
    sizes = np.array([1, 2, 3, 4])
    for budget, want in [(1, [0]), (2, [0, 1]), (3, [0, 1]), (4, [0, 1, 2]), (7, [0, 1, 2, 3])]:
        kept, _, _ = O.probe_by_definition(d1, d2, sizes, budget)
        assert sorted(kept) == want


def test_probe_margin_reports_near_ties():
    d1, d2 = np.array([0.0, 1.0]), np.array([0.0, 1.0 + 1e-9])
    sizes = np.array([1, 1, 1, 1])
    _, _, m = O.probe_by_definition(d1, d2, sizes, 2)   # cut between keys 1 and 1+1e-9
    assert m < 1e-8
    _, _, m2 = O.probe_by_definition(np.array([0.0, 5.0]), np.array([0.0, 1.0]), sizes, 2)
    assert m2 == pytest.approx(1.0)


# ----------------------------------------------------------------------------- Alg. 5
def _read_select(golden_dir):
    out = []
    for line in open(os.path.join(golden_dir, "alg5_threshold.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b, c, d = line.split(";")
        _, ns, R = a.split()
        hist = [int(v) for v in b.split()]
        lit = [int(v) for v in c.split()[1:]]
        pro = [int(v) for v in d.split()[1:]]
        out.append((int(ns), int(R), hist, lit, pro))
    return out


def _sc_from_hist(hist):
    return np.repeat(np.arange(len(hist)), hist)


def test_alg5_hand_examples(golden_dir):
    cases = _read_select(golden_dir)
    assert len(cases) == 5
    for ns, R, hist, lit, pro in cases:
        sc = _sc_from_hist(hist)
        for rule, want in [(O.SELECT_LITERAL, lit), (O.SELECT_PROSE, pro)]:
            C, num, last, h = O.candidate_selection(sc, ns, R, rule)
            assert [last, num] == want, (rule, hist, R)
            assert list(h) == hist
            assert len(C) == num


def _closed_form(hist, R, rule):
    """Independent statement of Alg. 5's stopping level: the largest j whose test fails,
    where for the literal rule the test at j is  2*h[j] + sum_{j'>j} h[j'] <= R  and for
    the prose rule  sum_{j'>=j} h[j'] <= R;  -1 if no level fails."""
    ns = len(hist) - 1
    for j in range(ns, -1, -1):
        above = sum(hist[j + 1:])
        if rule == O.SELECT_LITERAL:
            ok = 2 * hist[j] + above <= R
        else:
            ok = hist[j] + above <= R
        if not ok:
            return j
    return -1


def test_alg5_random_against_closed_form():
    rng = np.random.default_rng(12)
    for _ in range(300):
        ns = int(rng.integers(1, 12))
        n = int(rng.integers(1, 400))
        sc = rng.integers(0, ns + 1, n) * (rng.random(n) < rng.random())
        R = int(rng.integers(0, n + 3))
        hist = np.bincount(sc, minlength=ns + 1).tolist()
        for rule in (O.SELECT_LITERAL, O.SELECT_PROSE):
            C, num, last, _ = O.candidate_selection(sc, ns, R, rule)
            assert last == _closed_form(hist, R, rule)
            assert np.array_equal(C, np.nonzero(sc >= last)[0])
            assert num == len(C)               # Alg. 5 returns candidate_num = |C|


# ----------------------------------------------------------------------------- re-rank
def test_rerank_matches_brute_force_on_candidates():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(300, 9))
    q = rng.normal(size=9)
    C = np.sort(rng.choice(300, 120, replace=False))
    ids, dists, _ = O.rerank(x, q, C, 10)
    d = cdist(q[None, :], x[C])[0]
    order = np.argsort(d, kind="stable")[:10]
    assert np.array_equal(ids, C[order])
    assert np.allclose(dists, d[order], rtol=1e-12)


def test_rerank_ties_by_id_and_padding():
    x = np.array([[1.0, 0], [0, 1.0], [-1.0, 0], [5.0, 5.0]])
    ids, dists, _ = O.rerank(x, np.zeros(2), np.array([2, 0, 1]), 5)
    assert ids.tolist() == [0, 1, 2, -1, -1]
    assert np.allclose(dists[:3], 1.0) and np.all(np.isinf(dists[3:]))


# ----------------------------------------------------------------------------- end to end
@pytest.fixture(scope="module")
def small_index():
    w, data, queries = make_workload("tiny20k", n=4000, nq=12)
    ix = O.create_index(data, w.n_subspaces, w.sub_dim, 8, kmeans_iters=6, seed=1)
    return w, data, queries, ix


def test_collision_counts_sum_to_probed_sizes(small_index):
    w, data, queries, ix = small_index
    budget = budget_from_alpha(0.05, ix.n)
    for q in queries[:6]:
        t = O.search_one(ix, data, q, 10, budget, target_from_beta(0.01, ix.n),
                         heap_check=True)
        assert t.sc.sum() == t.retrieved_num.sum()
        assert t.sc.min() >= 0 and t.sc.max() <= ix.n_subspaces
        assert np.all(t.retrieved_num >= budget)
        # per subspace: an id is counted once when its cell is probed
        manual = np.zeros(ix.n, int)
        for i in range(ix.n_subspaces):
            manual += np.isin(ix.codes[i], t.probed[i])
        assert np.array_equal(manual, t.sc)
        assert t.candidate_num == t.n_candidates == int((t.sc >= t.last_collision).sum())


def test_full_budget_reduces_to_exact_knn(small_index):
    """alpha = 1: every cell is probed, every SC = N_s, C = all points, and the result is
    the exact k-NN (Def. 2)."""
    w, data, queries, ix = small_index
    truth_ids, truth_d = O.brute_force_knn(data, queries, 10)
    ids, dists, traces = O.search(ix, data, queries, 10, ix.n, target_from_beta(0.01, ix.n))
    for t in traces:
        assert np.all(t.sc == ix.n_subspaces)
        assert t.last_collision == ix.n_subspaces and t.n_candidates == ix.n
    assert np.array_equal(ids, truth_ids)
    # library routine: exact distances with scipy
    d = cdist(queries.astype(np.float64), data.astype(np.float64))
    want = np.sort(d, axis=1)[:, :10]
    assert np.allclose(dists, want, rtol=1e-12)


def test_brute_force_knn_matches_scipy():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(700, 5))
    q = rng.normal(size=(4, 5))
    ids, d = O.brute_force_knn(x, q, 7, chunk=100)
    dd = cdist(q, x)
    assert np.array_equal(ids, np.argsort(dd, axis=1, kind="stable")[:, :7])
    assert np.allclose(d, np.sort(dd, axis=1)[:, :7])


def test_high_sc_points_are_near(small_index):
    """Qualitative Pareto behaviour (Section 2.2): true neighbours collide more."""
    w, data, queries, ix = small_index
    truth_ids, _ = O.brute_force_knn(data, queries[:5], 10)
    for q, tids in zip(queries[:5], truth_ids):
        t = O.search_one(ix, data, q, 10, budget_from_alpha(0.05, ix.n),
                         target_from_beta(0.01, ix.n))
        assert t.sc[tids].mean() > 2 * t.sc.mean()


def test_recall_and_mre_definitions():
    assert O.recall(np.array([[1, 2, 3]]), np.array([[3, 4, 1]]), 3) == pytest.approx(2 / 3)
    assert O.mean_relative_error(np.array([[2.0, 3.0]]), np.array([[1.0, 3.0]])) == \
        pytest.approx(0.5)

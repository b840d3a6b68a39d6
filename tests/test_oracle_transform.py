"""Pins for the oracle's build side: Alg. 1 (transform), Alg. 2 (allocation), Lemma 1,
Alg. 3 (k-means and IMI cells). CPU only."""
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import taco_oracle as O


def _read_alg2_cases(path):
    cases, cur = [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "case":
            cur = {"buckets": []}
            cases.append(cur)
        elif key == "lam":
            cur["lam"] = [float(v) for v in vals]
        elif key == "bucket":
            cur["buckets"].append([int(v) for v in vals])
        else:
            cur[key] = int(vals[0])
    return cases


def test_alg2_hand_examples(golden_dir):
    """Alg. 2 on hand-worked eigenvalue lists (tests/golden/alg2_allocation.txt)."""
    cases = _read_alg2_cases(os.path.join(golden_dir, "alg2_allocation.txt"))
    assert len(cases) == 4
    for c in cases:
        buckets, _ = O.eigensystem_allocation(np.array(c["lam"]), c["n_subspaces"],
                                              c["sub_dim"])
        assert buckets == c["buckets"], c


def test_alg2_every_bucket_full_and_top_eigenvalues_used():
    rng = np.random.default_rng(5)
    for _ in range(50):
        d = int(rng.integers(4, 40))
        ns = int(rng.integers(1, 6))
        s = int(rng.integers(1, d // ns + 1))
        lam = rng.exponential(size=d) + 1e-3
        buckets, order = O.eigensystem_allocation(lam, ns, s)
        assert all(len(b) == s for b in buckets)
        used = sorted(e for b in buckets for e in b)
        # exactly the N_s*s largest (stable order)
        assert used == sorted(int(e) for e in order[:ns * s])
        assert sorted(np.argsort(-lam, kind="stable")[:ns * s].tolist()) == used


def test_alg2_products_balanced_greedy_invariant():
    """Each step appends to a bucket whose product was minimal among non-full buckets."""
    rng = np.random.default_rng(6)
    lam = np.sort(rng.exponential(size=24))[::-1] + 0.5
    buckets, order = O.eigensystem_allocation(lam, 4, 6)
    scaled = lam / lam.min()
    # replay: position of each eigenvector in descending order
    rank = {int(e): r for r, e in enumerate(order)}
    events = sorted((rank[e], j) for j, b in enumerate(buckets) for e in b)
    logp = np.zeros(4)
    fill = np.zeros(4, int)
    for r, j in events:
        open_b = [b for b in range(4) if fill[b] < 6]
        assert logp[j] <= min(logp[b] for b in open_b) + 1e-12
        logp[j] += np.log(scaled[order[r]])
        fill[j] += 1


def test_mean_covariance_matches_textbook():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(500, 7)) * np.arange(1, 8) + 3.0
    mu, sig = O.mean_and_covariance(x)
    assert np.allclose(mu, np.mean(x, axis=0), atol=1e-12)
    assert np.allclose(sig, np.cov(x, rowvar=False, ddof=1), atol=1e-10)


def _aniso(n, d, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    return (rng.normal(size=(n, d)) * np.linspace(5, 0.5, d)) @ q.T + 2.0


def test_transform_orthonormal_and_decorrelating():
    """B^T B = I, and cov(B^T (o - o_bar)) = diag(allocated eigenvalues) (Alg. 1)."""
    x = _aniso(3000, 12, 2)
    mu, sig = O.mean_and_covariance(x)
    lam, xi = O.spectral_decomposition(sig)
    # eigen-equation residual
    assert np.abs(sig @ xi - xi * lam[None, :]).max() <= 1e-9 * lam.max()
    buckets, _ = O.eigensystem_allocation(lam, 3, 3)
    B = O.transform_matrix(xi, buckets)
    assert B.shape == (12, 9)
    assert np.abs(B.T @ B - np.eye(9)).max() < 1e-12
    T = O.transform(x, mu, B)
    assert np.abs(T.mean(axis=0)).max() < 1e-9
    cov_t = np.cov(T, rowvar=False, ddof=1)
    want = np.array([lam[e] for b in buckets for e in b])
    assert np.allclose(cov_t, np.diag(want), atol=1e-8 * lam.max())


def test_lemma1_distance_preservation():
    """Lemma 1: ||B^T(x-y)|| <= ||x-y||, with equality when N_s*s = d."""
    x = _aniso(400, 16, 3)
    mu, sig = O.mean_and_covariance(x)
    lam, xi = O.spectral_decomposition(sig)
    full = O.transform_matrix(xi, O.eigensystem_allocation(lam, 4, 4)[0])
    part = O.transform_matrix(xi, O.eigensystem_allocation(lam, 2, 5)[0])
    a, b = x[:50], x[50:100]
    d0 = np.linalg.norm(a - b, axis=1)
    df = np.linalg.norm(O.transform(a, mu, full) - O.transform(b, mu, full), axis=1)
    dp = np.linalg.norm(O.transform(a, mu, part) - O.transform(b, mu, part), axis=1)
    assert np.allclose(df, d0, rtol=1e-12)
    assert np.all(dp <= d0 * (1 + 1e-12))
    assert np.any(dp < d0 * 0.999)


def test_kmeans_recovers_separated_blobs():
    rng = np.random.default_rng(4)
    centres = np.array([[0, 0], [100, 0], [0, 100], [100, 100]], float)
    lab = rng.integers(0, 4, 2000)
    x = centres[lab] + rng.normal(size=(2000, 2))
    # seed chosen so that the initial points fall in four distinct blobs
    for seed in range(50):
        init = np.random.Generator(np.random.PCG64(seed)).permutation(2000)[:4]
        if len(set(lab[init])) == 4:
            break
    c, a = O.kmeans(x, 4, 10, seed)
    # each found cluster is one blob, and centroid = mean of its points
    for j in range(4):
        members = lab[a == j]
        assert len(set(members)) == 1
        assert np.allclose(c[j], x[a == j].mean(axis=0))


def test_kmeans_fixed_point_and_nearest_assignment():
    rng = np.random.default_rng(9)
    x = rng.normal(size=(3000, 3))
    c, a = O.kmeans(x, 8, 60, 1)
    dist = cdist(x, c, "sqeuclidean")
    assert np.array_equal(a, np.argmin(dist, axis=1))
    for j in range(8):
        if np.any(a == j):
            assert np.allclose(c[j], x[a == j].mean(axis=0), atol=1e-9)


def test_nearest_centroid_ties_go_to_lowest_id():
    c = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0]])
    x = np.array([[0.0, 0.0], [0.0, 0.5], [0.0, -3.0]])
    # x0 equidistant to all three -> 0; x1 closest to 2; x2 equidistant to 0 and 1 -> 0
    assert O.nearest_centroid(x, c).tolist() == [0, 2, 0]


def test_create_index_cells_partition_ids_in_order():
    rng = np.random.default_rng(11)
    x = rng.normal(size=(1500, 8)) * np.arange(1, 9)
    ix = O.create_index(x, n_subspaces=2, sub_dim=4, sqrt_k=4, kmeans_iters=5, seed=3)
    for i in range(2):
        ids = np.concatenate(ix.cells[i])
        assert np.array_equal(np.sort(ids), np.arange(1500))
        for cell, members in enumerate(ix.cells[i]):
            assert np.all(np.diff(members) > 0)
            assert np.all(ix.codes[i, members] == cell)
        # codes are the nearest half-centroids of the transformed points
        T = O.transform(x, ix.o_bar, ix.B)[:, 4 * i:4 * i + 4]
        r = np.argmin(cdist(T[:, :2], ix.centroids[i, :, :2], "sqeuclidean"), axis=1)
        c = np.argmin(cdist(T[:, 2:], ix.centroids[i, :, 2:], "sqeuclidean"), axis=1)
        assert np.array_equal(ix.codes[i], r * 4 + c)


def test_half_distances_hand_example(golden_dir):
    vals = {}
    for line in open(os.path.join(golden_dir, "half_distances.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            vals[k] = np.array([float(t) for t in v])
    B = vals["B"].reshape(4, 4)
    cent = vals["cent"].reshape(1, 2, 4)
    codes = np.zeros((1, 3), dtype=np.int64)
    ix = O.index_from_parts(vals["obar"], B, cent, codes, 1, 4, 2)
    qt = O.transform(vals["q"][None, :], ix.o_bar, ix.B)[0]
    assert np.array_equal(qt, vals["qt"])
    d1, d2 = O.half_distances(ix, qt, 0)
    assert np.array_equal(d1, vals["d1"])
    assert np.array_equal(d2, vals["d2"])


def test_half_split_odd_subspace():
    """Reading R4: with s = 5, half 1 has 2 columns and half 2 has 3."""
    assert O.half_dims(5) == (2, 3)
    assert O.half_dims(16) == (8, 8)

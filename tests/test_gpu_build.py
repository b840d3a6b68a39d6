"""The library's own index build (taco_build_index) checked against the FP64 oracle's
build by invariants: Alg. 1 (mean, covariance eigenvectors), Alg. 2 (allocation),
Alg. 3 (k-means fixed point, IMI cells), and search quality on the built index."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoIndex, build_lib  # noqa: E402

build_lib.build()


@pytest.fixture(scope="module")
def built():
    w, data, queries = make_workload("tiny20k")
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=4)
    ex = ix.export()
    yield w, data, queries, ix, ex
    ix.close()


def test_transform_matches_oracle_eigensystem(built):
    w, data, queries, ix, ex = built
    mu, sigma = O.mean_and_covariance(data)
    assert np.allclose(ex["o_bar"], mu, rtol=1e-10, atol=1e-9)
    B = ex["B"]
    assert np.abs(B.T @ B - np.eye(B.shape[1])).max() < 1e-10
    lam, xi = O.spectral_decomposition(sigma)
    lam_desc = np.sort(lam)[::-1]
    assert np.allclose(ex["eigvals"], lam_desc, rtol=1e-9, atol=1e-9 * lam_desc[0])
    # every column of B is an eigenvector of the oracle's covariance with the eigenvalue of
    # its allocation rank
    for c in range(B.shape[1]):
        v = B[:, c]
        lv = lam_desc[ex["alloc"][c]]
        assert np.linalg.norm(sigma @ v - lv * v) <= 1e-7 * lam_desc[0]


def test_allocation_matches_oracle(built):
    w, data, queries, ix, ex = built
    mu, sigma = O.mean_and_covariance(data)
    lam, _ = O.spectral_decomposition(sigma)
    buckets, order = O.eigensystem_allocation(lam, w.n_subspaces, w.sub_dim)
    rank = {int(e): r for r, e in enumerate(order)}
    lam_sorted = np.sort(lam)[::-1]
    gaps = np.diff(lam_sorted) / lam_sorted[0]
    if np.min(np.abs(gaps[:w.n_subspaces * w.sub_dim])) > 1e-9:
        want = [[rank[e] for e in b] for b in buckets]
        got = ex["alloc"].reshape(w.n_subspaces, w.sub_dim).tolist()
        assert got == want


def test_kmeans_codes_are_nearest_centroids(built):
    w, data, queries, ix, ex = built
    T = O.transform(data, ex["o_bar"], ex["B"])
    h1 = w.sub_dim // 2
    mismatch = 0
    for i in range(w.n_subspaces):
        Ti = T[:, i * w.sub_dim:(i + 1) * w.sub_dim]
        C = ex["centroids"][i]
        d1 = ((Ti[:, None, :h1] - C[None, :, :h1]) ** 2).sum(-1)
        d2 = ((Ti[:, None, h1:] - C[None, :, h1:]) ** 2).sum(-1)
        r = ex["codes"][i].astype(np.int64) // w.sqrt_k
        c = ex["codes"][i].astype(np.int64) % w.sqrt_k
        # the assigned centroid is nearest up to FP32 rounding of the GPU distances
        best1, best2 = d1.min(1), d2.min(1)
        got1, got2 = d1[np.arange(len(r)), r], d2[np.arange(len(c)), c]
        mismatch += np.sum(got1 > best1 * (1 + 1e-4) + 1e-6) + np.sum(got2 > best2 * (1 + 1e-4) + 1e-6)
    assert mismatch == 0


@pytest.mark.parametrize("target", [200, 400])
def test_built_index_recall(built, target):
    """Recall of the library-built index is that of the oracle-built index (same method,
    different k-means seeds) within a small margin."""
    w, data, queries, ix, ex = built
    t_ids, _ = O.brute_force_knn(data, queries, 10)
    ids, _ = ix.search(torch.from_numpy(queries).cuda(), 10, w.budget, target)
    rec = O.recall(ids.cpu().numpy(), t_ids, 10)
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1)
    o_ids, _, _ = O.search(oix, data, queries, 10, w.budget, target)
    rec_o = O.recall(o_ids, t_ids, 10)
    assert rec >= rec_o - 0.05, (rec, rec_o)


def _host_lists(codes, n_slabs, K):
    """The cell lists as the index lays them out, built on the host from the codes: per
    subspace and cell the ids ascending (Alg. 3's IMI[cell].append(j) for j = 0..n-1), each
    list at a multiple of 4 and padded with 0xffffffff, and the slab table of absolute
    positions of the first id >= t * 2^15 (t = n_slabs: the list's end)."""
    ns, n = codes.shape
    sizes = np.zeros((ns, K), dtype=np.int64)
    split = np.zeros((ns, K, n_slabs + 1), dtype=np.int64)
    ids, pos = [], 0
    bounds = np.minimum(np.arange(n_slabs + 1, dtype=np.int64) << 15, n)
    for i in range(ns):
        order = np.argsort(codes[i], kind="stable")
        cuts = np.searchsorted(codes[i][order], np.arange(K + 1))
        for c in range(K):
            cell = order[cuts[c]:cuts[c + 1]]
            sizes[i, c] = len(cell)
            split[i, c] = pos + np.searchsorted(cell, bounds)
            ids.append(cell)
            pad = (-len(cell)) % 4
            ids.append(np.full(pad, 0xFFFFFFFF, dtype=np.int64))
            pos += len(cell) + pad
    return sizes, split, np.concatenate(ids)


@pytest.mark.parametrize("n,sk", [(20_000, 16), (100_003, 7), (300_001, 32)])
def test_device_cell_lists_equal_host_construction(n, sk):
    """The cell lists and slab table built on the device (a stable counting sort by code, one
    2^15-id slab at a time) equal the host construction from the exported codes, including a
    ragged last slab, odd sqrt_k and empty cells; the build reports its two phase times."""
    w, data, _ = make_workload("tiny20k", n=n, nq=1)
    ix = TacoIndex.build(data[:, :32], 4, 8, sk, kmeans_iters=4, seed=7)
    inf = ix.info()
    got = ix.lists()
    sizes, split, ids = _host_lists(ix.export()["codes"].astype(np.int64), inf["n_slabs"], sk * sk)
    assert inf["n_ids"] == len(ids)
    np.testing.assert_array_equal(got["sizes"], sizes)
    np.testing.assert_array_equal(got["split"], split)
    np.testing.assert_array_equal(got["ids"].astype(np.int64), ids)
    assert inf["build_ms_transform"] > 0 and inf["build_ms_index"] > 0
    ix.close()

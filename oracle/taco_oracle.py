"""FP64 CPU oracle for TaCo's index and query path (TEST INFRASTRUCTURE ONLY).

This module is the plain, slow reference that the GPU library is checked against. Only
the tests, the smoke check and the CPU-baseline leg of the benchmark may import it; the
library never calls it and never falls back to it.

Every function follows one step of the paper (arXiv 2603.24919, "TaCo: Data-adaptive and
Query-aware Subspace Collision for High-dimensional ANNS"), in the paper's order and
notation, in FP64. Library primitives serve as single steps (numpy.linalg.eigh for the
spectral decomposition, argsort/lexsort for sorting, bincount for counting). The oracle
shares no code with the CUDA path.

Readings where the paper is ambiguous (each is also listed in the design notes):
  R1  Alg. 6 step 1 says "transform q with the eigenvalues": the transform is the one of
      Alg. 1, r = B^T (q - o_bar), with B the allocated eigenvectors.
  R2  Alg. 2 step 3 scales the eigenvalues so that all are >= 1: multiply all d of them
      by 1 / lambda_min, with lambda_min floored at 1e-12 * lambda_max. Products are kept
      as sums of logarithms (same argmin, no overflow).
  R3  Ties: the eigenvalue sort is stable by original index; argmin over buckets picks
      the lowest bucket index.
  R4  A subspace splits into half 1 = its first floor(s/2) columns and half 2 = the rest
      (Alg. 3 step 6, Alg. 6 step 4). Columns of a subspace keep allocation order.
  R5  Per-half distances are squared Euclidean; a cell's key is d1[r] + d2[c], the squared
      distance to the product centroid (Alg. 4).
  R6  Cells are ordered by the total key (sum, r, c); r is the half-1 centroid id and c the
      half-2 centroid id (cell id = r * sqrtK + c). Argsorts of the per-half distances
      are stable, so equal distances keep centroid-id order.
  R7  Alg. 4 stops when every cell has been popped, even if the budget is not met.
  R8  The budget alpha*n enters as the integer B = ceil(alpha*n) >= 1; the re-rank test
      collision_num[j] <= beta*n - candidate_num enters as the integer R = floor(beta*n).
  R9  Alg. 5: the literal pseudocode (test after adding level j) is the default rule; the
      prose ("until the accumulated number exceeds beta*n") is rule "prose". Both keep
      the breaking level whole; a loop that never breaks leaves last_collision = -1.
  R10 The re-rank uses exact distances in the original d-dimensional space, orders by
      (distance, id), returns min(k, |C|) results padded with id -1 / distance +inf,
      and reports non-squared Euclidean distances.
  R11 K-means (Alg. 3): t Lloyd iterations from sqrtK distinct seeded data points, then a
      final assignment to the returned centroids; an empty cluster keeps its previous
      centroid; equal distances go to the lowest centroid id.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np

SELECT_LITERAL = "literal"
SELECT_PROSE = "prose"


# --------------------------------------------------------------------------------------
# Alg. 1: Subspace-oriented Data Transformation
# --------------------------------------------------------------------------------------
def mean_and_covariance(data):
    """Alg. 1 steps 2-3: o_bar = (1/n) sum o_i; Sigma = 1/(n-1) sum (o_i-o_bar)(o_i-o_bar)^T."""
    x = np.asarray(data, dtype=np.float64)
    n = x.shape[0]
    o_bar = x.sum(axis=0) / n
    xc = x - o_bar
    sigma = (xc.T @ xc) / (n - 1)
    return o_bar, sigma


def spectral_decomposition(sigma):
    """Alg. 1 step 4: eigenvalues and eigenvectors of the symmetric covariance.

    Returns (lam, xi) with xi[:, i] the eigenvector of lam[i], in numpy's ascending order;
    Alg. 2 does its own descending reorder.
    """
    lam, xi = np.linalg.eigh(np.asarray(sigma, dtype=np.float64))
    return lam, xi


def eigensystem_allocation(lam, n_subspaces, sub_dim, scale_floor=1e-12):
    """Alg. 2: greedy allocation of the N_s*s largest eigenvectors to N_s buckets.

    Returns (buckets, order): buckets[j] lists indices into lam (original numbering) in the
    order they were appended; order is the descending stable permutation of lam.
    """
    lam = np.asarray(lam, dtype=np.float64)
    d = lam.shape[0]
    if n_subspaces * sub_dim > d:
        raise ValueError("N_s * s must not exceed d")
    # step 3 (reading R2): scale all eigenvalues so that the smallest is 1
    lam_max = float(lam.max())
    lam_min = max(float(lam.min()), scale_floor * lam_max)
    scaled = np.maximum(lam, lam_min) / lam_min
    # step 4: descending order, stable by original index (reading R3)
    order = np.argsort(-scaled, kind="stable")
    # steps 1-2: empty buckets, products p_j = 1 (log p_j = 0)
    buckets = [[] for _ in range(n_subspaces)]
    log_p = [0.0] * n_subspaces
    # steps 5-8
    for i in range(n_subspaces * sub_dim):
        best = -1
        for j in range(n_subspaces):
            if len(buckets[j]) < sub_dim and (best < 0 or log_p[j] < log_p[best]):
                best = j
        e = int(order[i])
        buckets[best].append(e)
        log_p[best] += float(np.log(scaled[e]))
    return buckets, order


def transform_matrix(xi, buckets):
    """B = [B_1 ... B_{N_s}]: bucket j's eigenvectors as columns, in allocation order."""
    cols = [xi[:, e] for bucket in buckets for e in bucket]
    return np.stack(cols, axis=1).astype(np.float64)


def transform(points, o_bar, B):
    """Alg. 1 steps 6-11: o' = concat_j B_j^T (o - o_bar) = B^T (o - o_bar)."""
    x = np.asarray(points, dtype=np.float64)
    return (x - o_bar[None, :]) @ B


# --------------------------------------------------------------------------------------
# Alg. 3: Create Index
# --------------------------------------------------------------------------------------
def half_dims(sub_dim):
    """Reading R4: half 1 has floor(s/2) columns, half 2 the remaining ones."""
    h1 = sub_dim // 2
    return h1, sub_dim - h1


def nearest_centroid(points, centroids, chunk=1 << 16):
    """Index of the nearest centroid (squared L2), ties to the lowest centroid id."""
    x = np.asarray(points, dtype=np.float64)
    c = np.asarray(centroids, dtype=np.float64)
    out = np.empty(x.shape[0], dtype=np.int64)
    cn = (c * c).sum(axis=1)
    for a in range(0, x.shape[0], chunk):
        xb = x[a:a + chunk]
        # ||x - c||^2 = ||x||^2 - 2 x.c + ||c||^2; the ||x||^2 term does not change argmin
        dist = cn[None, :] - 2.0 * (xb @ c.T)
        out[a:a + chunk] = np.argmin(dist, axis=1)  # first minimum = lowest id
    return out


def kmeans(points, n_centroids, iters, seed):
    """Lloyd's k-means as used by Alg. 3 steps 7-8 (reading R11)."""
    x = np.asarray(points, dtype=np.float64)
    n = x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    init = rng.permutation(n)[:n_centroids]
    centroids = x[init].copy()
    for _ in range(iters):
        assign = nearest_centroid(x, centroids)
        counts = np.bincount(assign, minlength=n_centroids)
        for j in range(x.shape[1]):
            sums = np.bincount(assign, weights=x[:, j], minlength=n_centroids)
            nz = counts > 0
            centroids[nz, j] = sums[nz] / counts[nz]
    assign = nearest_centroid(x, centroids)
    return centroids, assign


@dataclass
class OracleIndex:
    """Index of Alg. 3: transform, per-subspace product centroids and IMI cells."""
    n: int
    d: int
    n_subspaces: int
    sub_dim: int
    sqrt_k: int
    o_bar: np.ndarray          # [d] f64
    B: np.ndarray              # [d, N_s*s] f64
    eigvals: np.ndarray        # [d] f64, ascending as returned by eigh
    buckets: list              # Alg. 2 allocation (eigen indices)
    centroids: np.ndarray      # [N_s, sqrtK, s] f64: cols [:h1] half 1, [h1:] half 2
    codes: np.ndarray          # [N_s, n] int64, cell = r * sqrtK + c
    cells: list                # cells[i][cell] -> int64 array of ids, ascending

    @property
    def n_cells(self):
        return self.sqrt_k * self.sqrt_k

    def cell_sizes(self, i):
        """|IMI_i[cell]| for every cell of subspace i (computed once, then reused)."""
        cache = self.__dict__.setdefault("_sizes", {})
        if i not in cache:
            cache[i] = np.array([len(c) for c in self.cells[i]], dtype=np.int64)
        return cache[i]


def imi_cells(codes_i, n_cells):
    """Alg. 3 steps 10-12: IMI[cell].append(j) for j = 0..n-1 (ids ascending per cell)."""
    order = np.argsort(codes_i, kind="stable")
    bounds = np.searchsorted(codes_i[order], np.arange(n_cells + 1))
    return [order[bounds[c]:bounds[c + 1]].astype(np.int64) for c in range(n_cells)]


def create_index(data, n_subspaces, sub_dim, sqrt_k, kmeans_iters=20, seed=0):
    """Alg. 3 (with Alg. 1 and Alg. 2 as its step 1)."""
    x = np.asarray(data, dtype=np.float64)
    n, d = x.shape
    o_bar, sigma = mean_and_covariance(x)
    lam, xi = spectral_decomposition(sigma)
    buckets, _ = eigensystem_allocation(lam, n_subspaces, sub_dim)
    B = transform_matrix(xi, buckets)
    T = transform(x, o_bar, B)
    h1, h2 = half_dims(sub_dim)
    centroids = np.zeros((n_subspaces, sqrt_k, sub_dim))
    codes = np.zeros((n_subspaces, n), dtype=np.int64)
    cells = []
    for i in range(n_subspaces):
        Ti = T[:, i * sub_dim:(i + 1) * sub_dim]
        c1, a1 = kmeans(Ti[:, :h1], sqrt_k, kmeans_iters, seed * 7919 + 2 * i)
        c2, a2 = kmeans(Ti[:, h1:], sqrt_k, kmeans_iters, seed * 7919 + 2 * i + 1)
        centroids[i, :, :h1] = c1
        centroids[i, :, h1:] = c2
        codes[i] = a1 * sqrt_k + a2
        cells.append(imi_cells(codes[i], sqrt_k * sqrt_k))
    return OracleIndex(n, d, n_subspaces, sub_dim, sqrt_k, o_bar, B, lam, buckets,
                       centroids, codes, cells)


def index_from_parts(o_bar, B, centroids, codes, n_subspaces, sub_dim, sqrt_k):
    """An OracleIndex from given transform, centroids and cell codes."""
    codes = np.asarray(codes, dtype=np.int64)
    cells = [imi_cells(codes[i], sqrt_k * sqrt_k) for i in range(n_subspaces)]
    d = B.shape[0]
    return OracleIndex(codes.shape[1], d, n_subspaces, sub_dim, sqrt_k,
                       np.asarray(o_bar, np.float64), np.asarray(B, np.float64),
                       np.zeros(d), [], np.asarray(centroids, np.float64), codes, cells)


# --------------------------------------------------------------------------------------
# Alg. 6 steps 1-5: transform the query and compute per-half centroid distances
# --------------------------------------------------------------------------------------
def half_distances(index, q_t, i):
    """Alg. 6 steps 4-5 for subspace i: dists_1, dists_2 (squared L2, reading R5)."""
    h1, _ = half_dims(index.sub_dim)
    qi = q_t[i * index.sub_dim:(i + 1) * index.sub_dim]
    C = index.centroids[i]
    d1 = ((qi[None, :h1] - C[:, :h1]) ** 2).sum(axis=1)
    d2 = ((qi[None, h1:] - C[:, h1:]) ** 2).sum(axis=1)
    return d1, d2


# --------------------------------------------------------------------------------------
# Alg. 4: Scalable Dynamic Activation, and the order it realises
# --------------------------------------------------------------------------------------
def scalable_dynamic_activation(d1, d2, sizes, budget):
    """Alg. 4 with the heap ordered by the total key (sum, r, c) (reading R6).

    sizes[r * sqrtK + c] is |IMI[r, c]|. Returns the retrieved cells in pop order.
    """
    sk = len(d1)
    idx1 = np.argsort(d1, kind="stable")
    idx2 = np.argsort(d2, kind="stable")
    retrieved = []
    retrieved_num = 0
    active_idx = [0] * sk

    def entry(pos):
        r, c = int(idx1[pos]), int(idx2[active_idx[pos]])
        return (float(d1[r] + d2[c]), r, c, pos)

    heap = [entry(0)]
    while heap:  # reading R7: stop once every cell has been popped
        top = heap[0]
        pos = top[3]
        r, c = int(idx1[pos]), int(idx2[active_idx[pos]])
        retrieved.append(r * sk + c)
        retrieved_num += int(sizes[r * sk + c])
        if retrieved_num >= budget:
            break
        if active_idx[pos] == 0 and pos < sk - 1:
            heapq.heappush(heap, (float(d1[int(idx1[pos + 1])] + d2[int(idx2[0])]),
                                  int(idx1[pos + 1]), int(idx2[0]), pos + 1))
        heapq.heappop(heap)
        if active_idx[pos] < sk - 1:
            active_idx[pos] += 1
            heapq.heappush(heap, entry(pos))
    return retrieved, retrieved_num


def probe_by_definition(d1, d2, sizes, budget):
    """The set Alg. 4 returns, from its definition (Section 4.2): sort every cell by
    (d1[r] + d2[c], r, c) ascending and keep the shortest prefix whose sizes sum to at
    least the budget (all cells if they never do).

    Also returns the FP64 boundary margin: the relative key gap between the last kept
    cell and its two neighbours in this order (inf where a neighbour does not exist).
    """
    sk = len(d1)
    r = np.repeat(np.arange(sk), sk)
    c = np.tile(np.arange(sk), sk)
    keys = d1[r] + d2[c]
    order = np.lexsort((c, r, keys))
    cum = np.cumsum(np.asarray(sizes, dtype=np.int64)[order])
    hit = np.nonzero(cum >= budget)[0]
    m = int(hit[0]) + 1 if hit.size else len(order)
    kept = order[:m]
    k_last = keys[order[m - 1]]
    scale = max(abs(k_last), np.finfo(np.float64).tiny)
    below = (k_last - keys[order[m - 2]]) / scale if m >= 2 else np.inf
    above = (keys[order[m]] - k_last) / scale if m < len(order) else np.inf
    return kept, int(cum[m - 1]), float(min(below, above))


# --------------------------------------------------------------------------------------
# SC-score (Def. 6), Alg. 5 and the re-rank of Alg. 6
# --------------------------------------------------------------------------------------
def collision_counts(index, probed):
    """Alg. 6 step 7: SC[id] = number of subspaces whose retrieved cells hold id."""
    sc = np.zeros(index.n, dtype=np.int64)
    for i in range(index.n_subspaces):
        for cell in probed[i]:
            sc[index.cells[i][cell]] += 1  # ids within one cell are distinct
    return sc


def candidate_selection(sc, n_subspaces, rerank_target, rule=SELECT_LITERAL):
    """Alg. 5 (reading R9). Returns (C, candidate_num, last_collision, collision_num)."""
    collision_num = np.bincount(np.asarray(sc, dtype=np.int64),
                                minlength=n_subspaces + 1).astype(np.int64)
    last_collision = n_subspaces
    candidate_num = 0
    for j in range(n_subspaces, -1, -1):
        candidate_num += int(collision_num[j])
        if rule == SELECT_LITERAL:
            keep_going = collision_num[j] <= rerank_target - candidate_num
        elif rule == SELECT_PROSE:
            keep_going = candidate_num <= rerank_target
        else:
            raise ValueError(rule)
        if keep_going:
            last_collision -= 1
        else:
            break
    C = np.nonzero(np.asarray(sc) >= last_collision)[0].astype(np.int64)
    return C, candidate_num, last_collision, collision_num


def rerank(data, q, C, k):
    """Alg. 6 step 9 (reading R10): exact top-k of C by (distance, id)."""
    x = np.asarray(data, dtype=np.float64)
    qq = np.asarray(q, dtype=np.float64)
    C = np.asarray(C, dtype=np.int64)
    d2 = ((x[C] - qq[None, :]) ** 2).sum(axis=1)
    order = np.lexsort((C, d2))
    take = order[:k]
    ids = np.full(k, -1, dtype=np.int64)
    dists = np.full(k, np.inf)
    ids[:len(take)] = C[take]
    dists[:len(take)] = np.sqrt(d2[take])
    # boundary margin of the k-th result: relative gap to the first excluded candidate
    if len(order) > k and k > 0:
        a, b = d2[order[k - 1]], d2[order[k]]
        kth_margin = float((b - a) / max(b, np.finfo(np.float64).tiny))
    else:
        kth_margin = np.inf
    return ids, dists, kth_margin


@dataclass
class QueryTrace:
    probed: list            # per subspace: array of probed cell ids
    retrieved_num: np.ndarray
    probe_margin: np.ndarray
    sc: np.ndarray
    collision_num: np.ndarray
    last_collision: int
    candidate_num: int
    n_candidates: int
    ids: np.ndarray
    dists: np.ndarray
    kth_margin: float


def search_one(index, data, q, k, budget, rerank_target, rule=SELECT_LITERAL,
               heap_check=False):
    """Alg. 6 for one query, returning every intermediate result."""
    q_t = transform(np.asarray(q, np.float64)[None, :], index.o_bar, index.B)[0]
    probed, rnum, margin = [], [], []
    for i in range(index.n_subspaces):
        d1, d2 = half_distances(index, q_t, i)
        sizes = index.cell_sizes(i)
        kept, num, m = probe_by_definition(d1, d2, sizes, budget)
        if heap_check:
            popped, num_h = scalable_dynamic_activation(d1, d2, sizes, budget)
            if popped != list(kept) or num_h != num:
                raise AssertionError("Alg. 4 heap order differs from the sorted order")
        probed.append(np.asarray(kept, dtype=np.int64))
        rnum.append(num)
        margin.append(m)
    sc = collision_counts(index, probed)
    C, cand_num, last, hist = candidate_selection(sc, index.n_subspaces, rerank_target,
                                                  rule)
    ids, dists, kth = rerank(data, q, C, k)
    return QueryTrace(probed, np.array(rnum), np.array(margin), sc, hist, last,
                      cand_num, len(C), ids, dists, kth)


def search(index, data, queries, k, budget, rerank_target, rule=SELECT_LITERAL):
    """Alg. 6 over a batch: (ids [nq,k], dists [nq,k]) plus the per-query traces."""
    traces = [search_one(index, data, q, k, budget, rerank_target, rule) for q in queries]
    ids = np.stack([t.ids for t in traces])
    dists = np.stack([t.dists for t in traces])
    return ids, dists, traces


# --------------------------------------------------------------------------------------
# Exact k-NN (Def. 2) and the quality measures of Section 6.1
# --------------------------------------------------------------------------------------
def brute_force_knn(data, queries, k, chunk=4096):
    """Exact k-NN by FP64 brute force, ordered by (distance, id)."""
    x = np.asarray(data, dtype=np.float64)
    Q = np.asarray(queries, dtype=np.float64)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k))
    all_ids = np.arange(x.shape[0])
    for qi in range(nq):
        best_d, best_i = None, None
        for a in range(0, x.shape[0], chunk):
            d2 = ((x[a:a + chunk] - Q[qi][None, :]) ** 2).sum(axis=1)
            cand_i = all_ids[a:a + chunk]
            if best_d is not None:
                d2 = np.concatenate([best_d, d2])
                cand_i = np.concatenate([best_i, cand_i])
            o = np.lexsort((cand_i, d2))[:k]
            best_d, best_i = d2[o], cand_i[o]
        ids[qi] = best_i
        dists[qi] = np.sqrt(best_d)
    return ids, dists


def recall(result_ids, truth_ids, k):
    """Section 6.1: |R intersect R*| / k, averaged over queries."""
    hits = [len(set(map(int, r[:k])) & set(map(int, t[:k]))) for r, t in
            zip(result_ids, truth_ids)]
    return float(np.mean(hits)) / k


def mean_relative_error(result_dists, truth_dists):
    """Section 6.1: (1/k) sum_i (||q,o_i|| - ||q,o*_i||) / ||q,o*_i||, averaged."""
    r = np.asarray(result_dists, np.float64)
    t = np.asarray(truth_dists, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(t > 0, (r - t) / t, 0.0)
    return float(np.mean(rel))

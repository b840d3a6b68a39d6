"""Per-query parameters resident on the device (taco_params_create / taco_search_batch_params)
and the search path inside a captured CUDA graph.

- A prepared batch with per-query k, budgets and targets returns exactly what
  taco_search_batch returns for the same host records, for FP32 and BF16 rows.
- With device queries and outputs, both taco_search_batch (batch parameters) and
  taco_search_batch_params only enqueue kernels once the workspace is sized, so a call can be
  captured into a CUDA graph; replays give the results of the direct call, replay after
  replay, and follow new query values written into the captured input buffer.
- Bad handles and mismatched sizes are refused before any launch."""
import numpy as np
import pytest

from oracle import taco_oracle as O
from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoError, TacoIndex, build_lib  # noqa: E402

build_lib.build()


@pytest.fixture(scope="module")
def tiny():
    w, data, queries = make_workload("tiny20k", nq=64)
    oix = O.create_index(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=10, seed=1)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              w.n_subspaces, w.sub_dim, w.sqrt_k, keep_bf16=True)
    yield w, data, queries, ix
    ix.close()


def _per_query(n, precision, seed):
    rng = np.random.default_rng(seed)
    return [dict(k=int(rng.choice([1, 10, 50, 100])), budget=int(rng.choice([200, 1000, 3000])),
                 rerank_target=int(rng.choice([50, 200, 1000])), precision=precision,
                 shortlist_mult=int(rng.choice([1, 2])) if precision != "fp32" else 1)
            for _ in range(n)]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_prepared_equals_host_records(tiny, precision):
    w, data, queries, ix = tiny
    q = torch.from_numpy(queries).cuda()
    pq = _per_query(len(queries), precision, 3)
    ids, dists = ix.search(q, 10, 1, 0, per_query=pq, k_stride=100, precision=precision)
    prep = ix.prepare(pq)
    assert prep.nq == len(queries) and prep.k_max == max(p["k"] for p in pq)
    for _ in range(2):
        p_ids, p_d = ix.search_prepared(q, prep, k_stride=100)
        torch.cuda.synchronize()
        assert torch.equal(p_ids, ids)
        assert torch.equal(p_d, dists)
    prep.close()


def _capture(fn):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        fn()
    return g


def test_graph_capture_of_batch_search(tiny):
    w, data, queries, ix = tiny
    q = torch.from_numpy(queries).cuda()
    ids = torch.empty((len(queries), 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((len(queries), 10), dtype=torch.float32, device="cuda")
    args = (10, w.budget, w.rerank_target)
    ref_ids, ref_d = ix.search(q, *args, out_ids=ids, out_dists=dists)   # sizes the workspace
    torch.cuda.synchronize()
    ref_ids, ref_d = ref_ids.clone(), ref_d.clone()
    g = _capture(lambda: ix.search(q, *args, out_ids=ids, out_dists=dists))
    for _ in range(3):
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids) and torch.equal(dists, ref_d)
    # the graph reads the captured query buffer: new values, new answers
    q2 = torch.from_numpy(queries[::-1].copy()).cuda()
    want_ids, want_d = ix.search(q2, *args)
    q.copy_(q2)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ids, want_ids) and torch.equal(dists, want_d)


def test_graph_capture_of_prepared_batch(tiny):
    w, data, queries, ix = tiny
    q = torch.from_numpy(queries).cuda()
    pq = _per_query(len(queries), "bf16", 4)
    prep = ix.prepare(pq)
    ids = torch.empty((len(queries), 100), dtype=torch.int64, device="cuda")
    dists = torch.empty((len(queries), 100), dtype=torch.float32, device="cuda")
    ix.search_prepared(q, prep, k_stride=100, out_ids=ids, out_dists=dists)
    torch.cuda.synchronize()
    ref_ids, ref_d = ids.clone(), dists.clone()
    g = _capture(lambda: ix.search_prepared(q, prep, k_stride=100, out_ids=ids, out_dists=dists))
    for _ in range(3):
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids) and torch.equal(dists, ref_d)
    assert ix.device_status() == 0
    prep.close()


def test_prepared_rejections(tiny):
    w, data, queries, ix = tiny
    q = torch.from_numpy(queries).cuda()
    prep = ix.prepare([dict(k=50, budget=1000, rerank_target=200)] * 8)
    with pytest.raises(ValueError):   # 64 queries for 8 records
        ix.search_prepared(q, prep)
    with pytest.raises(TacoError):    # k_stride below a prepared k
        ix.search_prepared(q[:8], prep, k_stride=10)
    with pytest.raises(TacoError):    # mixed precision in one batch
        ix.prepare([dict(k=1, budget=10, rerank_target=1),
                    dict(k=1, budget=10, rerank_target=1, precision="bf16")])
    with pytest.raises(TacoError):    # k above the compiled maximum
        ix.prepare([dict(k=600, budget=10, rerank_target=1)])
    prep.close()

"""taco_search_batch_noalloc, the entry point for callers that may not allocate device
memory, gives the same results as taco_search_batch, call after call. Collected last so a
failure here cannot hide the results of the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoError, TacoIndex, build_lib  # noqa: E402
from synth import make_workload  # noqa: E402

build_lib.build()


@pytest.fixture(scope="module")
def index():
    w, data, queries = make_workload("tiny20k", n=20_000, nq=100)
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=10, seed=2)
    yield w, queries, ix
    ix.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_noalloc_matches_search_batch_twice(index, precision):
    w, queries, ix = index
    q = torch.from_numpy(queries).cuda()
    ref_ids, ref_d = ix.search(q, 10, w.budget, w.rerank_target, precision=precision,
                               shortlist_mult=2)
    for _ in range(2):   # the shared scratch keeps the previous call's contents
        ids = torch.full((len(queries), 10), -7, dtype=torch.int64, device="cuda")
        dists = torch.full((len(queries), 10), -7.0, dtype=torch.float32, device="cuda")
        ix.search_noalloc(q, ids, dists, 10, w.budget, w.rerank_target, precision=precision,
                          shortlist_mult=2)
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        np.testing.assert_allclose(dists.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5)


def test_noalloc_rejects_batches_beyond_its_scratch(index):
    w, queries, ix = index
    q = torch.zeros((20_000, 128), device="cuda")
    ids = torch.empty((20_000, 10), dtype=torch.int64, device="cuda")
    dists = torch.empty((20_000, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(TacoError) as err:
        ix.search_noalloc(q, ids, dists, 10, w.budget, w.rerank_target)
    assert err.value.code == -5

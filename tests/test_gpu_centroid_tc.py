"""The query x centroid distance block (Alg. 6 steps 4-5) on CUDA cores and on the tcgen05
tensor cores, through taco_centroid_distances, and the search with probe_precision BF16.

FP32 block: equals the FP64 oracle's half distances within 1e-5 relative. BF16 block: BF16
operands with FP32 accumulation of |q|^2 + |c|^2 - 2 q.c, checked against the FP64
distances of the BF16-rounded operands within a bound set by FP32 rounding of the three
terms. Geometries: the 20k x 128 workload (sqrt(K) = 16, halves of 8) and a ragged one
(sqrt(K) = 7 padded to the MMA's N = 16, 15 subspaces with halves of 2 and 3 padded to K = 16)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import taco_oracle as O  # noqa: E402
from paper_2603_24919_gb300 import TacoIndex, build_lib  # noqa: E402
from synth import make_workload  # noqa: E402

build_lib.build()


def _bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _index(name, n, nq, ns, s, sk, d=None):
    w, data, queries = make_workload(name, n=n, nq=nq)
    if d is not None:
        data, queries = np.ascontiguousarray(data[:, :d]), np.ascontiguousarray(queries[:, :d])
    oix = O.create_index(data, ns, s, sk, kmeans_iters=5, seed=3)
    ix = TacoIndex.from_parts(data, oix.o_bar, oix.B, oix.centroids, oix.codes.astype(np.uint16),
                              ns, s, sk)
    return w, data, queries, oix, ix


@pytest.fixture(scope="module", params=["tiny", "ragged"])
def case(request):
    if request.param == "tiny":
        w, data, queries, oix, ix = _index("tiny20k", 20_000, 300, 8, 16, 16)
    else:
        w, data, queries, oix, ix = _index("tiny20k", 5_003, 200, 15, 5, 7, d=100)
    yield data, queries, oix, ix
    ix.close()


def _qt(ix, queries, oix):
    q = torch.from_numpy(queries).cuda()
    dbg = ix.search_debug(q, 1, 1, 0, want_sc=False)
    torch.cuda.synchronize()
    return dbg["query_t"]


def test_fp32_block_matches_oracle(case):
    data, queries, oix, ix = case
    qt = _qt(ix, queries, oix)
    hd = ix.centroid_distances(qt, "fp32").cpu().numpy()
    qt64 = qt.cpu().numpy().astype(np.float64)
    for j in range(0, len(queries), 7):
        for i in range(oix.n_subspaces):
            d1, d2 = O.half_distances(oix, qt64[j], i)
            np.testing.assert_allclose(hd[j, i, 0], d1, rtol=1e-5, atol=1e-4)
            np.testing.assert_allclose(hd[j, i, 1], d2, rtol=1e-5, atol=1e-4)


def test_tensor_core_block_matches_bf16_operands(case):
    data, queries, oix, ix = case
    assert ix.info()["has_centroid_tc"] == 1
    qt = _qt(ix, queries, oix)
    hd = ix.centroid_distances(qt, "bf16").cpu().numpy()
    assert ix.device_status() == 0
    qb = _bf16(qt.cpu().numpy())
    cb = _bf16(oix.centroids)
    h1, _ = O.half_dims(oix.sub_dim)
    s = oix.sub_dim
    for i in range(oix.n_subspaces):
        for h, (a, b) in enumerate(((0, h1), (h1, s))):
            qh = qb[:, i * s + a:i * s + b]              # [nq, len]
            ch = cb[i][:, a:b]                           # [sk, len]
            ref = ((qh[:, None, :] - ch[None, :, :]) ** 2).sum(-1)
            mag = (qh ** 2).sum(-1)[:, None] + (ch ** 2).sum(-1)[None, :]
            err = np.abs(hd[:, i, h, :] - ref)
            assert np.all(err <= 1e-5 * mag + 1e-5), (i, h, float((err / (mag + 1e-9)).max()))


def test_full_budget_search_is_the_same_with_either_block():
    """With a budget above n every cell is probed whatever the distances, so the search
    with the tensor-core block returns exactly the FP32 block's result."""
    w, data, queries, oix, ix = _index("tiny20k", 20_000, 50, 8, 16, 16)
    q = torch.from_numpy(queries).cuda()
    a_ids, a_d = ix.search(q, 10, 2 * oix.n, 300)
    b_ids, b_d = ix.search(q, 10, 2 * oix.n, 300, probe_precision="bf16")
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    assert ix.device_status() == 0
    ix.close()


def test_bf16_probe_recall_close_to_fp32():
    w, data, queries, oix, ix = _index("tiny20k", 20_000, 200, 8, 16, 16)
    q = torch.from_numpy(queries).cuda()
    t_ids, _ = O.brute_force_knn(data, queries, 10)
    f_ids, _ = ix.search(q, 10, w.budget, w.rerank_target)
    b_ids, b_d = ix.search(q, 10, w.budget, w.rerank_target, precision="bf16", shortlist_mult=2,
                           probe_precision="bf16")
    rf = O.recall(f_ids.cpu().numpy(), t_ids, 10)
    rb = O.recall(b_ids.cpu().numpy(), t_ids, 10)
    assert rb >= rf - 0.02, (rb, rf)
    assert ix.device_status() == 0
    ix.close()

"""The query x centroid distance block (Alg. 6 steps 4-5) on CUDA cores and on the tcgen05
tensor cores, through taco_centroid_distances, and the search with probe_precision BF16.

FP32 block: equals the FP64 oracle's half distances within 1e-5 relative. BF16 block: BF16
operands with FP32 accumulation of |q|^2 + |c|^2 - 2 q.c, checked against the FP64
distances of the BF16-rounded operands within a bound set by FP32 rounding of the three
terms. E4M3 block (kind::f8f6f4): operands c / s_c and q / s_q rounded to E4M3 (s_c = max |c|
/ 448 over the (subspace, half)'s centroids, s_q = max |q| / 448 over the half-query, both in
FP32), checked the same way against the FP64 distances of the values the rounded operands
stand for. Geometries: the 20k x 128 workload (sqrt(K) = 16, halves of 8) and a ragged one
(sqrt(K) = 7 padded to the MMA's N = 16, 15 subspaces with halves of 2 and 3 padded to K = 16)
and a wide one in the 1M x 960 workload's shape (10 subspaces of 96 dims: halves of 48, three
BF16 K-steps of 16 and an E4M3 K-step of 32 padded to 64; sqrt(K) = 64)."""
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


@pytest.fixture(scope="module", params=["tiny", "ragged", "wide"])
def case(request):
    if request.param == "tiny":
        w, data, queries, oix, ix = _index("tiny20k", 20_000, 300, 8, 16, 16)
    elif request.param == "wide":
        w, data, queries, oix, ix = _index("gist1m", 6_000, 130, 10, 96, 64)
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


def _e4m3(x32):
    """FP64 values of float32 x rounded to E4M3 (nearest, ties to even)."""
    t = torch.from_numpy(np.ascontiguousarray(x32, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def test_fp8_tensor_core_block_matches_e4m3_operands(case):
    data, queries, oix, ix = case
    qt = _qt(ix, queries, oix)
    hd = ix.centroid_distances(qt, "fp8").cpu().numpy()
    assert ix.device_status() == 0
    q32 = qt.cpu().numpy().astype(np.float32)
    c32 = oix.centroids.astype(np.float32)
    h1, _ = O.half_dims(oix.sub_dim)
    s = oix.sub_dim
    f448 = np.float32(448)
    for i in range(oix.n_subspaces):
        for h, (a, b) in enumerate(((0, h1), (h1, s))):
            qh, ch = q32[:, i * s + a:i * s + b], c32[i][:, a:b]
            amq = np.abs(qh).max(1)
            ok = amq > 0
            sq = np.where(ok, amq / f448, np.float32(0)).astype(np.float32)
            invq = np.where(ok, f448 / np.where(ok, amq, np.float32(1)), np.float32(0)).astype(np.float32)
            amc = np.float32(np.abs(ch).max())
            sc, invc = (amc / f448, f448 / amc) if amc > 0 else (np.float32(0), np.float32(0))
            qv = _e4m3(qh * invq[:, None]) * sq.astype(np.float64)[:, None]
            cv = _e4m3(ch * invc) * np.float64(sc)
            ref = ((qv[:, None, :] - cv[None, :, :]) ** 2).sum(-1)
            mag = (qv ** 2).sum(-1)[:, None] + (cv ** 2).sum(-1)[None, :]
            err = np.abs(hd[:, i, h, :] - ref)
            assert np.all(err <= 1e-5 * mag + 1e-5), (i, h, float((err / (mag + 1e-9)).max()))


def test_fp8_probe_recall_close_to_fp32():
    w, data, queries, oix, ix = _index("tiny20k", 20_000, 200, 8, 16, 16)
    q = torch.from_numpy(queries).cuda()
    t_ids, _ = O.brute_force_knn(data, queries, 10)
    f_ids, _ = ix.search(q, 10, w.budget, w.rerank_target)
    e_ids, _ = ix.search(q, 10, w.budget, w.rerank_target, precision="bf16", shortlist_mult=2,
                         probe_precision="fp8")
    rf = O.recall(f_ids.cpu().numpy(), t_ids, 10)
    re = O.recall(e_ids.cpu().numpy(), t_ids, 10)
    assert re >= rf - 0.03, (re, rf)
    assert ix.device_status() == 0
    ix.close()


def test_full_budget_search_is_the_same_with_either_block():
    """With a budget above n every cell is probed whatever the distances, so the search
    with the tensor-core block returns exactly the FP32 block's result."""
    w, data, queries, oix, ix = _index("tiny20k", 20_000, 50, 8, 16, 16)
    q = torch.from_numpy(queries).cuda()
    a_ids, a_d = ix.search(q, 10, 2 * oix.n, 300)
    b_ids, b_d = ix.search(q, 10, 2 * oix.n, 300, probe_precision="bf16")
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    e_ids, e_d = ix.search(q, 10, 2 * oix.n, 300, probe_precision="fp8")
    assert torch.equal(a_ids, e_ids) and torch.equal(a_d, e_d)
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

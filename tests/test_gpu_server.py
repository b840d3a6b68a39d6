"""The serving loop (taco_server_*): continuous batching over a resident index.

Requests with mixed k, budgets and targets arrive from several threads (or by an
open-loop Poisson replay) while earlier batches run; every result must equal the answer
the same query gets alone from taco_search_batch, ids exactly and distances within 1e-5
relative. Admission (queue capacity, slot workspace bytes) and CUDA-graph replay are
checked through the server's counters."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import TacoError, TacoIndex, TacoServer, build_lib  # noqa: E402
from paper_2603_24919_gb300 import taco as T  # noqa: E402
from synth import make_workload  # noqa: E402

build_lib.build()

KS = [1, 10, 50, 100]


@pytest.fixture(scope="module")
def index():
    w, data, queries = make_workload("tiny20k", n=20_000, nq=400)
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=10, seed=4)
    yield w, queries, ix
    ix.close()


def _mixed_params(n, precision, seed, probe_precision="fp32"):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        p = dict(k=int(rng.choice(KS)), budget=int(rng.choice([200, 1000, 3000])),
                 rerank_target=int(rng.choice([50, 200, 1000])), precision=precision,
                 probe_precision=probe_precision)
        if precision == "bf16":
            p["shortlist_mult"] = int(rng.choice([1, 2, 4]))
        out.append(p)
    return out


def _alone(ix, queries, params, k_stride):
    """Each query answered in a batch of its own through taco_search_batch."""
    ids = np.full((len(params), k_stride), -1, dtype=np.int64)
    dists = np.full((len(params), k_stride), np.inf, dtype=np.float32)
    for j, p in enumerate(params):
        q = torch.from_numpy(queries[j:j + 1]).cuda()
        a_i, a_d = ix.search(q, p["k"], p["budget"], p["rerank_target"],
                             precision=p["precision"], shortlist_mult=p.get("shortlist_mult", 4),
                             probe_precision=p.get("probe_precision", "fp32"), k_stride=k_stride)
        ids[j], dists[j] = a_i.cpu().numpy()[0], a_d.cpu().numpy()[0]
    return ids, dists


def _max_list(params):
    return max(min(p["k"] * p.get("shortlist_mult", 1), 512) if p["precision"] == "bf16"
               else p["k"] for p in params)


def _assert_same(ids, dists, ref_ids, ref_d):
    assert np.array_equal(ids, ref_ids)
    fin = np.isfinite(ref_d)
    assert np.array_equal(np.isfinite(dists), fin)
    np.testing.assert_allclose(dists[fin], ref_d[fin], rtol=1e-5)


@pytest.mark.parametrize("precision,use_graphs,probe", [("fp32", True, "fp32"), ("bf16", True, "fp32"),
                                                        ("fp32", False, "fp32"), ("bf16", True, "bf16")])
def test_results_alone_equal_results_in_the_mix(index, precision, use_graphs, probe):
    """probe = "bf16": the tcgen05 centroid block (bulk copies, mbarriers, tensor memory)
    inside the captured graphs."""
    w, queries, ix = index
    n = 240
    params = _mixed_params(n, precision, seed=7, probe_precision=probe)
    k_stride = max(KS)
    ref_ids, ref_d = _alone(ix, queries, params, k_stride)
    got_ids = np.zeros_like(ref_ids)
    got_d = np.zeros_like(ref_d)
    infos = [None] * n
    with TacoServer(ix, max_batch=32, slots=3, queue_capacity=64, max_list=_max_list(params),
                    precision=precision, max_wait_us=300, use_graphs=use_graphs,
                    probe_precision=probe) as srv:
        def client(rows):
            # each client keeps a few requests outstanding, so batches mix clients
            pend = []
            for j in rows:
                while True:
                    try:
                        pj = {k_: v for k_, v in params[j].items() if k_ != "probe_precision"}
                        pend.append((j, srv.submit(queries[j], **pj)))
                        break
                    except TacoError as e:
                        assert e.code == T.EAGAIN
                        if pend:
                            jj, t = pend.pop(0)
                            got_ids[jj], got_d[jj], infos[jj] = srv.wait(t, k_stride)
                if len(pend) >= 6:
                    jj, t = pend.pop(0)
                    got_ids[jj], got_d[jj], infos[jj] = srv.wait(t, k_stride)
            for jj, t in pend:
                got_ids[jj], got_d[jj], infos[jj] = srv.wait(t, k_stride)

        threads = [threading.Thread(target=client, args=(range(c, n, 4),)) for c in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        st = srv.stats()
    _assert_same(got_ids, got_d, ref_ids, ref_d)
    assert st["submitted"] == n and st["completed"] == n
    assert st["batches"] < n            # requests were batched together
    assert st["max_batch_seen"] > 1
    assert max(i["batch_size"] for i in infos) > 1
    assert all(i["submit_ns"] <= i["dispatch_ns"] <= i["done_ns"] for i in infos)
    if use_graphs:
        assert st["graph_launches"] > 0 and st["graph_captures"] > 0
    else:
        assert st["graph_launches"] == 0


def test_poisson_replay_overlaps_batches(index):
    w, queries, ix = index
    n = 400
    params = _mixed_params(n, "fp32", seed=11)
    k_stride = max(KS)
    rng = np.random.default_rng(3)
    arrival = np.cumsum(rng.exponential(1e9 / 100_000, size=n)).astype(np.int64)  # 100k QPS
    with TacoServer(ix, max_batch=64, slots=4, queue_capacity=256, max_list=_max_list(params),
                    max_wait_us=20) as srv:
        ids, dists, lat = srv.replay(queries[:n], params, arrival, k_stride)
        st = srv.stats()
    ref_ids, ref_d = _alone(ix, queries, params, k_stride)
    _assert_same(ids, dists, ref_ids, ref_d)
    assert np.all(lat > 0)
    assert st["completed"] == n and st["batches"] < n
    assert st["max_in_flight"] >= 2     # a batch was admitted while another ran


def test_admission_by_workspace_bytes_and_queue(index):
    w, queries, ix = index
    p = dict(k=10, budget=1000, rerank_target=200)
    with TacoServer(ix, max_batch=64, slots=1, queue_capacity=64, max_list=10,
                    use_graphs=False) as big:
        full = big.stats()["slot_bytes"]
    # a workspace that holds about 8 queries: batches stay below it
    with TacoServer(ix, max_batch=64, slots=1, queue_capacity=64, max_list=10,
                    slot_bytes=full // 8, use_graphs=False, max_wait_us=5000) as srv:
        tickets = [srv.submit(queries[j], **p) for j in range(64)]
        with pytest.raises(TacoError) as err:   # the queue holds 64 requests
            srv.submit(queries[0], **p)
        assert err.value.code == T.EAGAIN
        for t in tickets:
            srv.wait(t, 10)
        st = srv.stats()
    assert st["rejected"] == 1
    assert 1 < st["max_batch_seen"] <= 9
    with pytest.raises(TacoError) as err:   # a request needing a longer list than max_list
        with TacoServer(ix, max_batch=8, slots=1, max_list=10) as srv:
            srv.submit(queries[0], 50, 1000, 200)
    assert err.value.code == T.EINVAL


def test_wait_timeout_and_bad_tickets(index):
    w, queries, ix = index
    with TacoServer(ix, max_batch=8, slots=1, max_list=10) as srv:
        t = srv.submit(queries[0], 10, 1000, 200)
        ids, dists, info = srv.wait(t, 10)
        with pytest.raises(TacoError) as err:   # collected once
            srv.wait(t, 10)
        assert err.value.code == T.EINVAL
        with pytest.raises(TacoError) as err:
            srv.wait(12345, 10, timeout_us=10)
        assert err.value.code == T.EINVAL
        with pytest.raises(TacoError) as err:   # precision must match the server's
            srv.submit(queries[0], 10, 1000, 200, precision="bf16")
        assert err.value.code == T.EINVAL


def test_submit_many_takes_a_prefix_and_matches_alone(index):
    w, queries, ix = index
    params = _mixed_params(100, "fp32", seed=5)
    k_stride = max(KS)
    ref_ids, ref_d = _alone(ix, queries, params, k_stride)
    with TacoServer(ix, max_batch=32, slots=2, queue_capacity=64, max_list=_max_list(params),
                    max_wait_us=50) as srv:
        tickets = srv.submit_many(queries[:100], params)
        assert len(tickets) == 64            # the queue holds 64
        got = {}
        for j, t in enumerate(tickets):
            got[j] = srv.wait(t, k_stride)[:2]
        tickets2 = srv.submit_many(queries[64:100], params[64:100])
        assert len(tickets2) == 36
        for j, t in enumerate(tickets2):
            got[64 + j] = srv.wait(t, k_stride)[:2]
        st = srv.stats()
    ids = np.stack([got[j][0] for j in range(100)])
    dists = np.stack([got[j][1] for j in range(100)])
    _assert_same(ids, dists, ref_ids, ref_d)
    assert st["rejected"] == 36 and st["completed"] == 100

"""Searches run under a chosen build of the library (TACO_LIB), for tests/test_gpu_checked.py.

Usage: python tests/checked_workload.py OUT.npz INDEX_FILE. The 1M x 128 index is built and
saved to INDEX_FILE if the file does not exist, and every run searches the index loaded from
that file, so that runs under two builds search the same index (the GPU build's
floating-point atomics make two builds of an index differ in the last bits of the mean, the
covariance and the centroids). Runs: the FP32,
BF16 and FP8 forms over an (alpha, beta) grid up to alpha 0.1 / beta 0.01 (the 1M x 128
workload on 2,000 queries, FP8 shortlists 2k-8k), the cluster fallback (a target larger than
n: Alg. 5 keeps every level), the codes fallback, a multi-slab index and per-query k; saves
every result and the index's device status word after each case."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2603_24919_gb300 import TacoIndex  # noqa: E402
from synth import budget_from_alpha, make_workload, target_from_beta  # noqa: E402


def main(out_path, index_path):
    torch.cuda.set_device(0)
    res = {}
    # the 1M x 128 workload: the FP8 grid at large alpha / beta, BF16 and FP32 beside it
    w, data, queries = make_workload("sift1m", nq=2000)
    if not os.path.exists(index_path):
        built = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=10, seed=1)
        built.save(index_path)
        built.close()
    ix = TacoIndex.load(index_path, keep_bf16=True, keep_fp8=True)   # both runs: the same file
    q = torch.from_numpy(queries).cuda()
    n = w.n
    for a, b in [(0.01, 0.001), (0.05, 0.005), (0.1, 0.01), (0.1, 0.001)]:
        bud, tgt = budget_from_alpha(a, n), target_from_beta(b, n)
        for prec, mults in (("fp32", [1]), ("bf16", [1, 4]), ("fp8", [2, 4, 8])):
            for m in mults:
                ids, d = ix.search(q, 10, bud, tgt, precision=prec, shortlist_mult=m)
                res[f"sift_{a}_{b}_{prec}_{m}_ids"] = ids.cpu().numpy()
                res[f"sift_{a}_{b}_{prec}_{m}_d"] = d.cpu().numpy()
    res["sift_status"] = np.array([ix.device_status()])
    # every level kept (cluster fallback for all queries), then the codes fallback
    for name, codes in (("cluster", False), ("codes", True)):
        ix.set_codes_fallback(codes)
        ids, d = ix.search(q[:64], 10, budget_from_alpha(0.02, n), 10 * n, precision="bf16", shortlist_mult=2)
        res[f"sift_all_{name}_ids"], res[f"sift_all_{name}_d"] = ids.cpu().numpy(), d.cpu().numpy()
        ids, d = ix.search(q[:256], 10, budget_from_alpha(0.002, n), target_from_beta(0.01, n))
        res[f"sift_low_{name}_ids"], res[f"sift_low_{name}_d"] = ids.cpu().numpy(), d.cpu().numpy()
    res["fallback_status"] = np.array([ix.device_status()])
    # per-query k and budgets in one batch
    rng = np.random.default_rng(3)
    pq = [dict(k=int(rng.choice([1, 10, 50, 100])), budget=budget_from_alpha(float(rng.choice([0.005, 0.02])), n),
               rerank_target=target_from_beta(float(rng.choice([0.0005, 0.005])), n), precision="bf16",
               shortlist_mult=2) for _ in range(512)]
    ids, d = ix.search(q[:512], 10, 1, 0, per_query=pq, k_stride=100, precision="bf16")
    res["uneven_ids"], res["uneven_d"] = ids.cpu().numpy(), d.cpu().numpy()
    res["uneven_status"] = np.array([ix.device_status()])
    ix.close()
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])

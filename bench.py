#!/usr/bin/env python
"""Benchmark of the TaCo query path on one GB300: QPS at recall@10 >= 0.95, batched BF16
against the plain FP32 path.

Headline workload (the batched uneven form): 10,000,000 x 96 unit-normalised float32 points
(a 4096-component Gaussian mixture, a Yandex DEEP10M stand-in), batches of 4,096 queries
from the same mixture whose k is drawn per query from {1, 10, 50, 100}, N_s = 6 subspaces of
s = 8 dims, sqrt(K) = 64. Budgets are query-aware as the method makes them: each query meets
its collision budget at cell granularity (Alg. 4) and keeps its own candidate set (Alg. 5).
One step = the whole query path (transform, query x centroid block, cell probe, collision
counting, Alg. 5 selection, re-rank) over one batch, with the per-query parameters resident
on the device.

The operating point (alpha, beta, shortlist) of each form is the one with the highest QPS
whose mean recall@10 (over the queries with k >= 10) against exact k-NN is >= 0.95, on a grid
that reaches below the target. The headline `value` is the batched BF16 form; the plain FP32
form is `fp32_qps`. The 1M x 128 workload (the plain FP32 method's config) follows under
"sift1m": operating points at recall@10 0.9 / 0.95 / 0.99, recall@1 and recall@100 0.95, and
the serving loop.

Arms:
  default            the CUDA library (libtaco.so) through its C ABI
  --impl reference   the FP64 CPU oracle on the host cores, a bounded query sample per step

Multi-GPU (torchrun): every rank holds a replica of the index and answers its own batch;
no collective is on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10≥0.95, 1 GB300: batched BF16 vs plain FP32; p50/p99 latency"
WORKLOAD = "deep10m"          # the headline line: batched uneven form
EXTRA_WORKLOAD = "sift1m"     # extra keys of the same line
KS_BATCHED = (1, 10, 50, 100)   # per-query k of the batched form
# calibration grid: below the paper's ranges (alpha 0.01-0.1, beta 0.001-0.05) too, since
# recall@10 reaches 0.95 below them on these stand-ins
GRID_ALPHA = (0.0005, 0.001, 0.0015, 0.002, 0.0025, 0.003, 0.0035, 0.004, 0.0045, 0.005, 0.0075, 0.01,
              0.02, 0.05)
GRID_BETA = (0.0001, 0.0002, 0.00025, 0.0003, 0.0004, 0.0005, 0.00075, 0.001, 0.002, 0.005)
RECALL_TARGET = 0.95
# (alpha, beta) of the reference arm per workload, near the GPU operating points
REFERENCE_OP = {"deep10m": (0.005, 0.0005), "sift1m": (0.01, 0.001)}
SHORTLIST_MULTS = {"bf16": [1, 2, 4], "fp8": [2, 4, 8], "bf16_tc": [1, 2, 4]}   # FP32 re-rank of mult * k
# search arguments of each form: rows of the candidate re-rank, and the query x centroid block
HEADLINE = "bf16_tc"
FORMS = {"fp32": dict(precision="fp32"), "bf16": dict(precision="bf16"),
         "fp8": dict(precision="fp8"),
         "bf16_tc": dict(precision="bf16", probe_precision="bf16"),   # tcgen05 centroid block
         "fp8_tc": dict(precision="fp8", probe_precision="fp8")}      # E4M3 rows and block
K = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="taco", choices=["taco", "reference"])
    ap.add_argument("--nq", type=int, default=None, help="queries per batch of the workload")
    ap.add_argument("--nq-extra", type=int, default=10_000, help="queries per batch of the 1M x 128 keys")
    ap.add_argument("--no-extra", action="store_true", help="skip the 1M x 128 keys")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--alpha", type=float, default=None, help="skip calibration (both forms)")
    ap.add_argument("--beta", type=float, default=None)
    ap.add_argument("--no-serving", action="store_true", help="skip the Poisson serving runs")
    ap.add_argument("--count-layout", default=None, metavar="SLABS,WARPS,UNROLL",
                    help="use this counting layout instead of autotuning it (profiler runs, "
                         "whose timings mislead the tuner)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="deep10m (the headline line) or deep5m256 / gist1m (their own line: "
                         "serving form, precision form); with --impl reference any workload of "
                         "synth (e.g. tiny20k)")
    ap.add_argument("--serve-seconds", type=float, default=0.3,
                    help="arrival span of each offered load in the serving runs")
    ap.add_argument("--ncu-case", default=None, metavar="FORM",
                    help="profiling case (no calibration, tuning or timing): build --workload "
                         "(deep10m by default; --nq queries), then run --steps searches of FORM "
                         "(fp32, bf16, bf16_tc, fp8, fp8_tc) at --alpha / --beta, per-query k for "
                         "deep10m, with --count-layout if given; for runs under a profiler")
    ap.add_argument("--codes-fallback", action="store_true",
                    help="with --ncu-case: answer flagged queries by the codes fallback")
    ap.add_argument("--n", type=int, default=None,
                    help="with --ncu-case: points of the workload (a smaller case for full captures)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(total, ws, rank):
    """Half-open range of the units (queries) rank `rank` of `ws` answers: contiguous,
    disjoint, covering [0, total), sizes differing by at most one."""
    base, extra = divmod(total, ws)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(values, ws, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity when ws == 1)."""
    if ws == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------------------ helpers
def exact_knn_gpu(torch, data_t, queries_t, data_np, queries_np, k, extra=32, chunk=1000):
    """Exact k-NN for recall: FP32 brute force on the GPU for a candidate pool of k+extra,
    then FP64 re-check of the pool on the host (ordered by distance, then id)."""
    xn = (data_t * data_t).sum(1)
    out = np.empty((queries_t.shape[0], k), dtype=np.int64)
    for a in range(0, queries_t.shape[0], chunk):
        q = queries_t[a:a + chunk]
        d2 = (q * q).sum(1, keepdim=True) - 2.0 * (q @ data_t.T) + xn[None, :]
        pool = torch.topk(d2, k + extra, dim=1, largest=False).indices.cpu().numpy()
        qq = queries_np[a:a + chunk].astype(np.float64)
        for j in range(pool.shape[0]):
            cand = pool[j]
            dd = ((data_np[cand].astype(np.float64) - qq[j]) ** 2).sum(1)
            o = np.lexsort((cand, dd))[:k]
            out[a + j] = cand[o]
    return out


def recall_at(ids, truth, k):
    ids = np.asarray(ids)[:, :k]
    hits = [len(set(r.tolist()) & set(t.tolist())) for r, t in zip(ids, truth[:, :k])]
    return float(np.mean(hits)) / k


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="taco_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(nq, retrieved, ncells, cand, entries, d, d_pad, k, mult, n_ranges,
                      n_subspaces, sqrt_k):
    """Algorithmic bytes of one launch of each search kernel over a batch of nq queries
    (BF16 candidate rows, the headline form), and of the whole path ("path"): the ids of the
    probed cells (retrieved: their total over the batch and subspaces), the cells' offsets
    (ncells probed cells), the candidate rows (cand candidates), the exact FP32 shortlist of
    min(mult * k, 512) rows, each query's row and its k results; entries = level-list
    entries (ids with SC >= 2); 72 B of unit state per (query, id range). k is one value for
    the batch or one per query."""
    kq = np.broadcast_to(np.asarray(k, dtype=np.int64), (nq,))
    shortlist_rows = int(np.minimum(mult * kq, 512).sum())
    io = int(nq * d * 4 + 12 * kq.sum())
    units = nq * n_ranges * 72
    return {
        "count_lists": 4 * retrieved + 8 * ncells + 4 * entries + units,
        "select_rerank": cand * d_pad * 2 + shortlist_rows * d_pad * 4 + 4 * entries + units + io,
        "cluster_count_select": 4 * retrieved + 8 * ncells + cand * d_pad * 2 + io,
        "probe_cells": nq * n_subspaces * (sqrt_k ** 2) * 4 + 2 * ncells,
        "path": 4 * retrieved + 4 * ncells + cand * d * 2 + shortlist_rows * d * 4 + io,
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the counting kernel (its code and constants)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_24919_gb300", "csrc")
    for name in ("taco_count.cuh", "taco_select.cuh", "taco_rerank.cuh", "taco_internal.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_limiter(kernel, workload=WORKLOAD):
    """The ncu reading of what bounds `kernel` from the committed summary, if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        lim = json.load(f).get("limiter")
    if not lim or lim.get("source_hash") != kernel_source_hash():
        return None
    return {k: v for k, v in lim.items() if k != "source_hash"}


def ncu_traffic(kernel, precision, workload=WORKLOAD):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    entry = j.get(precision)
    if not entry or entry.get("source_hash") != kernel_source_hash():
        return None
    return entry.get("dram_bytes_per_launch_full_batch")


# ------------------------------------------------------------------------------ GPU arm
def _grid():
    return [(a, b) for a in GRID_ALPHA for b in GRID_BETA]


def _on_edge(a, b):
    """Whether (a, b) lies on the border of the calibration grid (then the true optimum may
    lie outside it)."""
    return a in (GRID_ALPHA[0], GRID_ALPHA[-1]) or b in (GRID_BETA[0], GRID_BETA[-1])


class Searcher:
    """Timed searches of one index over one batch: uniform parameters (k fixed) or per-query
    parameters prepared on the device once per operating point (taco_params_create), so the
    timed region holds the kernels alone."""

    def __init__(self, torch, ix, q_dev, n, ks=None, kmax=K):
        self.torch, self.ix, self.q, self.n = torch, ix, q_dev, n
        self.ks = ks   # per-query k (None: uniform k per call)
        self.kmax = kmax
        self.stream = torch.cuda.current_stream()
        nq = q_dev.shape[0]
        self.out_ids = torch.empty((nq, kmax), dtype=torch.int64, device="cuda")
        self.out_d = torch.empty((nq, kmax), dtype=torch.float32, device="cuda")
        self._prep = {}

    def per_query(self, form, a, b, mult, k=None):
        from synth import budget_from_alpha, target_from_beta
        bud, tgt = budget_from_alpha(a, self.n), target_from_beta(b, self.n)
        ks = self.ks if k is None else [k] * self.q.shape[0]
        return [dict(k=int(kq), budget=bud, rerank_target=tgt, shortlist_mult=mult, **FORMS[form])
                for kq in ks]

    def prepared(self, form, a, b, mult):
        key = (form, a, b, mult)
        if key not in self._prep:
            if len(self._prep) > 8:   # keep device memory bounded during calibration
                for v in self._prep.values():
                    v.close()
                self._prep.clear()
            self._prep[key] = self.ix.prepare(self.per_query(form, a, b, mult))
        return self._prep[key]

    def one(self, form, a, b, mult, k=None):
        """One search at (a, b); k=None: the per-query k (prepared), else uniform k."""
        from synth import budget_from_alpha, target_from_beta
        if k is None:
            self.ix.search_prepared(self.q, self.prepared(form, a, b, mult), k_stride=self.kmax,
                                    out_ids=self.out_ids, out_dists=self.out_d)
        else:
            self.ix.search(self.q, k, budget_from_alpha(a, self.n), target_from_beta(b, self.n),
                           shortlist_mult=mult, k_stride=self.kmax, out_ids=self.out_ids,
                           out_dists=self.out_d, **FORMS[form])

    def timed(self, form, a, b, mult, reps, k=None, warm=1):
        torch = self.torch
        for _ in range(warm):
            self.one(form, a, b, mult, k)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        evs[0].record(self.stream)
        for r in range(reps):
            self.one(form, a, b, mult, k)
            evs[r + 1].record(self.stream)
        torch.cuda.synchronize()
        return [evs[r].elapsed_time(evs[r + 1]) for r in range(reps)]

    def ids(self):
        return self.out_ids.cpu().numpy()

    def close(self):
        for v in self._prep.values():
            v.close()
        self._prep.clear()


def calibrate(srch, form, mults, targets, recall_fn, log_name, reps=2):
    """Per target (name -> (k or None, recall threshold)): the operating point of `form` with
    the highest QPS whose recall meets the threshold. Every grid point is searched once at the
    largest k to read its recalls (a smaller k's top list is a prefix of the larger one's), then
    the points meeting a target are timed at that target's k; the best is re-timed."""
    nq = srch.q.shape[0]
    rec = {}
    for mult in mults:
        for a, b in _grid():
            srch.one(form, a, b, mult, None if srch.ks is not None else srch.kmax)
            ids = srch.ids()
            rec[(a, b, mult)] = {t: recall_fn(ids, k) for t, (k, _) in targets.items()}
    out = {}
    for t, (k, thr) in targets.items():
        ok = [key for key, r in rec.items() if r[t] >= thr]
        if not ok:   # nothing meets the target: the highest-recall point
            ok = [max(rec, key=lambda key: rec[key][t])]
        timed = []
        for a, b, mult in ok:
            ms = float(np.median(srch.timed(form, a, b, mult, reps, k)))
            timed.append((nq / (ms * 1e-3), a, b, mult))
        timed.sort(reverse=True)
        best = None
        for qps0, a, b, mult in timed[:3]:   # re-time the three fastest
            ms = float(np.median(srch.timed(form, a, b, mult, 5, k)))
            if best is None or nq / (ms * 1e-3) > best["qps"]:
                best = {"alpha": a, "beta": b, "shortlist_mult": mult, "recall": round(rec[(a, b, mult)][t], 4),
                        "qps": round(nq / (ms * 1e-3), 1), "met": rec[(a, b, mult)][t] >= thr,
                        "on_grid_edge": _on_edge(a, b), "points_meeting": len(ok) if rec[ok[0]][t] >= thr else 0}
        out[t] = best
        log(f"[{log_name}] {form} {t}: {best}")
    return out


def run_steps(torch, srch, ix, form, op, steps, warmup, profile, ws, k=None):
    """The timed region of one form at its operating point: W warm-up searches, then K
    searches bracketed by CUDA events on the search stream (max over ranks outside)."""
    import torch.distributed as dist
    a, b, mult = op["alpha"], op["beta"], op["shortlist_mult"]
    for _ in range(warmup):
        srch.one(form, a, b, mult, k)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        ix.profile_read(reset=True)
        ix.profile(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(srch.stream)
    for s_ in range(steps):
        srch.one(form, a, b, mult, k)
        evs[s_ + 1].record(srch.stream)
    torch.cuda.synchronize()
    if profile:
        ix.profile(False)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    per = [evs[s_].elapsed_time(evs[s_ + 1]) for s_ in range(steps)]
    total = evs[0].elapsed_time(evs[-1])
    kt = ix.profile_read(reset=True) if profile else None
    return total, per, kt


def mre_of(d_np, truth_d, kq):
    """Mean relative error (Section 6.1) over each query's first kq[j] results."""
    vals = []
    for j, k in enumerate(kq):
        t = truth_d[j, :k]
        g = d_np[j, :k].astype(np.float64)
        ok = (t > 0) & np.isfinite(g)
        vals.append(float(np.mean((g[ok] - t[ok]) / t[ok])) if ok.any() else 0.0)
    return float(np.mean(vals))


def run_taco(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    torch.backends.cuda.matmul.allow_tf32 = False
    from paper_2603_24919_gb300 import TacoIndex, build_lib, query_param_array
    from synth import budget_from_alpha, make_workload, target_from_beta

    if rank == 0:
        build_lib.build()
    if ws > 1:
        dist.barrier()
    t0 = time.time()
    # weak scaling: every rank answers its own batch of the per-rank size, drawn from one
    # pool of ws * nq queries (rank r takes slice r); no collective on the data path
    w0 = _workload_spec(WORKLOAD)
    nq_rank = args.nq or w0.nq
    w, data, pool = make_workload(WORKLOAD, nq=nq_rank * ws)
    ks_pool = np.random.default_rng(4242).choice(KS_BATCHED, size=pool.shape[0])
    lo, hi = shard(pool.shape[0], ws, rank)
    queries = np.ascontiguousarray(pool[lo:hi])
    ks = ks_pool[lo:hi]
    del pool
    nq, n = queries.shape[0], w.n
    kmax = int(max(KS_BATCHED))
    log(f"[rank {rank}] workload {w.name}: n={n} d={w.d} nq={nq} ({time.time() - t0:.1f}s)")
    t0 = time.time()
    torch.cuda.synchronize()
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1,
                         keep_bf16=True, keep_fp8=True)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    info = ix.info()
    log(f"[rank {rank}] index built in {build_s:.1f}s: {info}")
    q_dev = torch.from_numpy(queries).cuda()
    data_dev = torch.from_numpy(data).cuda()
    truth = exact_knn_blocked(torch, data_dev, q_dev, data, queries, kmax)
    del data_dev
    torch.cuda.empty_cache()
    truth_d = np.sqrt(((data[truth].astype(np.float64) - queries[:, None, :].astype(np.float64)) ** 2).sum(-1))
    sel10 = ks >= 10

    def recall_fn(ids, k):
        return recall_at(ids[sel10], truth[sel10], K)

    srch = Searcher(torch, ix, q_dev, n, ks=ks, kmax=kmax)
    targets = {"r0.95": (None, RECALL_TARGET)}
    calib = {}
    for form in ("fp32", HEADLINE):
        calib[form] = calibrate(srch, form, SHORTLIST_MULTS.get(form, [1]), targets, recall_fn,
                                f"rank {rank} {w.name}")["r0.95"]
    # the other precision forms (FP32 centroid distances, like the plain path) at the plain
    # FP32 form's (alpha, beta), over their shortlists
    for form in ("bf16", "fp8"):
        pts = []
        for mult in SHORTLIST_MULTS[form]:
            op = {k_: calib["fp32"][k_] for k_ in ("alpha", "beta")}
            ms = float(np.median(srch.timed(form, op["alpha"], op["beta"], mult, 3)))
            pts.append(dict(op, shortlist_mult=mult, recall=round(recall_fn(srch.ids(), K), 4),
                            qps=round(nq / (ms * 1e-3), 1)))
        ok = [p_ for p_ in pts if p_["recall"] >= RECALL_TARGET]
        calib[form] = max(ok, key=lambda p_: p_["qps"]) if ok else max(pts, key=lambda p_: p_["recall"])

    # autotune the launch layout at each compared form's operating point (the tuner takes one
    # parameter struct: the batch's largest k at the point's budget and target)
    tune = {}
    for form in ("fp32", HEADLINE):
        op = calib[form]
        if args.count_layout:
            spc, warps, unroll = (int(x) for x in args.count_layout.split(","))
            ix.set_count_layout(slabs_per_range=spc, count_warps=warps, walk_unroll=unroll)
            tune[form] = {"slabs_per_range": spc, "n_ranges": -(-info["n_slabs"] // spc),
                          "count_warps": warps, "walk_unroll": unroll, "forced": True}
            continue
        tune[form] = ix.autotune(q_dev, kmax, budget_from_alpha(op["alpha"], n),
                                 target_from_beta(op["beta"], n), shortlist_mult=op["shortlist_mult"],
                                 reps=3, **FORMS[form])
    log(f"[rank {rank}] autotune: {tune}")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)   # nvidia-smi is sampling before the timed region starts
    res = {}
    for form in (HEADLINE, "fp32", "bf16", "fp8"):
        total, per, kt = run_steps(torch, srch, ix, form, calib[form], args.steps, args.warmup, True, ws)
        ids_np, d_np = srch.ids(), srch.out_d.cpu().numpy()
        res[form] = {"total": total, "per": per, "kt": kt, "recall": recall_fn(ids_np, K),
                     "recall_own_k": recall_per_query_k(ids_np, truth, ks),
                     "mre": mre_of(d_np, truth_d, ks)}
    clk = clocks.stop()
    device_status = ix.device_status()
    tots = max_over_ranks([res[f]["total"] for f in (HEADLINE, "fp32", "bf16", "fp8")], ws, device="cuda")
    for f, tot in zip((HEADLINE, "fp32", "bf16", "fp8"), tots):
        res[f]["qps"] = ws * nq * args.steps / (tot * 1e-3)
        res[f]["total"] = tot
    value, value_fp32 = res[HEADLINE]["qps"], res["fp32"]["qps"]

    # ---- end to end through the C ABI with host buffers: pinned queries in, per-query
    # parameters as host records (converted and copied by the call), results back ----------
    op = calib[HEADLINE]
    pq_host = query_param_array(srch.per_query(HEADLINE, op["alpha"], op["beta"], op["shortlist_mult"]))
    q_host = torch.from_numpy(queries).pin_memory()
    o_ids = torch.empty((nq, kmax), dtype=torch.int64).pin_memory()
    o_d = torch.empty((nq, kmax), dtype=torch.float32).pin_memory()
    qh, oi, od = q_host.numpy(), o_ids.numpy(), o_d.numpy()
    for _ in range(max(1, args.warmup)):
        ix.search(qh, K, 1, 0, per_query=pq_host, k_stride=kmax, out_ids=oi, out_dists=od, **FORMS[HEADLINE])
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ix.search(qh, K, 1, 0, per_query=pq_host, k_stride=kmax, out_ids=oi, out_dists=od, **FORMS[HEADLINE])
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks([e2e_s], ws, device="cuda")[0]
    e2e_recall = recall_fn(oi, K)

    # ---- roofline of the dominant kernel ----------------------------------------------
    pq_dbg = srch.per_query(HEADLINE, op["alpha"], op["beta"], op["shortlist_mult"])
    dbg = ix.search_debug(q_dev, K, 1, 0, per_query=pq_dbg, k_stride=kmax, want_sc=False,
                          **FORMS[HEADLINE])
    torch.cuda.synchronize()
    retrieved = int(dbg["retrieved_num"].sum().item())
    ncells = int(dbg["probed"].sum(dtype=torch.int64).item())
    cand = int(dbg["candidate_num"].sum().item())
    entries = int(dbg["collision_num"][:, 2:].sum().item())   # ids with SC >= 2 (level lists)
    del dbg
    kt_b = res[HEADLINE]["kt"]
    alg = algorithmic_bytes(nq, retrieved, ncells, cand, entries, d=w.d, d_pad=info["d_pad"], k=ks,
                            mult=op["shortlist_mult"], n_ranges=tune[HEADLINE]["n_ranges"],
                            n_subspaces=w.n_subspaces, sqrt_k=w.sqrt_k)
    path_bytes = alg.pop("path")
    dominant = max((k_ for k_ in kt_b if kt_b[k_]["launches"]), key=lambda k_: kt_b[k_]["ms"])
    kk_ = kt_b[dominant]
    launch_ms = kk_["ms"] / max(kk_["launches"], 1)
    peak, peak_kind = measured_peaks()
    alg_bytes = alg.get(dominant, 0)
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    shares = {name: round(v["ms"] / max(sum(x["ms"] for x in kt_b.values()), 1e-9), 4)
              for name, v in kt_b.items() if v["launches"]}

    def kms(form):
        return {k_: round(v["ms"] / max(args.steps, 1), 4) for k_, v in res[form]["kt"].items() if v["launches"]}

    per_b, per_f = res[HEADLINE]["per"], res["fp32"]["per"]
    forms_out = {}
    for f in (HEADLINE, "fp32", "bf16", "fp8"):
        forms_out[f] = {"qps": round(res[f]["qps"], 1), "recall_at_10": round(res[f]["recall"], 4),
                        "recall_at_own_k": round(res[f]["recall_own_k"], 4), "mre": round(res[f]["mre"], 6),
                        "alpha": calib[f]["alpha"], "beta": calib[f]["beta"],
                        "shortlist_mult": calib[f]["shortlist_mult"],
                        "batch_ms_p50": round(float(np.percentile(res[f]["per"], 50)), 4),
                        "batch_ms_p99": round(float(np.percentile(res[f]["per"], 99)), 4),
                        "kernel_ms_per_step": kms(f)}
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(res[HEADLINE]["total"] / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "form": "batched BF16: BF16 candidate rows with an exact FP32 re-rank of each query's "
                "shortlist, query x centroid block on tcgen05 (BF16 operands, FP32 accumulation), "
                "per-query k and parameters resident on the device; fp32_qps = the plain FP32 path "
                "(FP32 rows, FP32 centroid distances on CUDA cores) on the same batches",
        "data": "synthetic (seeded stand-in for Yandex DEEP10M: unit-normalised 4096-component "
                "Gaussian mixture)",
        "config": {"workload": f"deep10m-like batched uneven form: n={n:,} d={w.d} unit-normalised GMM, "
                               f"batches of {nq:,} queries, per-query k drawn from {{1,10,50,100}}, "
                               f"query-aware budgets (Alg. 4 cell granularity, Alg. 5 per-query |C|), "
                               f"N_s={w.n_subspaces}, s={w.sub_dim}, sqrtK={w.sqrt_k}",
                   "global_batch": ws * nq, "parallelism": f"replicas x{ws}",
                   "l2": f"inputs larger than L2 ({n * info['d_pad'] * 4 / 1e9:.2f} GB FP32 / "
                         f"{n * info['d_pad'] * 2 / 1e9:.2f} GB BF16 rows, {n * w.n_subspaces * 4 / 1e6:.0f} MB "
                         f"of cell id lists)",
                   "recall": "recall@10 over the queries with k >= 10 against exact k-NN",
                   "operating_point": calib},
        "recall_at_10": {f: round(res[f]["recall"], 4) for f in res},
        "fp32_qps": round(value_fp32, 1),
        "bf16_over_fp32": round(value / value_fp32, 3),
        "precision_forms": forms_out,
        "latency_ms": {"batch": nq,
                       "p50": round(float(np.percentile(per_b, 50)), 4),
                       "p99": round(float(np.percentile(per_b, 99)), 4),
                       "fp32_p50": round(float(np.percentile(per_f, 50)), 4),
                       "fp32_p99": round(float(np.percentile(per_f, 99)), 4)},
        "e2e": {"value": round(ws * nq * args.steps / e2e_s, 1), "unit": "queries/s",
                "h2d_bytes_per_step": int(queries.nbytes + nq * 24),
                "d2h_bytes_per_step": int(nq * kmax * (8 + 4)),
                "recall_at_10": round(e2e_recall, 4),
                "path": "taco_search_batch with host queries, host per-query records and host "
                        "outputs (pinned): record conversion, copies in and out and the "
                        "kernels inside the timed region"},
        "gpu_launches": int(sum(v["launches"] for v in kt_b.values())),   # headline timed region
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic(dominant, "bf16", w.name), "peak_kind": peak_kind,
                     "limiter": ncu_limiter(dominant, w.name),
                     "kernel": f"{dominant} ({HEADLINE} form)",
                     "algorithmic_bytes_per_launch": int(alg_bytes),
                     "launch_ms": round(launch_ms, 4),
                     # count_lists work per query: one shared-memory counter atomic per
                     # retrieved id, one level-list append per id reaching SC >= 2
                     "smem_atomics_per_query": round(retrieved / nq, 1),
                     "list_entries_per_query": round(entries / nq, 1),
                     "candidates_per_query": round(cand / nq, 1),
                     "kernel_share": shares},
        # the whole path against HBM: the method's algorithmic bytes per query (ids of the
        # probed cells, their offsets, the candidate rows at the form's width, the exact
        # shortlist rows, the query and the results) x queries per second
        "path_roofline": {"bytes_per_query": round(path_bytes / nq, 1),
                          "achieved": round(path_bytes / nq * value / 1e9, 1), "peak": peak,
                          "unit": "GB/s", "frac": round(path_bytes / nq * value / 1e9 / peak, 4)},
        "build_s": {"deep10m": round(build_s, 3)},
        "clocks": clk,
        "autotune": tune,
        "device_status": device_status,   # 0: no bounded device wait gave up
    }
    srch.close()
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(ix, data, queries, w, calib["fp32"], args.cpu_seconds)
        line["cpu_baseline"]["sample"] += "; k = 10 for every sampled query"
    ix.close()
    del data, queries, q_dev
    torch.cuda.empty_cache()
    if not args.no_extra:
        extra = run_sift_extra(args, ws, rank, local)
        line["sift1m"] = extra
        line["build_s"]["sift1m"] = extra.pop("build_s")
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sift_extra(args, ws, rank, local):
    """The 1M x 128 workload (plain FP32 method config): each compared form's operating point
    at recall@10 >= 0.9 / 0.95 / 0.99, recall@1 >= 0.95 (k = 1) and recall@100 >= 0.95
    (k = 100), each timed at its own k, plus the serving loop at the k = 10, 0.95 point."""
    import torch
    from paper_2603_24919_gb300 import TacoIndex
    from synth import make_workload

    nq_rank = args.nq_extra
    w, data, pool = make_workload(EXTRA_WORKLOAD, nq=nq_rank * ws)
    lo, hi = shard(pool.shape[0], ws, rank)
    queries = np.ascontiguousarray(pool[lo:hi])
    del pool
    nq, n = queries.shape[0], w.n
    t0 = time.time()
    torch.cuda.synchronize()
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1,
                         keep_bf16=True)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    q_dev = torch.from_numpy(queries).cuda()
    data_dev = torch.from_numpy(data).cuda()
    truth = exact_knn_gpu(torch, data_dev, q_dev, data, queries, 100)
    del data_dev
    torch.cuda.empty_cache()
    srch = Searcher(torch, ix, q_dev, n, ks=None, kmax=100)
    targets = {"k10_r0.95": (10, 0.95), "k10_r0.9": (10, 0.9), "k10_r0.99": (10, 0.99),
               "k1_r0.95": (1, 0.95), "k100_r0.95": (100, 0.95)}

    def recall_fn(ids, k):
        return recall_at(ids, truth, k)

    out = {"workload": f"sift1m-like: n={n:,} d={w.d} integer GMM, {nq:,} queries per batch, "
                       f"N_s={w.n_subspaces}, s={w.sub_dim}, sqrtK={w.sqrt_k}",
           "build_s": round(build_s, 3), "forms": {}}
    ops = {}
    for form in ("fp32", HEADLINE):
        ops[form] = calibrate(srch, form, SHORTLIST_MULTS.get(form, [1]), targets, recall_fn,
                              f"rank {rank} sift1m")
        out["forms"][form] = {}
        for t, op in ops[form].items():
            k = targets[t][0]
            per = srch.timed(form, op["alpha"], op["beta"], op["shortlist_mult"], max(args.steps // 4, 5), k)
            out["forms"][form][t] = dict(op, qps=round(nq / (float(np.mean(per)) * 1e-3), 1),
                                         batch_ms_p50=round(float(np.percentile(per, 50)), 4),
                                         batch_ms_p99=round(float(np.percentile(per, 99)), 4),
                                         recall=round(recall_fn(srch.ids(), k), 4))
    out["bf16_over_fp32"] = {t: round(out["forms"][HEADLINE][t]["qps"] / out["forms"]["fp32"][t]["qps"], 3)
                             for t in targets}
    srch.close()
    if not args.no_serving:
        from synth import budget_from_alpha, target_from_beta
        op = ops[HEADLINE]["k10_r0.95"]
        out["serving"] = run_serving(ix, queries, truth, budget_from_alpha(op["alpha"], n),
                                     target_from_beta(op["beta"], n), op["shortlist_mult"],
                                     args.serve_seconds)
    ix.close()
    return out


def run_serving(ix, queries, truth, bud, tgt, mult, span_s):
    """Open-loop Poisson arrivals through the continuous-batching server (taco_server_*,
    BF16 rows at the BF16 operating point): per offered load, achieved QPS and p50/p99
    latency (arrival to results in host memory), and recall@10 of the served answers.
    The mixed load draws k from {10, 100} per request."""
    from paper_2603_24919_gb300 import TacoServer, query_params

    rng = np.random.default_rng(1234)
    nq = queries.shape[0]
    kmax = 100
    max_list = min(mult * kmax, 512)
    out = []
    with TacoServer(ix, max_batch=2048, slots=4, queue_capacity=16384, max_list=max_list,
                    precision="bf16", max_wait_us=100, use_graphs=True,
                    probe_precision=FORMS[HEADLINE].get("probe_precision", "fp32")) as srv:
        def one(rate, mixed, n_req=None):
            n_req = n_req or max(2000, int(rate * span_s))
            rows = np.arange(n_req) % nq
            ks = rng.choice([10, 100], size=n_req) if mixed else np.full(n_req, 10)
            per = [query_params(int(k), bud, tgt, "bf16", "literal", mult,
                                FORMS[HEADLINE].get("probe_precision", "fp32")) for k in ks]
            arrival = np.cumsum(rng.exponential(1e9 / rate, size=n_req)).astype(np.int64)
            ids, _, lat = srv.replay(queries[rows], per, arrival, kmax)
            span = float(np.max(arrival + lat) - arrival[0]) * 1e-9
            sel = ks == 10
            return {"offered_qps": rate, "requests": int(n_req), "mixed_k": bool(mixed),
                    "achieved_qps": round(n_req / span, 1),
                    "p50_ms": round(float(np.percentile(lat, 50)) * 1e-6, 4),
                    "p99_ms": round(float(np.percentile(lat, 99)) * 1e-6, 4),
                    "recall_at_10": round(recall_at(ids[sel], truth[rows[sel]], K), 4)}
        one(500_000, True, n_req=20_000)   # warm-up: graphs for the batch buckets
        for rate in (10_000, 100_000, 200_000, 500_000, 1_000_000, 2_000_000):
            out.append(one(rate, False))
        out.append(one(200_000, True))
        st = srv.stats()
    return {"server": "max_batch 2048, 4 slots, max_wait 100 us, CUDA graphs, BF16 rows, "
                      "tcgen05 centroid block",
            "loads": out, "batches": st["batches"], "graph_launches": st["graph_launches"],
            "max_in_flight": st["max_in_flight"],
            "mean_batch": round(st["completed"] / max(st["batches"], 1), 1)}


def cpu_baseline(ix, data, queries, w, op, seconds):
    """The FP64 oracle's query routine (Alg. 6) on the host cores, over the same index
    (exported from the library), data and queries, for a bounded sample of queries."""
    ex = ix.export()
    parts = {k: ex[k] for k in ("o_bar", "B", "centroids", "codes")}
    return cpu_baseline_parts(parts, data, queries, (w.n_subspaces, w.sub_dim, w.sqrt_k), op,
                              seconds)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:   # pragma: no cover
        return os.cpu_count() or 1


def _oracle_worker(tmpdir, geom, k, bud, tgt, inq, out):
    """One process of the oracle pool: builds the oracle index from the parts saved in
    tmpdir, reports ready, then answers tasks from inq until None:
      ("deadline", start, stride, seconds): queries start, start + stride, ... for `seconds`;
      ("list", indices): those queries.
    Each task reports (queries answered, seconds, error or None)."""
    try:
        import numpy as np_
        from oracle import taco_oracle as O
        ld = lambda name: np_.load(os.path.join(tmpdir, name + ".npy"), mmap_mode="r")
        oix = O.index_from_parts(ld("o_bar"), ld("B"), ld("centroids"), ld("codes"), *geom)
        data, queries = ld("data"), ld("queries")
    except Exception as e:   # reported to the parent
        out.put(("ready", repr(e)))
        return
    out.put(("ready", None))
    while True:
        task = inq.get()
        if task is None:
            return
        try:
            t0 = time.perf_counter()
            done = 0
            if task[0] == "deadline":
                _, j, stride, seconds = task
                while j < len(queries) and time.perf_counter() - t0 < seconds:
                    O.search_one(oix, data, np_.asarray(queries[j]), k, bud, tgt)
                    done += 1
                    j += stride
            else:
                for j in task[1]:
                    O.search_one(oix, data, np_.asarray(queries[j]), k, bud, tgt)
                    done += 1
            out.put(("done", done, time.perf_counter() - t0, None))
        except Exception as e:
            out.put(("done", 0, 0.0, repr(e)))


class OraclePool:
    """`procs` spawned processes answering queries with the FP64 oracle's query routine, one
    NumPy thread each, over one index whose parts (and the data and queries) are shared
    through memory-mapped files. Raises RuntimeError if a process fails or times out."""

    def __init__(self, parts, data, queries, geom, bud, tgt, procs, setup_timeout=300.0):
        import multiprocessing as mp
        import tempfile

        self.procs = procs
        self.tmpdir = tempfile.mkdtemp(prefix="taco_oracle_")
        self.ps, self.inqs = [], []
        try:
            for name, arr in list(parts.items()) + [("data", data), ("queries", queries)]:
                np.save(os.path.join(self.tmpdir, name + ".npy"), np.ascontiguousarray(arr))
            ctx = mp.get_context("spawn")
            self.out = ctx.Queue()
            saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                    "MKL_NUM_THREADS")}
            os.environ.update({v: "1" for v in saved})
            try:
                for _ in range(procs):
                    q = ctx.Queue()
                    p = ctx.Process(target=_oracle_worker,
                                    args=(self.tmpdir, geom, K, bud, tgt, q, self.out), daemon=True)
                    p.start()
                    self.ps.append(p)
                    self.inqs.append(q)
            finally:
                for v, old in saved.items():
                    if old is None:
                        os.environ.pop(v, None)
                    else:
                        os.environ[v] = old
            for _ in range(procs):
                msg = self._get(setup_timeout)
                if msg[1] is not None:
                    raise RuntimeError(f"oracle process setup failed: {msg[1]}")
        except BaseException:
            self.close()
            raise

    def _get(self, timeout):
        import queue as queue_mod
        try:
            return self.out.get(timeout=timeout)
        except queue_mod.Empty:
            raise RuntimeError("oracle process did not answer in time") from None

    def run(self, tasks, timeout):
        """One task per process, all dispatched at once; returns (answered, longest time)."""
        for q, t in zip(self.inqs, tasks):
            q.put(t)
        res = [self._get(timeout) for _ in tasks]
        errs = [r[3] for r in res if r[3]]
        if errs:
            raise RuntimeError(f"oracle process failed: {errs[0]}")
        return sum(r[1] for r in res), max(r[2] for r in res)

    def close(self):
        import shutil
        for q in self.inqs:
            try:
                q.put(None)
            except Exception:
                pass
        for p in self.ps:
            p.join(timeout=5)
            if p.is_alive():
                p.kill()
        self.ps, self.inqs = [], []
        shutil.rmtree(self.tmpdir, ignore_errors=True)


def cpu_baseline_parts(parts, data, queries, geom, op, seconds, procs=None):
    """Time the oracle's query routine in `procs` spawned processes (default: every host core
    this process may run on), queries dealt round-robin, all started together and run for
    `seconds`. QPS = queries answered / the longest process time. Falls back to this process
    alone if the pool cannot run."""
    from synth import budget_from_alpha, target_from_beta

    n = parts["codes"].shape[1]
    bud, tgt = budget_from_alpha(op["alpha"], n), target_from_beta(op["beta"], n)
    procs = procs or host_cores()
    what = f"fp32 operating point alpha={op['alpha']} beta={op['beta']}, NumPy FP64"
    if procs > 1:
        try:
            pool = OraclePool(parts, data, queries, geom, bud, tgt, procs)
            try:
                done, el = pool.run([("deadline", r, procs, seconds) for r in range(procs)],
                                    timeout=seconds + 120)
            finally:
                pool.close()
            return {"value": round(done / el, 3), "unit": "queries/s", "cores": procs,
                    "kind": "oracle",
                    "sample": f"{done} of {len(queries)} queries dealt round-robin to {procs} "
                              f"processes for {seconds:.0f} s, {what}, one thread each"}
        except Exception as e:   # any failure of the pool: the single-process timing below
            log(f"cpu baseline: process pool failed ({e!r}); timing one process")
    from oracle import taco_oracle as O
    oix = O.index_from_parts(parts["o_bar"], parts["B"], parts["centroids"], parts["codes"], *geom)
    t0 = time.perf_counter()
    done = 0
    while done < len(queries) and time.perf_counter() - t0 < seconds:
        O.search_one(oix, data, queries[done], K, bud, tgt)
        done += 1
    el = time.perf_counter() - t0
    return {"value": round(done / el, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(queries)} queries, {what}, single process"}


# ------------------------------------------------------------------------ reference arm
def _kmeans_job(args):
    from oracle import taco_oracle as O
    cols, sk, iters, seed = args
    return O.kmeans(cols, sk, iters, seed)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp

    from oracle import taco_oracle as O
    from synth import budget_from_alpha, make_workload, target_from_beta

    t0 = time.time()
    w, data, queries = make_workload(args.workload, nq=args.nq)
    # the oracle's own index (Alg. 1-3 in FP64); k-means halves run in a spawn pool
    mu, sigma = O.mean_and_covariance(data)
    lam, xi = O.spectral_decomposition(sigma)
    buckets, _ = O.eigensystem_allocation(lam, w.n_subspaces, w.sub_dim)
    B = O.transform_matrix(xi, buckets)
    T = O.transform(data, mu, B)
    h1, _ = O.half_dims(w.sub_dim)
    jobs = []
    for i in range(w.n_subspaces):
        Ti = T[:, i * w.sub_dim:(i + 1) * w.sub_dim]
        jobs.append((np.ascontiguousarray(Ti[:, :h1]), w.sqrt_k, 20, 1 * 7919 + 2 * i))
        jobs.append((np.ascontiguousarray(Ti[:, h1:]), w.sqrt_k, 20, 1 * 7919 + 2 * i + 1))
    del T
    cores = os.cpu_count() or 1
    with ProcessPoolExecutor(max_workers=min(cores, len(jobs)),
                             mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_kmeans_job, jobs))
    cent = np.zeros((w.n_subspaces, w.sqrt_k, w.sub_dim))
    codes = np.zeros((w.n_subspaces, w.n), dtype=np.int64)
    for i in range(w.n_subspaces):
        (c1, a1), (c2, a2) = res[2 * i], res[2 * i + 1]
        cent[i, :, :h1], cent[i, :, h1:] = c1, c2
        codes[i] = a1 * w.sqrt_k + a2
    oix = O.index_from_parts(mu, B, cent, codes, w.n_subspaces, w.sub_dim, w.sqrt_k)
    log(f"[reference] oracle index built in {time.time() - t0:.1f}s")
    # the oracle is not calibrated itself: a fixed operating point near the one the GPU
    # calibration selects on the workload (its per-query cost barely depends on it)
    ref_a, ref_b = REFERENCE_OP.get(args.workload, (w.alpha, w.beta))
    alpha, beta = (args.alpha or ref_a), (args.beta or ref_b)
    bud, tgt = budget_from_alpha(alpha, w.n), target_from_beta(beta, w.n)
    per_step = max(1, int(os.environ.get("TACO_REF_QUERIES_PER_STEP", "2")))   # per process
    procs = host_cores()
    nqs = len(queries)
    pool = None
    if procs > 1:
        try:
            pool = OraclePool({"o_bar": mu, "B": B, "centroids": cent, "codes": codes}, data, queries,
                              (w.n_subspaces, w.sub_dim, w.sqrt_k), bud, tgt, procs)
        except Exception as e:   # any failure of the pool: time this process alone
            log(f"[reference] process pool failed ({e!r}); timing one process")
            procs, pool = 1, None
    def measure(pool, procs):
        times, qi = [], 0
        for step in range(args.warmup + args.steps):
            if pool is not None:   # per_step queries in each process, all dispatched at once
                tasks = [("list", [(qi + r * per_step + j) % nqs for j in range(per_step)])
                         for r in range(procs)]
                t1 = time.perf_counter()
                pool.run(tasks, timeout=600)
                el = time.perf_counter() - t1
            else:
                t1 = time.perf_counter()
                for j in range(per_step):
                    O.search_one(oix, data, queries[(qi + j) % nqs], K, bud, tgt)
                el = time.perf_counter() - t1
            qi += procs * per_step
            if step >= args.warmup:
                times.append(el)
        return times

    try:
        times = measure(pool, procs)
    except Exception as e:   # a pool process failed: time this process alone
        log(f"[reference] process pool failed ({e!r}); timing one process")
        pool.close()
        procs, pool = 1, None
        times = measure(None, 1)
    finally:
        if pool is not None:
            pool.close()
    total = sum(times)
    value = args.steps * procs * per_step / total
    sample = (f"{per_step} queries per process and step ({procs} processes, one NumPy thread "
              f"each) of the {nqs}-query batch, alpha={alpha} beta={beta}, FP64 oracle")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "queries/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": (f"{w.name}: n={w.n:,} d={w.d}, nq={nqs:,} per batch, k={K} for every "
                                f"sampled query, N_s={w.n_subspaces}, s={w.sub_dim}, sqrtK={w.sqrt_k}"),
                   "parallelism": "host cores"},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 3), "unit": "queries/s", "cores": procs,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def exact_knn_blocked(torch, data_t, queries_t, data_np, queries_np, k, extra=32, qchunk=256,
                      dchunk=1 << 20):
    """Exact k-NN for recall on large n: FP32 brute force over data blocks with a running
    top-(k+extra) per query, then FP64 re-check of that pool on the host."""
    xn = (data_t * data_t).sum(1)
    out = np.empty((queries_t.shape[0], k), dtype=np.int64)
    for a in range(0, queries_t.shape[0], qchunk):
        q = queries_t[a:a + qchunk]
        qn = (q * q).sum(1, keepdim=True)
        best_d, best_i = None, None
        for b in range(0, data_t.shape[0], dchunk):
            d2 = qn - 2.0 * (q @ data_t[b:b + dchunk].T) + xn[None, b:b + dchunk]
            v, i = torch.topk(d2, min(k + extra, d2.shape[1]), dim=1, largest=False)
            i = i + b
            if best_d is None:
                best_d, best_i = v, i
            else:
                cd, ci = torch.cat([best_d, v], 1), torch.cat([best_i, i], 1)
                v2, j = torch.topk(cd, k + extra, dim=1, largest=False)
                best_d, best_i = v2, torch.gather(ci, 1, j)
        pool = best_i.cpu().numpy()
        qq = queries_np[a:a + qchunk].astype(np.float64)
        for j in range(pool.shape[0]):
            cand = pool[j]
            dd = ((data_np[cand].astype(np.float64) - qq[j]) ** 2).sum(1)
            out[a + j] = cand[np.lexsort((cand, dd))[:k]]
    return out


def _workload_spec(name):
    from synth import WORKLOADS
    return WORKLOADS[name]


def recall_per_query_k(ids, truth, ks):
    """Mean recall@k_q over queries, each at its own k."""
    hits = [len(set(ids[j, :k].tolist()) & set(truth[j, :k].tolist())) / k for j, k in enumerate(ks)]
    return float(np.mean(hits))


WORKLOAD_FORMS = {
    # every row form with and without the tcgen05 query x centroid block
    "gist1m": {"fp32": dict(precision="fp32"), "fp32_tc": dict(precision="fp32", probe_precision="bf16"),
               "bf16": dict(precision="bf16"), "bf16_tc": dict(precision="bf16", probe_precision="bf16"),
               "fp8": dict(precision="fp8"), "fp8_tc": dict(precision="fp8", probe_precision="fp8")},
    "deep5m256": {"fp32": dict(precision="fp32"), "bf16_tc": dict(precision="bf16", probe_precision="bf16")},
}
WORKLOAD_MULTS = {"fp32": [1], "fp32_tc": [1], "bf16": [1, 2], "bf16_tc": [1, 2], "fp8": [2, 4], "fp8_tc": [2, 4]}
# (alpha, beta) grids: the 5M x 256 grid reaches below the paper's alpha range (recall@10
# saturates early on that stand-in); the 1M x 960 grid spans the paper's ranges
WORKLOAD_GRIDS = {
    "deep5m256": [(a, b) for a in (0.0002, 0.0005, 0.001, 0.002, 0.005, 0.01, 0.02, 0.05)
                  for b in (0.0001, 0.0002, 0.0005, 0.001, 0.002, 0.005)],
    "gist1m": [(a, b) for a in (0.002, 0.005, 0.01, 0.02, 0.05, 0.1)
               for b in (0.0005, 0.001, 0.002, 0.005, 0.01, 0.02)],
}


def run_workload(args):
    """One JSON line for another workload: gist1m (precision form: recall@10 and MRE of the
    FP32, BF16 and FP8 rows, each with the SIMT and the tcgen05 query x centroid block, at the
    fastest grid point with recall@10 >= 0.95) or deep5m256 (serving form: the BF16 and FP32
    servers under Poisson arrivals, mixed k in {10, 100}, recall targets 0.9 / 0.99 each
    mapped to the form's own fastest grid point meeting it)."""
    import torch
    from paper_2603_24919_gb300 import TacoIndex, TacoServer, build_lib, query_params
    from synth import budget_from_alpha, make_workload, target_from_beta

    torch.cuda.set_device(0)
    build_lib.build()
    name = args.workload
    if name not in WORKLOAD_FORMS:
        raise SystemExit(f"--workload {name}: the 10M x 96 headline runs without --workload; "
                         f"others: {sorted(WORKLOAD_FORMS)}")
    t0 = time.time()
    w, data, queries = make_workload(name, nq=args.nq)
    nq, n = queries.shape[0], data.shape[0]
    log(f"[{name}] n={n} d={w.d} nq={nq} generated in {time.time() - t0:.1f}s")
    t0 = time.time()
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1,
                         keep_bf16=True, keep_fp8=(name == "gist1m"))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    log(f"[{name}] index built in {build_s:.1f}s: {ix.info()}")
    q_dev = torch.from_numpy(queries).cuda()
    data_dev = torch.from_numpy(data).cuda()
    kmax = 100
    truth = exact_knn_blocked(torch, data_dev, q_dev, data, queries, kmax)
    del data_dev
    torch.cuda.empty_cache()
    truth_d = np.sqrt(((data[truth].astype(np.float64) - queries[:, None, :].astype(np.float64)) ** 2).sum(-1))
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(4242)
    forms = dict(WORKLOAD_FORMS[name])
    grid = WORKLOAD_GRIDS[name]
    ks = np.full(nq, K)

    def per(form, a, b):
        return [dict(k=int(k), budget=budget_from_alpha(a, n), rerank_target=target_from_beta(b, n),
                     **form) for k in ks]

    def timed(form, a, b, reps):
        pq = per(form, a, b)
        ids, d = ix.search(q_dev, K, 1, 0, per_query=pq, k_stride=K, **form)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        evs[0].record(stream)
        for r in range(reps):
            ids, d = ix.search(q_dev, K, 1, 0, per_query=pq, k_stride=K, **form)
            evs[r + 1].record(stream)
        torch.cuda.synchronize()
        per_ms = [evs[r].elapsed_time(evs[r + 1]) for r in range(reps)]
        ids, d = ids.cpu().numpy(), d.cpu().numpy()
        return (recall_at(ids, truth, K), mre_of(d, truth_d, ks), nq / (np.mean(per_ms) * 1e-3), per_ms)

    def fastest(form, target, mults, reps=2):
        best = None
        for mult in mults:
            f = dict(form, shortlist_mult=mult)
            for a, b in grid:
                r10, _, qps, _ = timed(f, a, b, reps)
                if r10 >= target and (best is None or qps > best["qps"]):
                    best = {"alpha": a, "beta": b, "recall_at_10": r10, "qps": qps, "mult": mult}
        return best

    out = {}
    for fname in list(forms):
        best = fastest(forms[fname], RECALL_TARGET, WORKLOAD_MULTS[fname])
        met = best is not None
        if best is None:
            best = {"alpha": grid[-1][0], "beta": grid[-1][1], "mult": WORKLOAD_MULTS[fname][-1]}
        a, b = best["alpha"], best["beta"]
        form = forms[fname] = dict(forms[fname], shortlist_mult=best["mult"])
        tune = ix.autotune(q_dev, K, budget_from_alpha(a, n), target_from_beta(b, n), reps=2, **form)
        r10, mre, qps, per_ms = timed(form, a, b, max(args.steps // 5, 5))
        out[fname] = {"alpha": a, "beta": b, "shortlist_mult": best["mult"], "met": met,
                      "on_grid_edge": (a, b) in (grid[0], grid[-1]),
                      "qps": round(float(qps), 1), "recall_at_10": round(r10, 4), "mre": round(mre, 6),
                      "batch_ms_p50": round(float(np.percentile(per_ms, 50)), 3),
                      "batch_ms_p99": round(float(np.percentile(per_ms, 99)), 3),
                      "autotune": {k_: tune[k_] for k_ in ("slabs_per_range", "lanes_per_row",
                                                           "count_warps", "walk_unroll")}}
        log(f"[{name}] {fname}: {out[fname]}")
    serving = None
    if name == "deep5m256":
        serving = {"server": "max_batch 2048, 4 slots, max_wait 100 us, CUDA graphs", "targets": {}, "loads": {}}
        for fname in ("bf16_tc", "fp32"):
            # each recall target mapped to the form's own fastest grid point meeting it on k = 10
            # (alpha, beta, shortlist multiple) per target; the FP32 rows have no shortlist
            targets = {}
            for tgt_r in (0.9, 0.99):
                best = fastest(forms[fname], tgt_r, WORKLOAD_MULTS[fname], reps=1)
                targets[tgt_r] = (best["alpha"], best["beta"], best["mult"]) if best else grid[-1] + (1,)
            serving["targets"][fname] = {str(t): v for t, v in targets.items()}
            form = forms[fname]
            max_list = kmax if form["precision"] == "fp32" else min(max(v[2] for v in targets.values()) * kmax, 512)
            with TacoServer(ix, max_batch=2048, slots=4, queue_capacity=16384, max_list=max_list,
                            precision=form["precision"], max_wait_us=100,
                            probe_precision=form.get("probe_precision", "fp32")) as srv:
                loads = []
                for rate in (10_000, 100_000, 200_000):
                    n_req = max(2000, int(rate * args.serve_seconds))
                    rows = np.arange(n_req) % nq
                    kq = rng.choice([10, 100], size=n_req)
                    tq = rng.choice([0.9, 0.99], size=n_req)
                    pq = [query_params(int(k), budget_from_alpha(targets[t][0], n),
                                       target_from_beta(targets[t][1], n), form["precision"],
                                       "literal", targets[t][2], form.get("probe_precision", "fp32"))
                          for k, t in zip(kq, tq)]
                    arrival = np.cumsum(rng.exponential(1e9 / rate, size=n_req)).astype(np.int64)
                    ids, _, lat = srv.replay(queries[rows], pq, arrival, kmax)
                    span = float(np.max(arrival + lat) - arrival[0]) * 1e-9
                    rec = {str(t): round(recall_per_query_k(ids[tq == t], truth[rows[tq == t]],
                                                            kq[tq == t]), 4) for t in (0.9, 0.99)}
                    loads.append({"offered_qps": rate, "achieved_qps": round(n_req / span, 1),
                                  "p50_ms": round(float(np.percentile(lat, 50)) * 1e-6, 4),
                                  "p99_ms": round(float(np.percentile(lat, 99)) * 1e-6, 4),
                                  "recall_by_target": rec})
                serving["loads"][fname] = loads
                log(f"[{name}] serving {fname}: {loads}")
    head = "bf16_tc"
    line = {"metric": f"QPS at recall@10>=0.95 on the {name} workload (batched, 1 GB300)",
            "value": out[head]["qps"], "unit": "queries/s", "n_gpus": 1,
            "higher_is_better": True, "impl": "taco", "workload": name, "dtype": "bf16",
            "config": {"n": n, "d": w.d, "nq_per_batch": nq, "n_subspaces": w.n_subspaces,
                       "sub_dim": w.sub_dim, "sqrt_k": w.sqrt_k, "k": K},
            "forms": out, "bf16_over_fp32": round(out[head]["qps"] / out["fp32"]["qps"], 3),
            "mre": "mean relative error of the k returned distances against the exact (FP64) k-NN distances",
            "build_s": round(build_s, 3), "device_status": ix.device_status(), "data": "synthetic"}
    if serving is not None:
        line["serving"] = serving
    ix.close()
    print(json.dumps(line), flush=True)


def run_ncu_case(args):
    """A fixed search case for a profiler: the workload's index (row copies only for the
    form's rows), --steps searches at (--alpha, --beta) with the form's shortlist 1 (FP8: 2)."""
    import torch
    from paper_2603_24919_gb300 import TacoIndex, build_lib
    from synth import budget_from_alpha, make_workload, target_from_beta

    torch.cuda.set_device(0)
    build_lib.build()
    form = FORMS[args.ncu_case]
    name = args.workload
    w, data, queries = make_workload(name, n=args.n, nq=args.nq)
    n, nq = data.shape[0], queries.shape[0]
    prec = form["precision"]
    ix = TacoIndex.build(data, w.n_subspaces, w.sub_dim, w.sqrt_k, kmeans_iters=20, seed=1,
                         keep_bf16=prec == "bf16", keep_fp8=prec == "fp8")
    del data
    if args.count_layout:
        spc, warps, unroll = (int(x) for x in args.count_layout.split(","))
        ix.set_count_layout(slabs_per_range=spc, count_warps=warps, walk_unroll=unroll)
    if args.codes_fallback:
        ix.set_codes_fallback(True)
    q = torch.from_numpy(queries).cuda()
    a = args.alpha or REFERENCE_OP.get(name, (w.alpha, w.beta))[0]
    b = args.beta or REFERENCE_OP.get(name, (w.alpha, w.beta))[1]
    mult = 2 if prec == "fp8" else 1
    ks = np.random.default_rng(4242).choice(KS_BATCHED, size=nq) if name == WORKLOAD else np.full(nq, K)
    prep = ix.prepare([dict(k=int(k), budget=budget_from_alpha(a, n), rerank_target=target_from_beta(b, n),
                            shortlist_mult=mult, **form) for k in ks])
    for _ in range(args.steps):
        ix.search_prepared(q, prep, k_stride=int(ks.max()))
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "workload": name, "n": n, "nq": nq, "alpha": a, "beta": b,
                      "steps": args.steps, "device_status": ix.device_status()}), flush=True)
    prep.close()
    ix.close()


def main():
    args = parse()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != WORKLOAD:
        run_workload(args)
    else:
        run_taco(args)


if __name__ == "__main__":
    main()

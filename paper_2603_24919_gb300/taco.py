"""Python binding of the TaCo C ABI (include/taco.h): argument marshalling only.

Every step of index build and search runs inside libtaco.so. Device buffers are PyTorch
CUDA tensors (PyTorch provides device memory and streams); host buffers are NumPy arrays.
If libtaco.so is missing the first call raises: there is no other implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# TACO_LIB selects another build of the library (the bounds-checked libtaco_checked.so)
LIB_PATH = os.environ.get("TACO_LIB") or os.path.join(_PKG, "libtaco.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECAPACITY, EIO, EAGAIN = -1, -2, -3, -4, -5, -6, -7
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
ROWS_BF16, ROWS_FP8 = 1, 2
OPT_CODES_FALLBACK = 1
OPT_SLABS_PER_RANGE = 2
OPT_COUNT_WARPS = 3
OPT_WALK_UNROLL = 4
SELECT_LITERAL, SELECT_PROSE = 0, 1
MAX_SUBSPACES, MAX_SQRT_K, MAX_K = 15, 128, 512

_PREC = {"fp32": PREC_FP32, "bf16": PREC_BF16, "fp8": PREC_FP8}
_RULE = {"literal": SELECT_LITERAL, "prose": SELECT_PROSE}


class BuildParams(C.Structure):
    _fields_ = [("n_subspaces", C.c_int32), ("sub_dim", C.c_int32), ("sqrt_k", C.c_int32),
                ("kmeans_iters", C.c_int32), ("seed", C.c_uint64), ("keep_rows", C.c_int32),
                ("reserved", C.c_int32)]


class QueryParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("precision", C.c_int32), ("budget", C.c_int64),
                ("rerank_target", C.c_int64), ("select_rule", C.c_int32),
                ("shortlist_mult", C.c_int32), ("probe_precision", C.c_int32),
                ("reserved", C.c_int32)]


class IndexParts(C.Structure):
    _fields_ = [("o_bar", C.c_void_p), ("B", C.c_void_p), ("centroids", C.c_void_p),
                ("codes", C.c_void_p), ("n_subspaces", C.c_int32), ("sub_dim", C.c_int32),
                ("sqrt_k", C.c_int32), ("reserved", C.c_int32)]


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("n_subspaces", C.c_int32),
                ("sub_dim", C.c_int32), ("sqrt_k", C.c_int32), ("d_pad", C.c_int32),
                ("has_bf16", C.c_int32), ("n_slabs", C.c_int32), ("cluster_size", C.c_int32),
                ("has_fp8", C.c_int32), ("fp8_pitch", C.c_int32), ("has_centroid_tc", C.c_int32),
                ("reserved", C.c_int32), ("device_bytes", C.c_int64), ("n_ids", C.c_int64),
                ("build_ms_transform", C.c_double), ("build_ms_index", C.c_double)]


class DebugOut(C.Structure):
    _fields_ = [("query_t", C.c_void_p), ("probed", C.c_void_p), ("retrieved_num", C.c_void_p),
                ("sc", C.c_void_p), ("collision_num", C.c_void_p),
                ("last_collision", C.c_void_p), ("candidate_num", C.c_void_p)]


class ServerParams(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("slots", C.c_int32), ("queue_capacity", C.c_int32),
                ("max_list", C.c_int32), ("precision", C.c_int32), ("select_rule", C.c_int32),
                ("max_wait_us", C.c_int64), ("slot_bytes", C.c_int64), ("use_graphs", C.c_int32),
                ("probe_precision", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("submit_ns", C.c_int64), ("dispatch_ns", C.c_int64), ("done_ns", C.c_int64),
                ("batch_size", C.c_int32), ("slot", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("batches", C.c_int64), ("graph_launches", C.c_int64),
                ("graph_captures", C.c_int64), ("max_batch_seen", C.c_int64),
                ("max_in_flight", C.c_int64), ("slot_bytes", C.c_int64)]


class TuneResult(C.Structure):
    _fields_ = [("slabs_per_range", C.c_int32), ("n_ranges", C.c_int32),
                ("lanes_per_row", C.c_int32), ("probe_walk", C.c_int32),
                ("count_warps", C.c_int32), ("walk_unroll", C.c_int32), ("ms_before", C.c_double), ("ms_after", C.c_double), ("trials", C.c_int32),
                ("reserved", C.c_int32)]


NUM_KERNELS = 7
KERNEL_NAMES = ("project", "probe_cells", "count_lists", "select_rerank", "cluster_count_select",
                "final_merge", "centroid_tc")


class KernelTimes(C.Structure):
    _fields_ = [("launches", C.c_int64 * NUM_KERNELS), ("ms", C.c_double * NUM_KERNELS)]


# name -> (restype, argtypes); the exported symbols of include/taco.h
SIGNATURES = {
    "taco_build_index": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(BuildParams),
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "taco_index_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(IndexParts),
                                    C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "taco_search_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.POINTER(QueryParams), C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "taco_params_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "taco_params_free": (None, [C.c_void_p]),
    "taco_search_batch_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "taco_search_batch_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64,
                                            C.POINTER(QueryParams), C.c_int32, C.c_void_p,
                                            C.c_void_p, C.c_void_p]),
    "taco_shard_count": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.POINTER(QueryParams), C.c_int32, C.c_void_p,
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "taco_shard_select": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "taco_shard_free": (C.c_int, [C.c_void_p]),
    "taco_search_debug": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.POINTER(QueryParams), C.c_int32, C.c_void_p, C.c_void_p,
                                    C.POINTER(DebugOut), C.c_void_p]),
    "taco_index_get_info": (C.c_int, [C.c_void_p, C.POINTER(IndexInfo)]),
    "taco_index_lists": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "taco_index_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "taco_save_index": (C.c_int, [C.c_void_p, C.c_char_p]),
    "taco_load_index": (C.c_int, [C.c_char_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "taco_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "taco_profile_read": (C.c_int, [C.c_void_p, C.POINTER(KernelTimes), C.c_int32]),
    "taco_free_index": (None, [C.c_void_p]),
    "taco_centroid_distances": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                          C.c_void_p, C.c_void_p]),
    "taco_device_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "taco_index_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "taco_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(QueryParams),
                                C.c_int32, C.c_void_p, C.POINTER(TuneResult)]),
    "taco_server_create": (C.c_int, [C.c_void_p, C.POINTER(ServerParams), C.POINTER(C.c_void_p)]),
    "taco_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(QueryParams),
                                     C.POINTER(C.c_uint64)]),
    "taco_server_submit_many": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_void_p, C.POINTER(C.c_int64)]),
    "taco_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.POINTER(RequestInfo)]),
    "taco_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "taco_server_replay": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "taco_server_destroy": (None, [C.c_void_p]),
    "taco_last_error": (C.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtaco.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2603_24919_gb300.build_lib.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TacoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"taco error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != OK:
        msg = load_library().taco_last_error().decode(errors="replace")
        raise TacoError(rc, msg)


def _torch():
    import torch
    return torch


def _is_cuda_tensor(x):
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _max_k(arr):
    """Largest k of a QueryParams array, read as int32 words of the records (no per-record
    Python objects: a batch of thousands is read in microseconds)."""
    assert QueryParams.k.offset == 0 and C.sizeof(QueryParams) % 4 == 0
    words = np.frombuffer(arr, dtype=np.int32)
    return int(words[::C.sizeof(QueryParams) // 4].max())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _as_f32(x):
    if _is_cuda_tensor(x):
        torch = _torch()
        return x.to(torch.float32).contiguous()
    if not isinstance(x, np.ndarray):
        try:
            x = x.detach().cpu().numpy()
        except AttributeError:
            x = np.asarray(x)
    return np.ascontiguousarray(x, dtype=np.float32)


def check_noalloc_args(queries, out_ids, out_dists, d):
    """Raise ValueError unless the buffers of search_noalloc have the layout the C entry
    point reads and writes: queries float32 [nq, d], out_ids int64 and out_dists float32 with
    the same [rows >= nq, k_stride] shape, all contiguous CUDA tensors (the entry point reads
    and writes them through raw pointers, so a wrong dtype or a short buffer would be read
    with the wrong layout or written past its end)."""
    torch = _torch()
    want = (("queries", queries, torch.float32), ("out_ids", out_ids, torch.int64),
            ("out_dists", out_dists, torch.float32))
    for name, t, dt in want:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, not {t.dtype}")
        if t.dim() != 2:
            raise ValueError(f"{name} must be 2-D, not {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    nq = queries.shape[0]
    if queries.shape[1] != d:
        raise ValueError(f"queries have {queries.shape[1]} columns, the index d = {d}")
    if out_ids.shape != out_dists.shape:
        raise ValueError(f"out_ids {tuple(out_ids.shape)} and out_dists {tuple(out_dists.shape)} differ")
    if out_ids.shape[0] < nq:
        raise ValueError(f"outputs have {out_ids.shape[0]} rows for {nq} queries")
    for name, t, _ in want:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")


def _rows(keep_bf16, keep_fp8):
    """TACO_ROWS_* mask of the row copies an index keeps."""
    return (ROWS_BF16 if keep_bf16 else 0) | (ROWS_FP8 if keep_fp8 else 0)


def query_params(k, budget, rerank_target, precision="fp32", select_rule="literal",
                 shortlist_mult=4, probe_precision="fp32"):
    return QueryParams(int(k), _PREC.get(precision, precision), int(budget), int(rerank_target),
                       _RULE.get(select_rule, select_rule), int(shortlist_mult),
                       _PREC.get(probe_precision, probe_precision), 0)


def query_param_array(per_query):
    """A C array of QueryParams from QueryParams structs or dicts of query_params arguments
    (build it once to pass the same per-query parameters to many searches)."""
    arr = (QueryParams * len(per_query))()
    for j, item in enumerate(per_query):
        arr[j] = item if isinstance(item, QueryParams) else query_params(**item)
    return arr


class TacoIndex:
    """An index owned by libtaco (device memory on the current CUDA device)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    # ---- construction --------------------------------------------------------------
    @classmethod
    def build(cls, data, n_subspaces, sub_dim, sqrt_k, kmeans_iters=20, seed=0, keep_bf16=True,
              keep_fp8=False, stream=None):
        lib = load_library()
        x = _as_f32(data)
        n, d = x.shape
        p = BuildParams(n_subspaces, sub_dim, sqrt_k, kmeans_iters, seed,
                        _rows(keep_bf16, keep_fp8), 0)
        out = C.c_void_p()
        _check(lib.taco_build_index(_ptr(x), n, d, C.byref(p), _stream_handle(stream), C.byref(out)))
        return cls(out.value)

    @classmethod
    def from_parts(cls, data, o_bar, B, centroids, codes, n_subspaces, sub_dim, sqrt_k,
                   keep_bf16=True, keep_fp8=False, stream=None):
        lib = load_library()
        x = _as_f32(data)
        n, d = x.shape
        ob = np.ascontiguousarray(o_bar, dtype=np.float64)
        Bm = np.ascontiguousarray(B, dtype=np.float64)
        ce = np.ascontiguousarray(centroids, dtype=np.float64)
        co = np.ascontiguousarray(codes, dtype=np.uint16)
        assert ob.shape == (d,) and Bm.shape == (d, n_subspaces * sub_dim)
        assert ce.shape == (n_subspaces, sqrt_k, sub_dim) and co.shape == (n_subspaces, n)
        parts = IndexParts(ob.ctypes.data, Bm.ctypes.data, ce.ctypes.data, co.ctypes.data,
                           n_subspaces, sub_dim, sqrt_k, 0)
        out = C.c_void_p()
        _check(lib.taco_index_create(_ptr(x), n, d, C.byref(parts), _rows(keep_bf16, keep_fp8),
                                     _stream_handle(stream), C.byref(out)))
        return cls(out.value)

    @classmethod
    def load(cls, path, keep_bf16=True, keep_fp8=False, stream=None):
        out = C.c_void_p()
        _check(load_library().taco_load_index(os.fsencode(path), _rows(keep_bf16, keep_fp8),
                                              _stream_handle(stream), C.byref(out)))
        return cls(out.value)

    def save(self, path):
        _check(load_library().taco_save_index(self._h, os.fsencode(path)))

    def close(self):
        if self._h is not None and self._h.value:
            load_library().taco_free_index(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- introspection -------------------------------------------------------------
    def info(self):
        inf = IndexInfo()
        _check(load_library().taco_index_get_info(self._h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in IndexInfo._fields_}

    def lists(self):
        """taco_index_lists: the device cell lists as NumPy arrays (sizes [N_s, K], split
        [N_s, K, n_slabs + 1], ids [n_ids])."""
        inf = self.info()
        ns, K = inf["n_subspaces"], inf["sqrt_k"] ** 2
        out = {"sizes": np.zeros((ns, K), dtype=np.uint32),
               "split": np.zeros((ns, K, inf["n_slabs"] + 1), dtype=np.uint32),
               "ids": np.zeros(inf["n_ids"], dtype=np.uint32)}
        _check(load_library().taco_index_lists(self._h, *[out[k].ctypes.data for k in ("sizes", "split", "ids")]))
        return out

    def export(self):
        inf = self.info()
        n, d = inf["n"], inf["d"]
        ns, s, sk = inf["n_subspaces"], inf["sub_dim"], inf["sqrt_k"]
        out = {
            "o_bar": np.zeros(d), "B": np.zeros((d, ns * s)), "eigvals": np.zeros(d),
            "alloc": np.zeros(ns * s, dtype=np.int32), "centroids": np.zeros((ns, sk, s)),
            "codes": np.zeros((ns, n), dtype=np.uint16),
        }
        _check(load_library().taco_index_export(
            self._h, *[out[k].ctypes.data for k in ("o_bar", "B", "eigvals", "alloc",
                                                     "centroids", "codes")]))
        return out

    # ---- per-kernel timing -----------------------------------------------------------
    def profile(self, enable=True):
        _check(load_library().taco_profile_enable(self._h, int(bool(enable))))

    def profile_read(self, reset=True):
        kt = KernelTimes()
        _check(load_library().taco_profile_read(self._h, C.byref(kt), int(bool(reset))))
        return {name: {"launches": int(kt.launches[j]), "ms": float(kt.ms[j])}
                for j, name in enumerate(KERNEL_NAMES)}

    # ---- search --------------------------------------------------------------------
    def _prepare(self, queries, k, budget, rerank_target, precision, select_rule,
                 shortlist_mult, per_query, k_stride, probe_precision="fp32"):
        q = _as_f32(queries)
        nq = q.shape[0]
        defaults = query_params(k, budget, rerank_target, precision, select_rule, shortlist_mult,
                                probe_precision)
        pq = None
        if per_query is not None:
            if isinstance(per_query, C.Array) and per_query._type_ is QueryParams:
                arr = per_query   # already in the C layout (see query_param_array)
            else:
                arr = query_param_array(per_query)
            if len(arr) != nq:
                raise ValueError(f"{len(arr)} parameter records for {nq} queries")
            pq = arr
            kmax = _max_k(arr) if nq else k
        else:
            kmax = k
        k_stride = int(k_stride or kmax)
        return q, nq, defaults, pq, k_stride

    def _outputs(self, q, nq, k_stride, out_ids, out_dists):
        if out_ids is None or out_dists is None:
            if _is_cuda_tensor(q):
                torch = _torch()
                out_ids = torch.empty((nq, k_stride), dtype=torch.int64, device=q.device)
                out_dists = torch.empty((nq, k_stride), dtype=torch.float32, device=q.device)
            else:
                out_ids = np.empty((nq, k_stride), dtype=np.int64)
                out_dists = np.empty((nq, k_stride), dtype=np.float32)
        return out_ids, out_dists

    def search(self, queries, k, budget, rerank_target, precision="fp32", select_rule="literal",
               shortlist_mult=4, per_query=None, k_stride=None, out_ids=None, out_dists=None,
               stream=None, probe_precision="fp32"):
        """Alg. 6 for a batch; returns (ids int64 [nq,k_stride], dists float32 [nq,k_stride])."""
        q, nq, defaults, pq, k_stride = self._prepare(queries, k, budget, rerank_target, precision,
                                                      select_rule, shortlist_mult, per_query, k_stride,
                                                      probe_precision)
        out_ids, out_dists = self._outputs(q, nq, k_stride, out_ids, out_dists)
        _check(load_library().taco_search_batch(
            self._h, _ptr(q), nq, C.cast(pq, C.c_void_p) if pq is not None else None,
            C.byref(defaults), k_stride, _ptr(out_ids), _ptr(out_dists), _stream_handle(stream)))
        return out_ids, out_dists

    def shard_count(self, shard, n_shards, queries, k, budget, rerank_target, precision="fp32",
                    select_rule="literal", shortlist_mult=4, per_query=None, k_stride=None,
                    stream=None, probe_precision="fp32"):
        """taco_shard_count: the transform, probe and counting of id-range shard `shard` of
        `n_shards`; returns (ShardSearch, its level counts [nq, N_s + 1] int64)."""
        q, nq, defaults, pq, k_stride = self._prepare(queries, k, budget, rerank_target, precision,
                                                      select_rule, shortlist_mult, per_query, k_stride,
                                                      probe_precision)
        hist = np.empty((nq, self.info()["n_subspaces"] + 1), dtype=np.int64)
        h = C.c_void_p()
        _check(load_library().taco_shard_count(
            self._h, int(shard), int(n_shards), _ptr(q), nq, C.cast(pq, C.c_void_p) if pq is not None else None,
            C.byref(defaults), k_stride, hist.ctypes.data, _stream_handle(stream), C.byref(h)))
        return ShardSearch(h, nq, k_stride, self), hist

    def search_sharded(self, queries, k, budget, rerank_target, n_shards, precision="fp32",
                       select_rule="literal", shortlist_mult=4, per_query=None, k_stride=None,
                       stream=None, probe_precision="fp32"):
        """Alg. 6 split over `n_shards` id-range shards of this index, run one after another
        on its device: every shard counted, the level counts summed, every shard selected,
        the shards' k nearest merged (paper_2603_24919_gb300.sharding). Returns host
        (ids int64 [nq, k_stride], dists float32 [nq, k_stride])."""
        from . import sharding
        shards, hists = [], []
        try:
            for s in range(n_shards):
                sh, hist = self.shard_count(s, n_shards, queries, k, budget, rerank_target, precision,
                                            select_rule, shortlist_mult, per_query, k_stride, stream,
                                            probe_precision)
                shards.append(sh)
                hists.append(hist)
            g = sharding.reduce_counts(hists)
            parts = [sh.select(g, stream) for sh in shards]
        finally:
            for sh in shards:
                sh.close()
        ks = None
        if per_query is not None:
            arr = per_query if isinstance(per_query, C.Array) else query_param_array(per_query)
            ks = np.frombuffer(arr, dtype=np.int32)[::C.sizeof(QueryParams) // 4].astype(np.int64)
        elif k < parts[0][0].shape[1]:
            ks = [k] * parts[0][0].shape[0]
        return sharding.merge_topk(parts, parts[0][0].shape[1], ks)

    def prepare(self, per_query, stream=None):
        """taco_params_create: the per-query parameters (QueryParams or dicts for query_params)
        copied to the device once; pass the result to search_prepared."""
        return PreparedParams(self, per_query, stream)

    def search_prepared(self, queries, params, k_stride=None, out_ids=None, out_dists=None,
                        stream=None):
        """taco_search_batch_params: Alg. 6 for the prepared batch (queries [params.nq, d])."""
        q = _as_f32(queries)
        if q.shape[0] != params.nq:
            raise ValueError(f"{q.shape[0]} queries for {params.nq} prepared records")
        k_stride = int(k_stride or params.k_max)
        out_ids, out_dists = self._outputs(q, params.nq, k_stride, out_ids, out_dists)
        _check(load_library().taco_search_batch_params(
            self._h, _ptr(q), params.handle, k_stride, _ptr(out_ids), _ptr(out_dists),
            _stream_handle(stream)))
        return out_ids, out_dists

    def centroid_distances(self, qt, probe_precision="fp32", stream=None):
        """taco_centroid_distances: [nq, N_s, 2, sqrt_k] squared half-distances of the
        transformed queries qt (CUDA [nq, N_s*s]) to the centroids."""
        torch = _torch()
        inf = self.info()
        nq = int(qt.shape[0])
        out = torch.empty((nq, inf["n_subspaces"], 2, inf["sqrt_k"]), dtype=torch.float32,
                          device=qt.device)
        _check(load_library().taco_centroid_distances(
            self._h, _ptr(qt.contiguous()), nq, _PREC.get(probe_precision, probe_precision),
            _ptr(out), _stream_handle(stream)))
        return out

    def autotune(self, queries, k, budget, rerank_target, precision="fp32", select_rule="literal",
                 shortlist_mult=4, probe_precision="fp32", reps=3, stream=None):
        """taco_autotune on a sample batch (CUDA queries); reps <= 0 restores the defaults.
        Returns the chosen layout and the sample's time before and after."""
        p = query_params(k, budget, rerank_target, precision, select_rule, shortlist_mult,
                         probe_precision)
        r = TuneResult()
        q = queries if queries is not None else None
        nq = int(q.shape[0]) if q is not None else 0
        _check(load_library().taco_autotune(self._h, _ptr(q) if q is not None else None, nq,
                                            C.byref(p), int(reps), _stream_handle(stream),
                                            C.byref(r)))
        return {f: getattr(r, f) for f, _ in TuneResult._fields_ if not f.startswith("reserved")}

    def set_codes_fallback(self, enable=True):
        """taco_index_set_option(TACO_OPT_CODES_FALLBACK): answer flagged queries from the cell
        codes instead of the cluster kernel."""
        _check(load_library().taco_index_set_option(self._h, OPT_CODES_FALLBACK, int(bool(enable))))

    def set_count_layout(self, slabs_per_range=None, count_warps=None, walk_unroll=None):
        """taco_index_set_option for the counting layout taco_autotune chooses (slabs of
        counters per id range, warps per counting CTA, loads in flight per lane)."""
        lib = load_library()
        for opt, v in ((OPT_SLABS_PER_RANGE, slabs_per_range), (OPT_COUNT_WARPS, count_warps),
                       (OPT_WALK_UNROLL, walk_unroll)):
            if v is not None:
                _check(lib.taco_index_set_option(self._h, opt, int(v)))

    def device_status(self, clear=True):
        """The index's device status word (0 = no bounded device wait gave up)."""
        v = C.c_int32()
        _check(load_library().taco_device_status(self._h, C.byref(v), int(bool(clear))))
        return int(v.value)

    def search_noalloc(self, queries, out_ids, out_dists, k, budget, rerank_target,
                       precision="fp32", select_rule="literal", shortlist_mult=4, stream=None):
        """taco_search_batch_noalloc: CUDA queries and caller-owned CUDA outputs; the
        library allocates nothing (its scratch is a fixed device array). The tensors are
        checked first and used as given (no copy is made): queries float32 [nq, d], out_ids
        int64 and out_dists float32 [>= nq, k_stride], all contiguous CUDA tensors."""
        check_noalloc_args(queries, out_ids, out_dists, self.info()["d"])
        p = query_params(k, budget, rerank_target, precision, select_rule, shortlist_mult)
        _check(load_library().taco_search_batch_noalloc(
            self._h, _ptr(queries), int(queries.shape[0]), C.byref(p), int(out_ids.shape[1]),
            _ptr(out_ids), _ptr(out_dists), _stream_handle(stream)))
        return out_ids, out_dists

    def search_debug(self, queries, k, budget, rerank_target, precision="fp32",
                     select_rule="literal", shortlist_mult=4, per_query=None, k_stride=None,
                     want_sc=True, stream=None, probe_precision="fp32"):
        """search() plus every intermediate result (device tensors); queries on CUDA."""
        torch = _torch()
        q, nq, defaults, pq, k_stride = self._prepare(queries, k, budget, rerank_target, precision,
                                                      select_rule, shortlist_mult, per_query, k_stride,
                                                      probe_precision)
        assert _is_cuda_tensor(q), "search_debug needs CUDA queries"
        inf = self.info()
        ns, K, n = inf["n_subspaces"], inf["sqrt_k"] ** 2, inf["n"]
        dev = q.device
        dbg = {
            "query_t": torch.empty((nq, ns * inf["sub_dim"]), dtype=torch.float32, device=dev),
            "probed": torch.empty((nq, ns, K), dtype=torch.uint8, device=dev),
            "retrieved_num": torch.empty((nq, ns), dtype=torch.int64, device=dev),
            "sc": torch.empty((nq, n), dtype=torch.uint8, device=dev) if want_sc else None,
            "collision_num": torch.empty((nq, ns + 1), dtype=torch.int64, device=dev),
            "last_collision": torch.empty((nq,), dtype=torch.int32, device=dev),
            "candidate_num": torch.empty((nq,), dtype=torch.int64, device=dev),
        }
        d = DebugOut(*[_ptr(dbg[f]) for f, _ in DebugOut._fields_])
        out_ids, out_dists = self._outputs(q, nq, k_stride, None, None)
        _check(load_library().taco_search_debug(
            self._h, _ptr(q), nq, C.cast(pq, C.c_void_p) if pq is not None else None,
            C.byref(defaults), k_stride, _ptr(out_ids), _ptr(out_dists), C.byref(d),
            _stream_handle(stream)))
        dbg["ids"], dbg["dists"] = out_ids, out_dists
        return dbg


class ShardSearch:
    """A shard's device state between taco_shard_count and taco_shard_select."""

    def __init__(self, handle, nq, k_stride, index=None):
        self.handle, self.nq, self.k_stride = handle, nq, k_stride
        self.index = index   # the handle refers to the index: keep it alive

    def select(self, global_hist, stream=None):
        """taco_shard_select with the level counts summed over all shards; returns the
        shard's (ids int64 [nq, k_stride], dists float32 [nq, k_stride]) on the host."""
        if self.handle is None or not self.handle.value:
            raise ValueError("the shard handle is closed")
        ih = getattr(self.index, "_h", None)
        if self.index is not None and (ih is None or not ih.value):
            raise ValueError("the shard's index is closed")
        g = np.ascontiguousarray(global_hist, dtype=np.int64)
        n_sub = self.index.info()["n_subspaces"] if self.index is not None else g.shape[-1] - 1
        if g.shape != (self.nq, n_sub + 1):
            raise ValueError(f"global_hist must be [{self.nq}, {n_sub + 1}] (got {list(g.shape)})")
        ids = np.empty((self.nq, self.k_stride), dtype=np.int64)
        dists = np.empty((self.nq, self.k_stride), dtype=np.float32)
        _check(load_library().taco_shard_select(self.handle, g.ctypes.data, ids.ctypes.data,
                                                dists.ctypes.data, _stream_handle(stream)))
        return ids, dists

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().taco_shard_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PreparedParams:
    """Per-query parameters resident on the device (taco_params_create / taco_params_free)."""

    def __init__(self, index, per_query, stream=None):
        self.index = index   # the handle is tied to the index: keep it alive
        self.nq = len(per_query)
        arr = per_query if isinstance(per_query, C.Array) else query_param_array(per_query)
        self.k_max = max(arr[j].k for j in range(self.nq))
        out = C.c_void_p()
        _check(load_library().taco_params_create(index._h, C.cast(arr, C.c_void_p), self.nq,
                                                 _stream_handle(stream), C.byref(out)))
        self.handle = out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().taco_params_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TacoServer:
    """Continuous-batching request loop over a resident index (taco_server_* in the C ABI).

    Requests are single host queries; the library's dispatcher thread batches them onto
    `slots` CUDA streams and a completion thread hands back each request's result."""

    def __init__(self, index, max_batch=256, slots=2, queue_capacity=None, max_list=10,
                 precision="fp32", select_rule="literal", max_wait_us=200, slot_bytes=0,
                 use_graphs=True, probe_precision="fp32"):
        self.index = index   # keeps the index alive while the server runs
        self.d = index.info()["d"]
        self.probe_precision = probe_precision
        p = ServerParams(int(max_batch), int(slots), int(queue_capacity or 4 * max_batch),
                         int(max_list), _PREC.get(precision, precision),
                         _RULE.get(select_rule, select_rule), int(max_wait_us), int(slot_bytes),
                         int(bool(use_graphs)), _PREC.get(probe_precision, probe_precision))
        h = C.c_void_p()
        _check(load_library().taco_server_create(index._h, C.byref(p), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().taco_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, query, k, budget, rerank_target, precision="fp32", select_rule="literal",
               shortlist_mult=4):
        """Queue one query (host array [d]); returns its ticket. Raises TacoError with code
        EAGAIN when the queue is full."""
        q = np.ascontiguousarray(query, dtype=np.float32).reshape(-1)
        assert q.shape[0] == self.d
        p = query_params(k, budget, rerank_target, precision, select_rule, shortlist_mult,
                         self.probe_precision)
        t = C.c_uint64()
        _check(load_library().taco_server_submit(self._h, q.ctypes.data, C.byref(p), C.byref(t)))
        return t.value

    def submit_many(self, queries, per_query):
        """Queue a burst of host queries [m, d] with per-request parameter dicts; returns the
        tickets of the accepted prefix (all m unless the queue filled)."""
        q = np.ascontiguousarray(queries, dtype=np.float32)
        m = q.shape[0]
        arr = (QueryParams * m)()
        for j, item in enumerate(per_query):
            arr[j] = item if isinstance(item, QueryParams) else query_params(
                **dict(item, probe_precision=item.get("probe_precision", self.probe_precision)))
        tickets = np.zeros(m, dtype=np.uint64)
        got = C.c_int64()
        rc = load_library().taco_server_submit_many(self._h, q.ctypes.data, m, C.cast(arr, C.c_void_p),
                                                    tickets.ctypes.data, C.byref(got))
        if rc not in (OK, EAGAIN):
            _check(rc)
        return [int(t) for t in tickets[:got.value]]

    def wait(self, ticket, k_stride, timeout_us=-1):
        """(ids int64 [k_stride], dists float32 [k_stride], info dict) of a request."""
        ids = np.empty(k_stride, dtype=np.int64)
        dists = np.empty(k_stride, dtype=np.float32)
        info = RequestInfo()
        _check(load_library().taco_server_wait(self._h, C.c_uint64(ticket), int(timeout_us),
                                               int(k_stride), ids.ctypes.data, dists.ctypes.data,
                                               C.byref(info)))
        return ids, dists, {f: getattr(info, f) for f, _ in RequestInfo._fields_}

    def replay(self, queries, per_query, arrival_ns, k_stride):
        """Open-loop replay: query j is submitted arrival_ns[j] ns after the start. Returns
        (ids [nq,k_stride], dists [nq,k_stride], latency_ns [nq])."""
        q = np.ascontiguousarray(queries, dtype=np.float32)
        nq = q.shape[0]
        arr = (QueryParams * nq)()
        for j, item in enumerate(per_query):
            arr[j] = item if isinstance(item, QueryParams) else query_params(**item)
        arrival = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        ids = np.empty((nq, k_stride), dtype=np.int64)
        dists = np.empty((nq, k_stride), dtype=np.float32)
        lat = np.empty(nq, dtype=np.int64)
        _check(load_library().taco_server_replay(
            self._h, q.ctypes.data, nq, C.cast(arr, C.c_void_p), arrival.ctypes.data,
            int(k_stride), ids.ctypes.data, dists.ctypes.data, lat.ctypes.data))
        return ids, dists, lat

    def stats(self):
        st = ServerStats()
        _check(load_library().taco_server_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

"""The C-ABI library loads without a GPU, exports every symbol include/taco.h declares,
and the binding's structs match the header's layout. No compute calls."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2603_24919_gb300 import build_lib
from paper_2603_24919_gb300 import taco as T

HEADER = os.path.join(build_lib.INCLUDE, "taco.h")


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return T.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(taco_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["taco_build_index", "taco_index_create", "taco_search_batch", "taco_search_debug",
                 "taco_index_get_info", "taco_index_export", "taco_save_index",
                 "taco_load_index", "taco_free_index", "taco_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s+(taco_\w+)", out))
    assert set(_declared_functions()) <= exported
    assert set(T.SIGNATURES) == set(_declared_functions())


def test_last_error_empty_and_null_args(lib):
    assert lib.taco_last_error() is not None
    # argument checks run before any CUDA call
    assert lib.taco_search_batch(None, None, 0, None, None, 1, None, None, None) == T.EINVAL
    assert b"null index" in lib.taco_last_error()
    assert lib.taco_index_get_info(None, None) == T.EINVAL
    assert lib.taco_save_index(None, b"/nonexistent") == T.EINVAL
    out = ctypes.c_void_p()
    assert lib.taco_load_index(b"/nonexistent/file", 0, None, ctypes.byref(out)) == T.EIO
    lib.taco_free_index(None)
    out = ctypes.c_void_p()
    assert lib.taco_server_create(None, None, ctypes.byref(out)) == T.EINVAL
    assert lib.taco_server_submit(None, None, None, None) == T.EINVAL
    lib.taco_server_destroy(None)
    for opt in (T.OPT_CODES_FALLBACK, T.OPT_SLABS_PER_RANGE, T.OPT_COUNT_WARPS, T.OPT_WALK_UNROLL):
        assert lib.taco_index_set_option(None, opt, 1) == T.EINVAL
    assert lib.taco_autotune(None, None, 0, None, 1, None, None) == T.EINVAL
    assert b"null" in lib.taco_last_error()


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "taco.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
#define S(T) printf(#T " %zu\n", sizeof(T))
int main(void) {
  S(taco_build_params); P(taco_build_params, seed); P(taco_build_params, keep_rows);
  S(taco_query_params); P(taco_query_params, budget); P(taco_query_params, rerank_target);
  P(taco_query_params, select_rule); P(taco_query_params, shortlist_mult);
  P(taco_query_params, probe_precision);
  S(taco_index_parts); P(taco_index_parts, codes); P(taco_index_parts, sqrt_k);
  S(taco_index_info); P(taco_index_info, d_pad); P(taco_index_info, cluster_size);
  P(taco_index_info, has_fp8); P(taco_index_info, fp8_pitch); P(taco_index_info, has_centroid_tc);
  P(taco_index_info, device_bytes); P(taco_index_info, n_ids); P(taco_index_info, build_ms_index);
  S(taco_debug_out); P(taco_debug_out, candidate_num);
  S(taco_server_params); P(taco_server_params, max_wait_us); P(taco_server_params, slot_bytes);
  P(taco_server_params, use_graphs); P(taco_server_params, probe_precision);
  S(taco_request_info); P(taco_request_info, batch_size); P(taco_request_info, slot);
  S(taco_server_stats); P(taco_server_stats, slot_bytes);
  S(taco_tune_result); P(taco_tune_result, count_warps); P(taco_tune_result, walk_unroll);
  P(taco_tune_result, ms_before);
  P(taco_tune_result, trials);
  return 0;
}
"""


def test_struct_layouts_match_header():
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "layout.c")
        exe = os.path.join(td, "layout")
        open(src, "w").write(_LAYOUT_C)
        subprocess.run(["gcc", "-I", build_lib.INCLUDE, src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    want = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    cmap = {"taco_build_params": T.BuildParams, "taco_query_params": T.QueryParams,
            "taco_index_parts": T.IndexParts, "taco_index_info": T.IndexInfo,
            "taco_debug_out": T.DebugOut, "taco_server_params": T.ServerParams,
            "taco_request_info": T.RequestInfo, "taco_server_stats": T.ServerStats,
            "taco_tune_result": T.TuneResult}
    for key, val in want.items():
        if "." in key:
            s, f = key.split(".")
            assert getattr(cmap[s], f).offset == int(val), key
        else:
            assert ctypes.sizeof(cmap[key]) == int(val), key


def test_option_constants_match_header():
    hdr = open(os.path.join(build_lib.INCLUDE, "taco.h")).read()
    opts = dict(re.findall(r"#define TACO_(OPT_\w+) (\d+)", hdr))
    assert set(opts) == {"OPT_CODES_FALLBACK", "OPT_SLABS_PER_RANGE", "OPT_COUNT_WARPS", "OPT_WALK_UNROLL"}
    for name, val in opts.items():
        assert getattr(T, name) == int(val), name


# ------------------------------------------------ search_noalloc: buffers checked before the call
def _noalloc_bufs(torch, nq=4, d=8, ks=5):
    return (torch.zeros((nq, d), dtype=torch.float32), torch.zeros((nq, ks), dtype=torch.int64),
            torch.zeros((nq, ks), dtype=torch.float32))


@pytest.mark.parametrize("case", ["queries_dtype", "queries_cols", "queries_noncontig",
                                  "ids_dtype", "dists_dtype", "ids_short", "shape_mismatch",
                                  "ids_1d", "not_tensor", "not_cuda"])
def test_noalloc_rejects_bad_buffers(case):
    """Every buffer search_noalloc hands to the entry point is checked before any library call:
    a wrong dtype, a short or mis-shaped output or a non-contiguous or host tensor raises
    ValueError (the entry point would otherwise read or write through the raw pointer)."""
    torch = pytest.importorskip("torch")
    q, ids, dists = _noalloc_bufs(torch)
    msg = {"queries_dtype": "queries must be", "queries_cols": "columns",
           "queries_noncontig": "contiguous", "ids_dtype": "out_ids must be",
           "dists_dtype": "out_dists must be", "ids_short": "rows for",
           "shape_mismatch": "differ", "ids_1d": "2-D", "not_tensor": "torch tensor",
           "not_cuda": "CUDA"}[case]
    d = 8
    if case == "queries_dtype":
        q = q.half()
    elif case == "queries_cols":
        d = 9
    elif case == "queries_noncontig":
        q = torch.zeros((8, 4), dtype=torch.float32).t()
    elif case == "ids_dtype":
        ids = ids.int()
    elif case == "dists_dtype":
        dists = dists.double()
    elif case == "ids_short":
        ids, dists = ids[:3], dists[:3]
    elif case == "shape_mismatch":
        dists = torch.zeros((4, 6), dtype=torch.float32)
    elif case == "ids_1d":
        ids = ids.reshape(-1)
    elif case == "not_tensor":
        q = q.numpy()
    with pytest.raises(ValueError) as err:
        T.check_noalloc_args(q, ids, dists, d)
    assert msg in str(err.value)


def test_noalloc_method_checks_before_calling(monkeypatch):
    """TacoIndex.search_noalloc runs the check before it touches the library."""
    torch = pytest.importorskip("torch")
    ix = T.TacoIndex(None)
    monkeypatch.setattr(ix, "info", lambda: {"d": 8})
    monkeypatch.setattr(T, "load_library", lambda: pytest.fail("library called"))
    q, ids, dists = _noalloc_bufs(torch)
    with pytest.raises(ValueError):
        ix.search_noalloc(q, ids.int(), dists, 5, 10, 1)
    ix._h = None


def test_max_k_reads_the_records():
    import numpy as np
    from paper_2603_24919_gb300 import taco as T
    ks = np.random.default_rng(1).integers(1, 300, 1000)
    arr = T.query_param_array([dict(k=int(k), budget=7, rerank_target=3) for k in ks])
    assert T._max_k(arr) == int(ks.max())

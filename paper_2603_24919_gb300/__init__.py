"""GB300 (sm_103a) implementation of the TaCo query path (arXiv 2603.24919).

The library libtaco.so (C ABI in include/taco.h) builds the index of Alg. 3 and answers
batches of k-ANN queries (Alg. 6) with hand-written CUDA kernels. This package holds the
CUDA sources (csrc/), the build script (build_lib.py) and a thin ctypes binding (taco.py).
"""
from .taco import (  # noqa: F401
    LIB_PATH,
    MAX_K,
    MAX_SQRT_K,
    MAX_SUBSPACES,
    PREC_BF16,
    PREC_FP8,
    PREC_FP32,
    SELECT_LITERAL,
    SELECT_PROSE,
    SIGNATURES,
    PreparedParams,
    TacoError,
    TacoIndex,
    TacoServer,
    load_library,
    query_param_array,
    query_params,
)

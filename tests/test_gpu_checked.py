"""The bounds-checked build of the library (-DTACO_CHECKED, libtaco_checked.so): every search
kernel checks the indexes of its gathers and scatters (id-list chunks, counter words, level
lists, arena slots, candidate buffers, candidate ids, list rows) and records a failed check
in the index's device status word instead of trapping.

The same searches (tests/checked_workload.py: the FP8 grid up to alpha 0.1 / beta 0.01 on
the 1M x 128 workload, BF16 and FP32 beside it, the cluster and codes fallbacks, a per-query
batch) run in two processes, one per build, on one index (built and saved by the first,
loaded by the second); the checked run must leave the status word at 0 and return exactly
the results of the product build."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_24919_gb300 import build_lib  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "checked_workload.py")


def _run(lib, out, index_file):
    env = dict(os.environ, TACO_LIB=lib)
    r = subprocess.run([sys.executable, SCRIPT, out, index_file], capture_output=True, text=True, env=env,
                       timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_flags_nothing_and_changes_nothing(tmp_path):
    plain_lib = build_lib.build()
    checked_lib = build_lib.build(checked=True)
    index_file = str(tmp_path / "sift1m.taco")   # built by the first run, loaded by the second
    plain = _run(plain_lib, str(tmp_path / "plain.npz"), index_file)
    checked = _run(checked_lib, str(tmp_path / "checked.npz"), index_file)
    status = {k: int(v[0]) for k, v in checked.items() if k.endswith("_status")}
    assert status and all(v == 0 for v in status.values()), status
    assert set(plain) == set(checked)
    for k in plain:
        if not k.endswith("_status"):
            np.testing.assert_array_equal(checked[k], plain[k], err_msg=k)

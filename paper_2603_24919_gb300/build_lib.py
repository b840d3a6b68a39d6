"""Compile libtaco.so (the C-ABI library) for sm_103a, in-tree.

Every translation unit is compiled by nvcc with one -gencode (compute_103a -> sm_103a)
in parallel, then linked into paper_2603_24919_gb300/libtaco.so. Objects live in
paper_2603_24919_gb300/_build/ and are reused while no source is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtaco.so")
# the checked build: every search kernel bounds-checks its gathers and scatters and records a
# failed check in the index's device status word (-DTACO_CHECKED); a test aid, not the product
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libtaco_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtaco.so")


def _units():
    """(object name, source, extra flags) for every translation unit."""
    units = [
        ("taco_host.o", "taco_host.cpp", []),
        ("taco_build_kernels.o", "taco_build_kernels.cu", []),
        ("taco_search.o", "taco_search.cu", []),
        ("taco_api.o", "taco_api.cu", []),
        ("taco_noalloc.o", "taco_noalloc.cu", []),
        ("taco_server.o", "taco_server.cu", []),
        ("taco_tc.o", "taco_tc.cu", []),
        ("taco_tune.o", "taco_tune.cu", []),
        ("taco_shard.o", "taco_shard.cu", []),
    ]
    for bf16 in (0, 1, 2):
        for r in (1, 4, 16):
            units.append((f"taco_rerank_b{bf16}_r{r}.o", "taco_rerank_inst.cu",
                          [f"-DTACO_INST_BF16={bf16}", f"-DTACO_INST_R={r}"]))
    return units


def _deps_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(verbose: bool = False, jobs: int | None = None, ptxas_verbose: bool = False,
          checked: bool = False) -> str:
    """Build (or reuse) libtaco.so, or with checked=True libtaco_checked.so (bounds-checked
    kernels, -DTACO_CHECKED), and return its path."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    newest = _deps_mtime()
    units = _units()
    todo = []
    for obj, src, extra in units:
        out = os.path.join(build_dir, obj)
        if not os.path.exists(out) or os.path.getmtime(out) < newest or ptxas_verbose:
            flags = list(extra) + (["-DTACO_CHECKED"] if checked else [])
            if ptxas_verbose:
                flags += ["-Xptxas", "-v"]
            todo.append([nvcc, *ARCH, *NVCC_FLAGS, *flags, "-c", os.path.join(CSRC, src), "-o", out])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        return cmd, p.returncode, p.stdout

    jobs = jobs or min(len(todo) or 1, os.cpu_count() or 4)
    failed = []
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        for cmd, rc, out in ex.map(run, todo):
            if out and (verbose or rc != 0 or ptxas_verbose):
                print(out, file=sys.stderr if rc else sys.stdout)
            if rc != 0:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    objs = [os.path.join(build_dir, u[0]) for u in units]
    if todo or not os.path.exists(lib) or os.path.getmtime(lib) < max(map(os.path.getmtime, objs)):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + p.stdout)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv)
    print(LIB)

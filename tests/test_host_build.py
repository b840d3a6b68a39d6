"""The library's host-side FP64 build steps on the CPU: the symmetric eigensolver
(Householder tridiagonalisation + implicit QR; Alg. 1 step 4) and the eigensystem allocation
(Alg. 2) of `csrc/taco_host.cpp`.

A small harness is compiled with nvcc from the library's own source (host code only; no
CUDA call is made) and checked against what fixes these steps independently of the oracle:
the eigen-equation A v = lambda v with orthonormal V and NumPy's eigenvalues, the
hand-worked allocations of tests/golden/alg2_allocation.txt, and the same allocation as the
FP64 oracle's on random eigenvalue lists (ties, values below the scaling floor, N_s*s < d).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import taco_oracle as O
from paper_2603_24919_gb300 import build_lib

HERE = os.path.dirname(os.path.abspath(__file__))

_HARNESS = r"""
#include <cstdio>
#include <vector>
namespace taco {
void symmetric_eigen(int d, std::vector<double>& a, std::vector<double>& vecs, std::vector<double>& vals);
void eigensystem_allocation(const std::vector<double>& lam, int n_subspaces, int sub_dim,
                            std::vector<std::vector<int>>& buckets);
}
int main() {
    char mode[16];
    while (std::scanf("%15s", mode) == 1) {
        if (mode[0] == 'e') {          // eig d, then d*d values
            int d;
            if (std::scanf("%d", &d) != 1) return 1;
            std::vector<double> a(size_t(d) * d), v, w;
            for (double& x : a) if (std::scanf("%lf", &x) != 1) return 1;
            taco::symmetric_eigen(d, a, v, w);
            for (double x : w) std::printf("%.17g ", x);
            std::printf("\n");
            for (double x : v) std::printf("%.17g ", x);
            std::printf("\n");
        } else {                       // alloc d n_subspaces sub_dim, then d values
            int d, ns, s;
            if (std::scanf("%d %d %d", &d, &ns, &s) != 3) return 1;
            std::vector<double> lam(d);
            for (double& x : lam) if (std::scanf("%lf", &x) != 1) return 1;
            std::vector<std::vector<int>> b;
            taco::eigensystem_allocation(lam, ns, s, b);
            for (auto& bucket : b) {
                for (int e : bucket) std::printf("%d ", e);
                std::printf("\n");
            }
        }
        std::fflush(stdout);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    td = tmp_path_factory.mktemp("host_build")
    src = td / "harness.cu"
    src.write_text(_HARNESS)
    exe = td / "harness"
    subprocess.run([nvcc, *build_lib.ARCH, "-O2", "-std=c++17", "-I", build_lib.INCLUDE,
                    "-I", build_lib.CSRC, str(src), os.path.join(build_lib.CSRC, "taco_host.cpp"),
                    "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


def _run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout


def _eig(exe, a):
    d = a.shape[0]
    out = _run(exe, "eig %d %s\n" % (d, " ".join("%.17g" % x for x in a.ravel()))).splitlines()
    vals = np.array(out[0].split(), dtype=np.float64)
    vecs = np.array(out[1].split(), dtype=np.float64).reshape(d, d)
    return vals, vecs


def _alloc(exe, lam, ns, s):
    out = _run(exe, "alloc %d %d %d %s\n" % (len(lam), ns, s, " ".join("%.17g" % x for x in lam)))
    return [[int(t) for t in line.split()] for line in out.splitlines()]


@pytest.mark.parametrize("d,spread", [(1, 1.0), (2, 3.0), (8, 1e2), (37, 1e6), (128, 1e4), (300, 1e8)])
def test_eigensolver_solves_the_eigen_equation(harness, d, spread):
    rng = np.random.default_rng(d)
    q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    lam = np.geomspace(spread, 1.0, d)
    if d > 2:
        lam[d // 2] = lam[d // 2 + 1]       # one exact double eigenvalue
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    vals, vecs = _eig(harness, a)
    top = float(np.abs(lam).max())
    assert np.abs(a @ vecs - vecs * vals).max() <= 1e-9 * top
    assert np.abs(vecs.T @ vecs - np.eye(d)).max() <= 1e-12 * d
    np.testing.assert_allclose(np.sort(vals), np.sort(np.linalg.eigvalsh(a)), rtol=1e-10,
                               atol=1e-12 * top)


@pytest.mark.parametrize("case", ["diagonal", "zero", "indefinite", "cluster", "tridiagonal"])
def test_eigensolver_special_matrices(harness, case):
    """Inputs that skip or stress a stage: already diagonal (every reflector is the
    identity), zero, negative eigenvalues, a tight cluster of eigenvalues, and an already
    tridiagonal matrix with zero off-diagonal gaps (the QR steps split into blocks)."""
    rng = np.random.default_rng(11)
    d = 40
    if case == "diagonal":
        a = np.diag(rng.uniform(-5, 5, d))
    elif case == "zero":
        a = np.zeros((d, d))
    elif case == "indefinite":
        q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        a = (q * np.linspace(-3, 7, d)) @ q.T
    elif case == "cluster":
        q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        a = (q * (1.0 + 1e-9 * rng.standard_normal(d))) @ q.T
    else:
        a = np.diag(rng.uniform(1, 2, d)) + np.diag(rng.uniform(-1, 1, d - 1), 1)
        a[np.arange(9, d - 1, 10), np.arange(10, d, 10)] = 0.0
        a = np.triu(a) + np.triu(a, 1).T
    a = 0.5 * (a + a.T)
    vals, vecs = _eig(harness, a)
    scale = max(1.0, float(np.abs(a).max()))
    assert np.abs(a @ vecs - vecs * vals).max() <= 1e-10 * scale * d
    assert np.abs(vecs.T @ vecs - np.eye(d)).max() <= 1e-12 * d
    np.testing.assert_allclose(np.sort(vals), np.sort(np.linalg.eigvalsh(a)), atol=1e-10 * scale)


def test_eigensolver_on_a_sample_covariance(harness):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4000, 24)) * np.linspace(5, 0.1, 24) @ np.linalg.qr(rng.standard_normal((24, 24)))[0]
    _, sigma = O.mean_and_covariance(x)
    vals, vecs = _eig(harness, sigma)
    assert np.abs(sigma @ vecs - vecs * vals).max() <= 1e-9 * float(vals.max())


def _golden_cases():
    cases, cur = [], None
    for line in open(os.path.join(HERE, "golden", "alg2_allocation.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "case":
            cur = {"buckets": []}
            cases.append(cur)
        elif t[0] in ("n_subspaces", "sub_dim"):
            cur[t[0]] = int(t[1])
        elif t[0] == "lam":
            cur["lam"] = [float(v) for v in t[1:]]
        elif t[0] == "bucket":
            cur["buckets"].append([int(v) for v in t[1:]])
    return cases


def test_allocation_hand_worked_cases(harness):
    cases = _golden_cases()
    assert len(cases) == 4
    for c in cases:
        assert _alloc(harness, c["lam"], c["n_subspaces"], c["sub_dim"]) == c["buckets"], c


def test_allocation_equals_oracle_on_random_spectra(harness):
    rng = np.random.default_rng(11)
    for trial in range(60):
        d = int(rng.integers(2, 64))
        ns = int(rng.integers(1, min(d, 10) + 1))
        s = int(rng.integers(1, d // ns + 1))
        kind = trial % 3
        if kind == 0:
            lam = rng.exponential(size=d) + 1e-3
        elif kind == 1:   # many exact ties
            lam = rng.integers(1, 5, size=d).astype(np.float64)
        else:             # a spectrum reaching below the 1e-12 scaling floor, with zeros
            lam = np.geomspace(1.0, 1e-16, d)
            lam[rng.integers(0, d, size=max(1, d // 8))] = 0.0
        want, _ = O.eigensystem_allocation(lam, ns, s)
        assert _alloc(harness, lam.tolist(), ns, s) == want, (d, ns, s, kind)

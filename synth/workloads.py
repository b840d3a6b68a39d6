"""Seeded synthetic stand-ins for the paper's datasets (Section 6.1).

The paper evaluates on DEEP1M, GIST1M, SIFT10M, Yandex DEEP10M and SPACEV10M, none of
which is available here. Each generator below draws a dataset with the shape and value
structure of one of those workloads from NumPy's PCG64 generator:

  data seed  = 1000 + workload number
  query seed = data seed + 1

Queries are fresh draws from the same distribution, never dataset points (the paper
removes its query points from the datasets, Section 6.1).

Nothing here computes any part of the TaCo method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gmm_isotropic(n, d, n_comp, centre_lo, centre_hi, sigma, seed, nq, q_seed,
                  chunk=1 << 18):
    """Isotropic Gaussian mixture: centres U[lo,hi]^d, components chosen uniformly."""
    rng = _rng(seed)
    centres = rng.uniform(centre_lo, centre_hi, size=(n_comp, d))
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        comp = rng.integers(0, n_comp, size=b - a)
        data[a:b] = centres[comp] + sigma * rng.standard_normal((b - a, d))
    qr = _rng(q_seed)
    comp = qr.integers(0, n_comp, size=nq)
    queries = (centres[comp] + sigma * qr.standard_normal((nq, d))).astype(np.float32)
    return data, queries


def gmm_integer(n, d, n_comp, centre_lo, centre_hi, sigma, seed, nq, q_seed,
                chunk=1 << 18):
    """SIFT-like data: isotropic mixture rounded to integers and clipped to [0, 255]."""
    rng = _rng(seed)
    centres = rng.uniform(centre_lo, centre_hi, size=(n_comp, d))
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        comp = rng.integers(0, n_comp, size=b - a)
        x = centres[comp] + sigma * rng.standard_normal((b - a, d))
        data[a:b] = np.clip(np.rint(x), 0, 255)
    qr = _rng(q_seed)
    comp = qr.integers(0, n_comp, size=nq)
    q = centres[comp] + sigma * qr.standard_normal((nq, d))
    queries = np.clip(np.rint(q), 0, 255).astype(np.float32)
    return data, queries


def _haar_orthogonal(d, rng):
    a = rng.standard_normal((d, d))
    qm, r = np.linalg.qr(a)
    return qm * np.sign(np.diag(r))[None, :]


def powerlaw_mixture(n, d, n_comp, spread, exponent, seed, nq, q_seed, chunk=1 << 16):
    """GIST-like: a mixture of n_comp components whose centres and within-component noise
    are both anisotropic Gaussians with eigenvalues i^-exponent under one Haar rotation
    (the noise scaled by spread), components chosen uniformly."""
    rng = _rng(seed)
    rot = _haar_orthogonal(d, rng)
    scale = np.sqrt(np.arange(1, d + 1, dtype=np.float64) ** (-exponent))
    centres = (rng.standard_normal((n_comp, d)) * scale[None, :]) @ rot.T
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        comp = rng.integers(0, n_comp, size=b - a)
        z = spread * rng.standard_normal((b - a, d)) * scale[None, :]
        data[a:b] = centres[comp] + z @ rot.T
    qr = _rng(q_seed)
    comp = qr.integers(0, n_comp, size=nq)
    z = spread * qr.standard_normal((nq, d)) * scale[None, :]
    return data, (centres[comp] + z @ rot.T).astype(np.float32)


def gmm_unit_normalised(n, d, n_comp, spread, seed, nq, q_seed, chunk=1 << 18):
    """Deep10M-like: unit-normalised centres plus spread * noise, renormalised."""
    rng = _rng(seed)
    centres = rng.standard_normal((n_comp, d))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        comp = rng.integers(0, n_comp, size=b - a)
        x = centres[comp] + spread * rng.standard_normal((b - a, d))
        data[a:b] = x / np.linalg.norm(x, axis=1, keepdims=True)
    qr = _rng(q_seed)
    comp = qr.integers(0, n_comp, size=nq)
    x = centres[comp] + spread * qr.standard_normal((nq, d))
    return data, (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def gmm_anisotropic(n, d, n_comp, centre_lo, centre_hi, sigma0, decay, seed, nq, q_seed,
                    chunk=1 << 18):
    """DEEP-like: per-component diagonal sigma_{c,j} = sigma0 * rank_c(j)^-decay."""
    rng = _rng(seed)
    centres = rng.uniform(centre_lo, centre_hi, size=(n_comp, d))
    ranks = np.stack([rng.permutation(d) + 1 for _ in range(n_comp)])
    sig = sigma0 * ranks.astype(np.float64) ** (-decay)
    data = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        comp = rng.integers(0, n_comp, size=b - a)
        data[a:b] = centres[comp] + sig[comp] * rng.standard_normal((b - a, d))
    qr = _rng(q_seed)
    comp = qr.integers(0, n_comp, size=nq)
    q = centres[comp] + sig[comp] * qr.standard_normal((nq, d))
    return data, q.astype(np.float32)


def budget_from_alpha(alpha: float, n: int) -> int:
    """Collision budget B = ceil(alpha * n), computed once in FP64 (never below 1)."""
    return max(1, int(math.ceil(alpha * n - 1e-9 * n)))


def target_from_beta(beta: float, n: int) -> int:
    """Re-rank target floor(beta * n): the integer form of the test h <= beta*n - c."""
    return int(math.floor(beta * n + 1e-9 * n))


@dataclass
class Workload:
    name: str
    n: int
    d: int
    nq: int
    n_subspaces: int
    sub_dim: int
    sqrt_k: int
    k: int
    alpha: float
    beta: float
    gen: str
    gen_args: dict = field(default_factory=dict)

    def generate(self, n=None, nq=None):
        n = self.n if n is None else n
        nq = self.nq if nq is None else nq
        fn = _GENERATORS[self.gen]
        return fn(n=n, d=self.d, nq=nq, **self.gen_args)

    @property
    def budget(self):
        return budget_from_alpha(self.alpha, self.n)

    @property
    def rerank_target(self):
        return target_from_beta(self.beta, self.n)


_GENERATORS = {
    "gmm_isotropic": gmm_isotropic,
    "gmm_integer": gmm_integer,
    "powerlaw_mixture": powerlaw_mixture,
    "gmm_unit_normalised": gmm_unit_normalised,
    "gmm_anisotropic": gmm_anisotropic,
}

# The five workloads. Index parameters follow the paper's ranges (Section 6.1) and
# Table 3 where a dataset there matches the shape.
WORKLOADS = {
    "tiny20k": Workload(
        "tiny20k", n=20_000, d=128, nq=100, n_subspaces=8, sub_dim=16, sqrt_k=16,
        k=10, alpha=0.05, beta=0.01, gen="gmm_isotropic",
        gen_args=dict(n_comp=64, centre_lo=0.0, centre_hi=100.0, sigma=8.0,
                      seed=1001, q_seed=1002)),
    "sift1m": Workload(
        "sift1m", n=1_000_000, d=128, nq=10_000, n_subspaces=8, sub_dim=16, sqrt_k=64,
        k=10, alpha=0.05, beta=0.005, gen="gmm_integer",
        gen_args=dict(n_comp=1024, centre_lo=0.0, centre_hi=128.0, sigma=20.0,
                      seed=1002, q_seed=1003)),
    "gist1m": Workload(
        "gist1m", n=1_000_000, d=960, nq=1_000, n_subspaces=10, sub_dim=96, sqrt_k=64,
        k=10, alpha=0.05, beta=0.005, gen="powerlaw_mixture",
        gen_args=dict(n_comp=1024, spread=0.5, exponent=1.2, seed=1003, q_seed=1004)),
    "deep10m": Workload(
        "deep10m", n=10_000_000, d=96, nq=4_096, n_subspaces=6, sub_dim=8, sqrt_k=64,
        k=100, alpha=0.02, beta=0.002, gen="gmm_unit_normalised",
        gen_args=dict(n_comp=4096, spread=0.05, seed=1004, q_seed=1005)),
    "deep5m256": Workload(
        "deep5m256", n=5_000_000, d=256, nq=10_000, n_subspaces=6, sub_dim=8, sqrt_k=64,
        k=10, alpha=0.02, beta=0.002, gen="gmm_anisotropic",
        gen_args=dict(n_comp=2048, centre_lo=0.0, centre_hi=100.0, sigma0=8.0,
                      decay=0.6, seed=1005, q_seed=1006)),
}


def make_workload(name: str, n=None, nq=None):
    """Return (workload, data float32 [n,d], queries float32 [nq,d])."""
    w = WORKLOADS[name]
    data, queries = w.generate(n=n, nq=nq)
    return w, np.ascontiguousarray(data), np.ascontiguousarray(queries)

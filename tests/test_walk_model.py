"""CPU model of the counting walk's index arithmetic (`walk_batch` in csrc/taco_rerank.cuh),
checked against the direct definition on adversarial run-length mixes.

The staged runs of one batch are non-empty id-array runs (start_r, len_r), concatenated in
order; element e lies in run r with cpre[r] <= e < cpre[r + 1] and has id-array index
rbase[r] + e, with cpre[nr] = total and cpre[nr + 1 .. nr + 32] = 0xffffffff. A round takes
WU windows of 32 elements; lane u of the warp finds the run of window u's first element by
binary search; in window E, lane j reads boundary cpre[cw + 1 + j] - E, the boundaries inside
the window form a 32-bit mask (PTX shl, whose shift amounts clamp at 32: a boundary at or past
the window end gives 0), and lane l's run is cw + popcount(mask & lanes 0..l), capped at
nr - 1. Lanes past the end get a sentinel whose nibble shift comes out as 32 (adds 0). The
model also checks that every shared-memory read stays inside the staged arrays
(rbase: kCellBatch entries; cpre: kCellBatch + kRunPad).
"""
import numpy as np
import pytest

K_CELL_BATCH, K_RUN_PAD, K_PAST_END = 512, 36, 0x80000000
M32 = 0xFFFFFFFF


def shl_clamped(a, b):
    return 0 if b >= 32 else (a << b) & M32


def stage(lengths, starts):
    """The staged form: cpre (with its padding), rbase, total, nr."""
    nz = [(s, l) for s, l in zip(starts, lengths) if l > 0]
    nr = len(nz)
    cpre = np.full(K_CELL_BATCH + K_RUN_PAD, 0xDEADBEEF, dtype=np.int64)   # unwritten entries
    rbase = np.full(K_CELL_BATCH, 0xDEADBEEF, dtype=np.int64)
    acc = 0
    for r, (s, l) in enumerate(nz):
        cpre[r] = acc
        rbase[r] = (s - acc) & M32
        acc += l
    cpre[nr] = acc
    cpre[nr + 1:nr + 33] = M32
    return cpre, rbase, acc, nr


def find_cell(cpre, nr, key):
    lo, hi = 0, nr - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if cpre[mid] <= key:
            lo = mid
        else:
            hi = mid - 1
    return lo


def walk_indices(cpre, rbase, total, nr, wu, last_idx):
    """Id-array index per element as the walk computes it (None for lanes past the end),
    asserting every shared-memory index the walk reads."""
    out = {}
    rnd = 32 * wu
    for g in range((total + rnd - 1) // rnd):
        e = g * rnd
        cwl = [find_cell(cpre, nr, min(e + 32 * (lane % wu), total - 1)) for lane in range(32)]
        for u in range(wu):
            E = e + 32 * u
            cw = cwl[u]
            mask = 0
            for j in range(32):
                idx = cw + 1 + j
                assert idx < K_CELL_BATCH + K_RUN_PAD
                pb = (int(cpre[idx]) - E) & M32
                mask |= shl_clamped(1, pb)
            for lane in range(32):
                r = min(cw + bin(mask & ((2 << lane) - 1) & M32).count("1"), nr - 1)
                assert 0 <= r < K_CELL_BATCH
                x = min((int(rbase[r]) + E + lane) & M32, last_idx)
                if E + lane < total:
                    out[E + lane] = x
                else:
                    sentinel = K_PAST_END
                    sh = ((sentinel << 2) & 28) | (sentinel >> 26)
                    assert sh == 32 and shl_clamped(1, sh) == 0 and ((sentinel & ~K_PAST_END) >> 3) == 0
    return out


def direct_indices(lengths, starts):
    out, e = {}, 0
    for s, l in zip(starts, lengths):
        for t in range(l):
            out[e] = s + t
            e += 1
    return out


MIXES = {
    "singletons": lambda rng, m: np.ones(m, dtype=int),
    "with_empty": lambda rng, m: rng.integers(0, 3, m),
    "long": lambda rng, m: rng.integers(50, 300, m),
    "mixed": lambda rng, m: np.where(rng.random(m) < 0.5, 1, rng.integers(1, 90, m)),
    "exact_windows": lambda rng, m: np.full(m, 32),
}


@pytest.mark.parametrize("mix", sorted(MIXES))
@pytest.mark.parametrize("wu", [8, 16])
def test_walk_maps_every_element_to_its_id(mix, wu):
    rng = np.random.default_rng(hash((mix, wu)) % 2**32)
    for m in (1, 7, 64, 511, 512):
        lengths = [int(v) for v in MIXES[mix](rng, m)]
        if sum(lengths) == 0:
            lengths[0] = 1
        starts = [int(v) for v in rng.integers(0, 10**6, m)]
        cpre, rbase, total, nr = stage(lengths, starts)
        got = walk_indices(cpre, rbase, total, nr, wu, last_idx=2**32 - 1)
        assert got == direct_indices(lengths, starts), (mix, wu, m)

"""CPU model of the counting walks' index arithmetic, checked against the direct definition
on adversarial run-length mixes: `walk_batch` (csrc/taco_rerank.cuh, the cluster kernel;
elements are ids) and `walk_chunks` (csrc/taco_count.cuh, the counting pass; elements are
4-id chunks of the 16-byte aligned, padded cell lists, filtered by the unit's id range).

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


# ------------------------------------------------------------ the chunk walk (count_lists_kernel)
PAD = 0xFFFFFFFF


def padded_lists(codes, n_cells):
    """Cell lists of one subspace laid out as the library does: ids ascending per cell, each
    list starting at a multiple of 4 and padded to the next one with 0xffffffff; returns the
    array and the start of every cell."""
    ids, starts = [], []
    for c in range(n_cells):
        starts.append(len(ids))
        members = [int(p) for p in np.nonzero(codes == c)[0]]
        ids += members + [PAD] * ((-len(members)) % 4)
    return np.array(ids, dtype=np.int64), starts


@pytest.mark.parametrize("wu", [4, 8])
@pytest.mark.parametrize("n_cells,n", [(7, 3000), (64, 20000), (300, 5000)])
def test_chunk_walk_counts_exactly_the_probed_ids_of_the_range(wu, n_cells, n):
    """The chunk runs [b / 4, ceil(e / 4)) of the probed cells' runs in a range, walked with
    the window/mask lookup and filtered by the range test, visit every id of those runs once
    and nothing else (padding and the cells' ids of other ranges fail the test). Counting
    with an entry tagged j each time a count reaches a level j >= 2 gives, for every j, one
    entry tagged j per id with SC >= j (so the candidates at threshold t are the entries
    tagged t), and ge[1] = events - entries."""
    rng = np.random.default_rng(n_cells * 1000 + wu)
    ns = 4
    lists = [padded_lists(rng.integers(0, n_cells, n), n_cells) for _ in range(ns)]
    base, arrays = 0, []
    for arr, st in lists:   # subspaces one after another (each a multiple of 4 long)
        arrays.append((base, st))
        base += len(arr)
    allids = np.concatenate([a for a, _ in lists])
    last_chunk = len(allids) // 4 - 1
    slab = 997   # a range of ids [lo, hi)
    for lo in range(0, n, slab * 3):
        hi = min(lo + slab * 3, n)
        probed = [sorted(rng.choice(n_cells, size=max(1, n_cells // 3), replace=False)) for _ in range(ns)]
        starts, lengths, want = [], [], []
        for i in range(ns):
            off, st = arrays[i]
            arr = lists[i][0]
            for c in probed[i]:
                end = st[c + 1] if c + 1 < n_cells else len(arr)
                cell = arr[st[c]:end]
                real = cell[cell != PAD]
                b = off + st[c] + int(np.searchsorted(real, lo))
                e = off + st[c] + int(np.searchsorted(real, hi))
                want += [int(x) for x in real if lo <= x < hi]
                s0, ln = b >> 2, (((e + 3) >> 2) - (b >> 2)) if e > b else 0
                starts.append(s0)
                lengths.append(ln)
        if sum(lengths) == 0:
            continue
        cpre, rbase, total, nr = stage(lengths, starts)
        chunks = walk_indices(cpre, rbase, total, nr, wu, last_idx=last_chunk)
        got, cnt, entries = [], {}, []
        for e_, x in sorted(chunks.items()):
            for h in range(4):
                v = int(allids[4 * x + h])
                rel = (v - lo) & M32
                if rel < hi - lo:
                    got.append(v)
                    old = cnt.get(rel, 0)
                    cnt[rel] = old + 1
                    if old >= 1:
                        entries.append((rel, old + 1))
        assert sorted(got) == sorted(want)
        for j in range(2, ns + 1):
            tagged = sorted(r for r, t in entries if t == j)
            assert tagged == sorted(r for r, c in cnt.items() if c >= j), j
        ge1 = sum(1 for c in cnt.values() if c >= 1)
        assert ge1 == len(got) - len(entries)


# ------------------------------------------------------------------------ counter packing
def test_three_bit_counter_word_and_shift():
    """3-bit counters (10 a word): word(x) = high 32 bits of x * ceil(2^32 / 10) equals
    x // 10 for every id offset of a 15-slab range (and far beyond), shift = 3 (x mod 10) stays
    inside the low 30 bits, and a count of at most 7 never carries into a neighbour."""
    x = np.arange(0, 1 << 22, dtype=np.uint64)
    word = (x * np.uint64(429496730)) >> np.uint64(32)
    assert np.array_equal(word, x // np.uint64(10))
    top = np.array([2**30 - 1, 2**30 - 10, 2**29 + 7], dtype=np.uint64)
    assert np.array_equal((top * np.uint64(429496730)) >> np.uint64(32), top // np.uint64(10))
    shift = (x[:1000] - word[:1000] * np.uint64(10)) * np.uint64(3)
    assert shift.max() == 27
    rng = np.random.default_rng(7)
    for _ in range(200):   # ten counters packed by repeated adds, each at most 7
        counts = rng.integers(0, 8, 10)
        w = 0
        for j, c in enumerate(counts):
            for _ in range(int(c)):
                old = w
                w = (w + (1 << (3 * j))) & M32
                assert (old >> (3 * j)) & 7 == ((w >> (3 * j)) & 7) - 1
        assert [(w >> (3 * j)) & 7 for j in range(10)] == list(counts)
        assert w < 2**30

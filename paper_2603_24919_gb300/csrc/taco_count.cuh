// Collision counting of the two-pass search (Alg. 6 step 7, Def. 6), pass 1.
//
// Persistent CTAs take queries and, for each, its id ranges in turn (a (query, range) pair is
// a unit). A unit's collisions are counted in 4-bit shared-memory counters. Each time an
// id's count reaches a level j >= 2 (the shared-memory atomic's old value is j - 1), the id
// (relative to the range) is appended to the unit's arena slot tagged with j: the entries
// tagged j are then exactly the range's ids with SC >= j, one each, so the unit's level
// counts ge[j] = #{ids with SC >= j} are the counts of the tags, ge[1] = events - entries,
// and the candidates at an Alg. 5 threshold t >= 2 are the entries tagged t. Pass 2
// (select_rerank_kernel) sums the level counts of a query's ranges, applies Alg. 5 and
// re-ranks those entries. Queries whose threshold falls below 2, or whose entries do not fit
// a slot, are flagged for a fallback.
//
// The cell lists are stored 16-byte aligned and padded to a multiple of 4 ids (with kIdPad),
// so the run of a probed cell that falls in the unit's id range is covered by whole 4-id
// chunks of its own list: the walk loads one chunk (uint4) per lane and keeps the ids that
// lie in the range (the chunk's other ids belong to the same cell's neighbouring ranges, or
// are padding, and fail the range test).
#pragma once

#include "taco_rerank.cuh"

namespace taco {

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint4 ldg_keep_u4(const uint4* p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

// Bulk prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global address into L2;
// no completion to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Shared memory of count_lists_kernel past the counters and their 32 spare words (bytes):
// split bounds of the staged cells for two ranges, two staging buffers of chunk runs, the
// level counts and the staged cells.
__host__ __device__ __forceinline__ size_t count_lists_extra() {
    return size_t(2) * kCellBatch * 8 + size_t(2) * kCellBatch * 4 + size_t(2) * (kCellBatch + kRunPad) * 4 +
           16 * 4 + size_t(kCellBatch) * 4;
}

// The chunk run of id positions [b, e) of one cell list: chunks [b / 4, ceil(e / 4)), none
// when the run is empty. Cell lists start on chunk boundaries, so the chunks stay inside the
// cell's padded list.
__device__ __forceinline__ void chunk_run(uint32_t b, uint32_t e, uint32_t& start, uint32_t& len) {
    start = b >> 2;
    len = e > b ? ((e + 3u) >> 2) - start : 0u;
}

// Packing of the shared-memory counters: CB = 4 bits, 8 counters a word (any N_s up to 15), or
// CB = 3 bits, 10 counters in the low 30 bits of a word (N_s <= 7, so a count never exceeds 7;
// 15 slabs of 2^15 ids fit the 192 KB that 12 slabs take at 4 bits).
template <int CB>
struct CounterGeom;
template <>
struct CounterGeom<4> {
    static constexpr uint32_t kPer = 8, kMask = 15u;
    __device__ __forceinline__ static uint32_t word(uint32_t x) { return x >> 3; }
    __device__ __forceinline__ static uint32_t shift(uint32_t x, uint32_t w) { return (x - (w << 3)) << 2; }
};
template <>
struct CounterGeom<3> {
    static constexpr uint32_t kPer = 10, kMask = 7u;
    // x / 10 for x < 2^30: the product with ceil(2^32 / 10) errs by less than 0.1 x / 2^30
    __device__ __forceinline__ static uint32_t word(uint32_t x) { return __umulhi(x, 429496730u); }
    __device__ __forceinline__ static uint32_t shift(uint32_t x, uint32_t w) { return (x - w * 10u) * 3u; }
};

// Counter words of a range of `ids` ids.
__host__ __device__ __forceinline__ int counter_words_for(int64_t ids, int cb) {
    const int64_t per = cb == 3 ? 10 : 8;
    return int((ids + per - 1) / per);
}

// One walk round's loads, held in registers from the issue to the count.
template <int WU>
struct WalkRound {
    uint4 v[WU];
    uint32_t live;   // bit u: this lane's chunk of window u is inside the batch
};

// Issue the loads of round g (WU windows of 32 chunks) of a staged batch of chunk runs
// (total chunks in nr non-empty runs; run r covers chunks rbase[r] + [cpre[r], cpre[r + 1])
// of the id array). Lane u finds the run of the first chunk of window u (binary search); in a
// window, lane j reads the j-th next run boundary, the boundaries inside the window form a
// bit mask, and a lane's run is the window's first run plus the mask bits at or below it
// (runs are non-empty, so at most 32 boundaries fall in a window). Lanes past the end load a
// valid chunk and are not live.
template <int WU>
__device__ __forceinline__ void issue_round(WalkRound<WU>& R, const uint4* __restrict__ ids4, uint32_t last_chunk,
                                            uint32_t g, uint32_t total, uint32_t nr, const uint32_t* cpre,
                                            const uint32_t* rbase, uint64_t pol, int lane, int* status) {
    const uint32_t lane_le = (2u << lane) - 1u;   // lanes 0..lane
    const uint32_t e0 = g * 32u * WU;
    const uint32_t key = min(e0 + 32u * uint32_t(lane % WU), total - 1u);
    const uint32_t cwl = uint32_t(find_cell(cpre, int(nr), key));
    R.live = 0;
#pragma unroll
    for (int u = 0; u < WU; ++u) {
        const uint32_t E = e0 + 32u * uint32_t(u);
        const uint32_t cw = __shfl_sync(kFull, cwl, u);
        const uint32_t pb = cpre[cw + 1u + uint32_t(lane)] - E;                 // >= 1 inside
        const uint32_t mask = __reduce_or_sync(kFull, shl_clamped(1u, pb));     // 0 for pb >= 32
        const uint32_t r = min(cw + __popc(mask & lane_le), nr - 1u);
        const uint32_t xr = rbase[r] + E + uint32_t(lane);
        const bool in = E + uint32_t(lane) < total;
        (void)TACO_CHECK(status, !in || xr <= last_chunk, kStatusCount);
        const uint32_t x = min(xr, last_chunk);
        R.v[u] = ldg_keep_u4(ids4 + x, pol);
        R.live |= (in ? 1u : 0u) << u;
    }
}

// Count a round whose loads are in R against the unit's range [lo, lo + rlen): every id of a
// live chunk in the range adds 1 to its CB-bit counter; when the atomic's old value v is >= 1
// the id has just reached level v + 1 >= 2 and is appended to the unit's arena slot `out` as
// (id - lo) | (v + 1) << kLevelShift, and ge[v + 1] counts it. (One row of level counts per
// warp, summed at the end of the unit, was measured slower: the sum lengthens the unit's
// barrier-to-barrier tail.) Ids outside the range (the
// chunk's neighbours in the same cell list, padding) and idle lanes add 0 to the lane's own
// spare word cnt[counter_words + lane] (which stays 0), so no branch depends on the data and
// every atomic is a shared-memory one on cnt. Entries beyond `cap` are counted in *s_app but
// not stored (the caller sees the overflow).
template <int WU, int CB>
__device__ __forceinline__ void count_round(WalkRound<WU>& R, uint32_t lo, uint32_t rlen, uint32_t* cnt,
                                            uint32_t* out, uint32_t cap, uint32_t* ge, uint32_t* s_app, int lane,
                                            int* status, uint32_t counter_words) {
    using Geom = CounterGeom<CB>;
    // all atomics of the round are independent
    uint32_t amask = 0;
    uint32_t rel[WU][4];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
        const uint32_t w4[4] = {R.v[u].x, R.v[u].y, R.v[u].z, R.v[u].w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t x = w4[h] - lo;
            const uint32_t xw = Geom::word(x);
            const bool ok = ((R.live >> u) & 1u) && x < rlen &&
                            TACO_CHECK(status, xw < counter_words, kStatusCount);
            const uint32_t sh = Geom::shift(x, xw);
            const uint32_t w = ok ? xw : counter_words + uint32_t(lane);
            const uint32_t old = atomicAdd(&cnt[w], ok ? 1u << sh : 0u);
            const uint32_t v = (old >> sh) & Geom::kMask;
            amask |= (v != 0u ? 1u : 0u) << (4 * u + h);
            rel[u][h] = x | ((v + 1u) << kLevelShift);
        }
    }
    // append the ids that reached a level >= 2: one reservation per warp and round
    if (__any_sync(kFull, amask != 0u)) {
        const uint32_t na = __popc(amask);
        uint32_t incl = na;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += t;
        }
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        uint32_t base = 0;
        if (lane == 31) base = atomicAdd(s_app, tot);
        uint32_t pos = __shfl_sync(kFull, base, 31) + incl - na;
#pragma unroll
        for (int u = 0; u < WU; ++u)
#pragma unroll
            for (int h = 0; h < 4; ++h)
                if ((amask >> (4 * u + h)) & 1u) {
                    if (pos < cap) out[pos] = rel[u][h];
                    atomicAdd(&ge[rel[u][h] >> kLevelShift], 1u);
                    ++pos;
                }
    }
}

// Walk one staged batch: rounds of WU windows handed to warps by a shared counter (*s_round,
// zero on entry), so warps that drew short work take more; a warp claims its next round only
// when it has counted the current one. (Measured alternatives that were slower on the
// 10M x 96 workload: claiming the next round before counting the current one, which fixes
// the owners of a range's last rounds early and lengthens its tail, and issuing the next
// range's first round before the range barriers.) Warp-level; no barrier.
template <int NW, int WU, int CB>
__device__ __forceinline__ void walk_chunks(const uint4* __restrict__ ids4, uint32_t last_chunk, uint32_t lo,
                                            uint32_t rlen, uint32_t total, uint32_t nr, uint32_t* cnt,
                                            uint32_t* out, uint32_t cap, uint32_t* ge, uint32_t* s_app,
                                            uint32_t* s_round, const uint32_t* cpre, const uint32_t* rbase,
                                            uint64_t pol, int lane, int* status, uint32_t counter_words) {
    static_assert(WU >= 1 && WU <= 8, "one lane finds the run of each window; 4 WU append bits a lane");
    constexpr uint32_t kRound = 32u * WU;
    const uint32_t nrounds = (total + kRound - 1) / kRound;
    WalkRound<WU> R;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(s_round, 1u);
        g = __shfl_sync(kFull, g, 0);   // warp-uniform
        if (g >= nrounds) break;
        issue_round<WU>(R, ids4, last_chunk, g, total, nr, cpre, rbase, pol, lane, status);
        count_round<WU, CB>(R, lo, rlen, cnt, out, cap, ge, s_app, lane, status, counter_words);
    }
}

// One warp stages the chunk runs of the ncell staged cells of one range (their id-position
// bounds in pr[]): the non-empty runs in cell order, run r covering chunks
// rbase[r] + [cpre[r], cpre[r + 1]), cpre[nr] = total and cpre[nr + 1 .. nr + 32] =
// 0xffffffff (the walk's boundary reads). Lane l takes the contiguous cells
// [l per, (l + 1) per) so that cell order is kept. Returns (total chunks, nr) and the ids the
// runs hold in the range (*ev). Warp-level; no barrier.
__device__ __forceinline__ uint2 warp_stage(const uint2* pr, int ncell, uint32_t* rbase, uint32_t* cpre,
                                            uint32_t* ev, int lane) {
    const int per = (ncell + 31) >> 5;
    const int c0 = min(ncell, lane * per), c1 = min(ncell, c0 + per);
    uint32_t nrl = 0, totl = 0, evl = 0;
    for (int c = c0; c < c1; ++c) {
        const uint2 be = pr[c];
        uint32_t start, len;
        chunk_run(be.x, be.y, start, len);
        nrl += len != 0u;
        totl += len;
        evl += be.y - be.x;
    }
    uint32_t inr = nrl, itot = totl;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t a = __shfl_up_sync(kFull, inr, off), b = __shfl_up_sync(kFull, itot, off);
        if (lane >= off) {
            inr += a;
            itot += b;
        }
    }
    uint32_t r = inr - nrl, t = itot - totl;
    for (int c = c0; c < c1; ++c) {
        const uint2 be = pr[c];
        uint32_t start, len;
        chunk_run(be.x, be.y, start, len);
        if (len) {
            cpre[r] = t;
            rbase[r] = start - t;
            ++r;
            t += len;
        }
    }
    const uint32_t nr = __shfl_sync(kFull, inr, 31), total = __shfl_sync(kFull, itot, 31);
    __syncwarp();
    cpre[nr + 1u + uint32_t(lane)] = 0xffffffffu;
    if (lane == 0) cpre[nr] = total;
    *ev = __reduce_add_sync(kFull, evl);
    __syncwarp();
    return make_uint2(total, nr);
}

// NW warps per CTA, WU windows of 32 chunks per walk round, CB-bit counters.
//
// Ranges of a query are pipelined when its probed cells fit one staging batch (at most
// kCellBatch cells): warp NW - 1 (the stager) owns the split bounds (asynchronous copies two
// ranges ahead) and, while the other warps walk range r, prefetches range r + 1's id runs
// into L2 and stages its chunk runs into the second staging buffer, then joins the walk. A
// range costs two barriers: after its walk (counters final), and after the unit's outputs
// and the clearing of the counters.
template <int NW, int WU, int CB>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : 1)
count_lists_kernel(const RerankParams P) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kStager = NW - 1;
    constexpr int kPre = kCellBatch + kRunPad;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);                        // counters + 32 spare
    uint2* pairs = reinterpret_cast<uint2*>(smem + P.region_a);               // [2][kCellBatch]
    uint32_t* rbase = reinterpret_cast<uint32_t*>(pairs + 2 * kCellBatch);    // [2][kCellBatch]
    uint32_t* cpre = rbase + 2 * kCellBatch;                                  // [2][kPre]
    uint32_t* ge = cpre + 2 * kPre;                                           // [16]
    uint32_t* qcell = ge + 16;                                                // kCellBatch
    __shared__ int s_pre[TACO_MAX_SUBSPACES + 1];
    __shared__ uint32_t s_tmp[2 * NW];
    __shared__ uint32_t s_app, s_ev;
    __shared__ uint32_t s_round;    // walk round counter of the current range
    __shared__ uint32_t s_tot2[2], s_nr2[2], s_ev2[2];   // staged batch of each buffer
    __shared__ int64_t s_next;
    const int Ns = P.Ns, K = P.K;
    const int sstride = P.n_slabs + 1;
    const uint64_t pol_keep = l2_policy_keep();
    const uint4* ids4 = reinterpret_cast<const uint4*>(P.ids);
    const uint32_t last_chunk = uint32_t(P.n_ids / 4) - 1u;
    const uint32_t cap = P.arena_per_unit;
    // the counters and, past them, one spare word per lane for the walk's idle atomics
    for (int w = tid; w < P.counter_words + 32; w += NW * 32) cnt[w] = 0u;
    if (tid < 16) ge[tid] = 0u;
    if (tid == 0) {
        s_app = 0u;
        s_round = 0u;
        s_ev = 0u;
    }
    // stager: the split bounds of every staged cell for range r into pairs[slot] (asynchronous)
    auto load_bounds = [&](int total_cells, int r, int slot) {
        const int slo = r * P.slabs_per_cta, shi = min(slo + P.slabs_per_cta, P.n_slabs);
        for (int t = lane; t < total_cells; t += 32) {
            const uint32_t qc = qcell[t];
            const uint32_t* sp = P.split + (size_t(qc >> 16) * K + (qc & 0xffffu)) * sstride;
            cp_async4(&pairs[slot * kCellBatch + t].x, sp + slo);
            cp_async4(&pairs[slot * kCellBatch + t].y, sp + shi);
        }
        cp_async_commit();
    };
    // stager: range r's id runs (bounds in pairs[slot]) into L2, then its chunk runs into
    // staging buffer `buf`
    auto stage_range = [&](int total_cells, int slot, int buf, bool prefetch) {
        const uint2* pr = pairs + slot * kCellBatch;
        if (prefetch)
            for (int t = lane; t < total_cells; t += 32) {
                uint32_t start, len;
                chunk_run(pr[t].x, pr[t].y, start, len);
                if (len) prefetch_l2_bulk(ids4 + start, len * 16u);
            }
        uint32_t ev;
        const uint2 st = warp_stage(pr, total_cells, rbase + buf * kCellBatch, cpre + buf * kPre, &ev, lane);
        if (lane == 0) {
            s_tot2[buf] = st.x;
            s_nr2[buf] = st.y;
            s_ev2[buf] = ev;
        }
    };
    // work item: ranges [rb, re) of query q (all its ranges unless a small batch splits them
    // into range_parts runs so that more CTAs work on it)
    // (a shard counts its ranges [shard_r0, shard_r1) only)
    const int parts = P.range_parts;
    const int per_part = (P.shard_r1 - P.shard_r0 + parts - 1) / parts;
    const int64_t items = P.nq * parts;
    for (int64_t it = blockIdx.x; it < items; it = next_query(P.work, &s_next)) {
        const int64_t q = it / parts;
        const int rb = P.shard_r0 + int(it % parts) * per_part;
        const int re = min(P.shard_r1, rb + per_part);
        __syncthreads();   // the previous item is finished with the shared state
        if (warp == 0) load_cell_prefix(P, q, s_pre, lane);
        __syncthreads();
        const int total_cells = s_pre[Ns];
        const bool staged = total_cells <= kCellBatch;   // one batch: cells kept for every range
        if (staged) {
            for (int t = tid; t < total_cells; t += NW * 32) {
                int i = 0;
                while (t >= s_pre[i + 1]) ++i;
                const int j = t - s_pre[i];
                qcell[t] = (uint32_t(i) << 16) |
                           (TACO_CHECK(P.status, j < K, kStatusCount) ? P.cells[(q * Ns + i) * K + j] : 0u);
            }
            __syncthreads();
            if (warp == kStager && rb < re) {   // bounds of ranges rb and rb + 1, then rb staged
                load_bounds(total_cells, rb, 0);
                if (re - rb > 1) {
                    load_bounds(total_cells, rb + 1, 1);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    cp_async_wait_all();
                }
                __syncwarp();
                stage_range(total_cells, 0, 0, false);
            }
            __syncthreads();   // range rb's staging is visible
        }
        for (int r = rb; r < re; ++r) {
            const int64_t u = q * P.n_ranges + r;
            const int slab_lo = r * P.slabs_per_cta;
            const int slab_hi = min(slab_lo + P.slabs_per_cta, P.n_slabs);
            const int64_t lo = int64_t(slab_lo) << kSlabLog2;
            const int64_t hi = min(int64_t(slab_hi) << kSlabLog2, P.n);
            const int words = hi > lo ? counter_words_for(hi - lo, CB) : 0;
            const uint32_t rlen = uint32_t(hi - lo);
            uint32_t* out = P.arena + size_t(u) * P.arena_per_unit;
            (void)TACO_CHECK(P.status, (size_t(u) + 1) * P.arena_per_unit <= P.arena_words, kStatusCount);
            // (the counters are clear, ge / s_app / s_round zero, range r staged)
            if (staged) {
                const int buf = (r - rb) & 1;   // staging buffer and bounds slot of range r
                if (warp == kStager && r + 1 < re) {
                    cp_async_wait_all();   // the bounds of range r + 1 (slot buf ^ 1)
                    __syncwarp();
                    stage_range(total_cells, buf ^ 1, buf ^ 1, true);
                    if (r + 2 < re) load_bounds(total_cells, r + 2, buf);   // slot of range r: staged
                }
                const uint32_t tot = s_tot2[buf];
                if (tot) walk_chunks<NW, WU, CB>(ids4, last_chunk, uint32_t(lo), rlen, tot, s_nr2[buf], cnt, out, cap, ge,
                                                 &s_app, &s_round, cpre + buf * kPre, rbase + buf * kCellBatch, pol_keep,
                                                 lane, P.status, uint32_t(P.counter_words));
            } else {
                // batches of one cell per thread, at most kCellBatch (the staging arrays)
                constexpr int kBatch = NW * 32 < kCellBatch ? NW * 32 : kCellBatch;
                for (int cb0 = 0; cb0 < total_cells; cb0 += kBatch) {
                    if (cb0) __syncthreads();   // the previous batch is walked
                    uint32_t b = 0, e = 0;
                    const int g = cb0 + tid;
                    if (tid < kBatch && g < total_cells) {
                        int i = 0;
                        while (g >= s_pre[i + 1]) ++i;
                        const int cell = P.cells[(q * Ns + i) * K + (g - s_pre[i])];
                        const uint32_t* sp = P.split + (size_t(i) * K + cell) * sstride;
                        b = ldg_keep_u32(sp + slab_lo, pol_keep);
                        e = ldg_keep_u32(sp + slab_hi, pol_keep);
                    }
                    uint32_t start, len;
                    chunk_run(b, e, start, len);
                    const uint32_t ev = __reduce_add_sync(kFull, e - b);
                    if (lane == 0 && ev) atomicAdd(&s_ev, ev);
                    if (tid == 0) s_round = 0u;   // read after the staging's barriers
                    const uint2 st = stage_runs<NW>(start, len, rbase, cpre, s_tmp, tid, lane, warp);
                    if (st.x) walk_chunks<NW, WU, CB>(ids4, last_chunk, uint32_t(lo), rlen, st.x, st.y, cnt, out, cap, ge,
                                                      &s_app, &s_round, cpre, rbase, pol_keep, lane, P.status,
                                                      uint32_t(P.counter_words));
                }
            }
            __syncthreads();   // the range's counters, entries and level counts are final
            if (P.dbg_sc) {
                debug_sc<NW, CounterGeom<CB>::kPer, CB>(P, q, lo, hi, words, cnt, tid);
                __syncthreads();   // every counter is read before any is cleared
            }
            if (warp == 0) {
                // the unit's outputs: ge[1] = events - entries (an id with SC = s has s - 1
                // entries), ge[j >= 2] = entries tagged j; then the shared state for the next range
                const uint32_t apps = s_app;
                const bool fits = apps <= cap;
                if (lane == 0) {
                    ge[1] = (staged ? s_ev2[(r - rb) & 1] : s_ev) - apps;
                    P.unit_off[u] = fits ? uint32_t(u) * P.arena_per_unit : 0xffffffffu;
                    P.unit_len[u] = fits ? apps : 0u;
                    if (!fits) P.qflag[q] = 1u;   // entries lost: the query takes the fallback
                }
                __syncwarp();
                if (lane < 16) {
                    P.unit_ge[u * 16 + lane] = ge[lane];
                    ge[lane] = 0u;
                }
                if (lane == 0) {
                    s_app = 0u;
                    s_round = 0u;
                    s_ev = 0u;
                }
            }
            uint4* c4 = reinterpret_cast<uint4*>(cnt);
            for (int w = tid; w < (words + 3) / 4; w += NW * 32) c4[w] = make_uint4(0, 0, 0, 0);
            __syncthreads();   // counters clear, outputs written; range r + 1 is staged
        }
    }
}

}  // namespace taco

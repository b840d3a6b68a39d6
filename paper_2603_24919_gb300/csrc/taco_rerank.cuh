// Fused collision counting (Alg. 6 step 7, Def. 6), query-aware candidate selection
// (Alg. 5) and exact re-rank (Alg. 6 step 9). One thread-block cluster answers a query;
// the clusters of a persistent grid loop over the batch.
//
// Layout: the n point ids are split into slabs of 2^15. CTA r of a cluster owns a
// contiguous range of slabs and holds one 4-bit SC counter per owned id in shared memory
// (N_s <= 15), plus one bit per counter word marking the words the query touched. Cell id
// lists are ascending, so the ids of a probed cell that fall in the CTA's range form one
// contiguous run; a per-cell table of slab boundaries gives the run.
//   1. count:   the runs of all probed cells are staged (start, prefix of lengths) and
//               walked by all warps; each id adds 1 to its nibble with a shared-memory
//               atomic whose old value also tells which SC level the id just reached, so
//               the per-level counts (ids with SC >= j) come for free.
//   2. select:  the cluster sums the per-level counts through distributed shared memory,
//               giving collision_num over all n points; every CTA evaluates Alg. 5 to the
//               same threshold.
//   3. re-rank: the touched words are scanned (and cleared, so the counters are zero for
//               the next query); ids whose SC reaches the threshold are buffered, their rows
//               gathered (G lanes per row, 16-byte loads) and each warp keeps a sorted top
//               list in registers (insertion by ballot + shuffle).
//   4. lists:   every warp writes its sorted top list to global memory. A second kernel
//               merges a query's lists (one warp per query: per CTA, then across the
//               cluster); with BF16 rows the merged list is a shortlist that it re-ranks with
//               FP32 rows before writing the top k.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "taco_internal.h"

namespace taco {
namespace cg = cooperative_groups;

constexpr int kRrThreads = 512;
constexpr int kRrWarps = kRrThreads / 32;
static_assert(kRrWarps == kListsPerCta, "one top list per warp of the fused kernel");
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoId = 0xffffffffu;

struct RerankParams {
    const float* queries;   // [nq][d]
    const float* data;      // [n][d_pad]
    const __nv_bfloat16* data_bf16;  // [n][d_pad]
    const uint8_t* data_fp8;   // [n][dp8] e4m3 of the transformed points
    const float* fp8_scale;    // [2][dp8] per-dimension scale, then 1/scale
    const float* qt;           // [nq][Dp] transformed queries
    const float* obar;         // [d] data mean (FP8 rows of the centred points)
    int Dp, dp8;
    int fp8_space;             // 0: FP8 rows of B^T (o - o_bar), 1: of o - o_bar
    const uint32_t* ids;    // [n_ids] cell lists (16-byte aligned, padded with kIdPad)
    const uint32_t* split;  // [Ns][K][n_slabs+1] absolute positions in ids
    int64_t n_ids;
    const uint16_t* cells;  // [nq][Ns][K]
    const int32_t* ncells;  // [nq][Ns]
    const QueryParamsDev* params;
    QueryParamsDev defaults;
    int64_t n;
    int d, d_pad, Ns, K, n_slabs, slabs_per_cta;
    int counter_words;      // slabs_per_cta * kSlabWords
    int kk;                 // list length (<= 32*R)
    int kkc;                // power of two >= kk
    size_t region_a;        // bytes of the counter region (multiple of 16)
    int64_t nq;             // queries of this launch
    int buf_cap;            // candidate buffer entries: max(kBufCap, 16 * kkc)
    float* lists_d;         // [nq][cluster][kRrWarps][kk] each warp's best kk (dist^2), sorted
    uint32_t* lists_i;      // [nq][cluster][kRrWarps][kk] their ids
    const uint32_t* qmask;  // [nq] or null: only queries with qmask[q] != 0 are processed
    int64_t* out_ids;       // [nq][k_stride] (two-pass form writes results directly)
    float* out_dists;
    int k_stride;
    // two-pass form: per (query, id range) unit
    int n_ranges;           // id ranges per query
    int range_parts;        // count_lists_kernel: work items per query, each a run of its ranges
    int shard_r0, shard_r1; // the ranges this launch counts and selects from (all: 0, n_ranges)
    const int64_t* ghist;   // [nq][N_s + 1] level counts summed over all shards, or null
    uint32_t arena_per_unit;  // arena entries reserved per unit
    uint32_t* unit_ge;      // [nq][n_ranges][16] ids with SC >= j, j = 1..N_s
    uint32_t* unit_off;     // [nq][n_ranges] start of the unit's entries in the arena
    uint32_t* unit_len;     // [nq][n_ranges] entries (one per level >= 2 an id reaches)
    uint32_t* arena;        // entries: id relative to the range | level << 27
    uint32_t* qflag;        // [nq] set when a query needs the fallback (cluster or codes)
    uint32_t* work;         // [2] zeroed query counters of the counting and the select pass
    int* status;            // the index's device status word (checked build: bounds bits)
    size_t arena_words;     // entries of the arena (checked build)
    size_t list_rows;       // rows of kk entries in lists_d / lists_i (checked build)
    int32_t* qlast;         // [nq] last_collision of Alg. 5 of every flagged query
    const uint16_t* codes;  // [Ns][n] cell of every point (codes fallback)
    int fb_mode;            // select_rerank_kernel: 0 two-pass pass 2, 1 codes fallback
    uint8_t* dbg_sc;
    int64_t* dbg_hist;
    int32_t* dbg_last;
    int64_t* dbg_cand;
};

// The next query of a persistent CTA: the grid's first gridDim.x queries are the CTAs' own,
// later ones are handed out in order by an atomic counter (zeroed before the launch), so a
// CTA that drew light queries takes more of them. Block-wide (two barriers).
__device__ __forceinline__ int64_t next_query(uint32_t* counter, int64_t* s_next) {
    __syncthreads();   // every thread holds the current query in a register
    if (threadIdx.x == 0) *s_next = int64_t(gridDim.x) + int64_t(atomicAdd(counter, 1u));
    __syncthreads();
    return *s_next;
}

__device__ __forceinline__ bool lt_pair(float a, uint32_t ia, float b, uint32_t ib) {
    return a < b || (a == b && ia < ib);
}

// Sorted (ascending by (dist, id)) list of 32*R entries spread over a warp: element
// e = 32*r + lane lives in register r of that lane.
template <int R>
struct WarpTop {
    float d[R];
    uint32_t i[R];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            d[r] = __int_as_float(0x7f800000);
            i[r] = kNoId;
        }
    }
    // element kk-1, broadcast to all lanes
    __device__ __forceinline__ void kth(int kk, float& kd, uint32_t& ki) const {
        const int rr = (kk - 1) >> 5, ll = (kk - 1) & 31;
        float v = d[0];
        uint32_t vi = i[0];
#pragma unroll
        for (int r = 1; r < R; ++r)
            if (r == rr) {
                v = d[r];
                vi = i[r];
            }
        kd = __shfl_sync(kFull, v, ll);
        ki = __shfl_sync(kFull, vi, ll);
    }
    // insert (x, xi) (warp-uniform values) if it ranks among the first kk
    __device__ __forceinline__ void insert(float x, uint32_t xi, int kk, int lane) {
        int pos = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) pos += __popc(__ballot_sync(kFull, lt_pair(d[r], i[r], x, xi)));
        if (pos >= kk) return;
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            float up = __shfl_up_sync(kFull, d[r], 1);
            uint32_t upi = __shfl_up_sync(kFull, i[r], 1);
            float cd = x;
            uint32_t ci = xi;
            if (r > 0) {
                cd = __shfl_sync(kFull, d[r > 0 ? r - 1 : 0], 31);
                ci = __shfl_sync(kFull, i[r > 0 ? r - 1 : 0], 31);
            }
            if (lane == 0) {
                up = cd;
                upi = ci;
            }
            const int e = r * 32 + lane;
            if (e > pos) {
                d[r] = up;
                i[r] = upi;
            } else if (e == pos) {
                d[r] = x;
                i[r] = xi;
            }
        }
    }
};

__device__ __forceinline__ float sq4(float4 o, float4 q, float acc) {
    float dx = o.x - q.x;
    acc = fmaf(dx, dx, acc);
    dx = o.y - q.y;
    acc = fmaf(dx, dx, acc);
    dx = o.z - q.z;
    acc = fmaf(dx, dx, acc);
    dx = o.w - q.w;
    return fmaf(dx, dx, acc);
}

// Row kinds of the re-rank: FP32 rows, BF16 rows, FP8-e4m3 rows of the transformed points.
constexpr int kRowF32 = 0, kRowBF16 = 1, kRowFP8 = 2;

// Row chunk = 16 bytes: 4 floats, 8 bf16 or 16 e4m3.
template <int RK>
struct RowChunk {
    static constexpr int kElems = RK == kRowF32 ? 4 : (RK == kRowBF16 ? 8 : 16);
};

// L2 eviction policies: candidate rows are read once per query and streamed (evict
// first); the cell id lists and slab tables are re-read by every query and kept (evict
// last), so the row stream does not push them out of L2.
__device__ __forceinline__ uint64_t l2_policy_stream() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ldg_stream_u4(const void* p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ldg_keep_u32(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
// PTX shl / shr clamp a shift amount above 32 to 32, so a shift by >= 32 gives 0 (a C++
// shift by >= 32 is undefined).
__device__ __forceinline__ uint32_t shl_clamped(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t shr_clamped(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("shr.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// FP8 rows: the query's coordinates are divided by kFp8Pre (and clamped to kFp8Clamp / kFp8Pre)
// in half precision, so that a difference is at most (kFp8Clamp + 448) / kFp8Pre = 70, its
// square at most 4,900 and a half2 lane's sum over 8 dimensions at most 39,200 < 65,504.
constexpr float kFp8Pre = 32.f;
constexpr float kFp8Clamp = 4.f * 448.f;

// Squared distance contribution of one 16-byte row chunk f. FP32 / BF16: qv is the query
// (d_pad floats). FP8: qv holds 48 bytes per chunk, the query's 16 coordinates in half
// precision (q'_c / scale_f / kFp8Pre) and the chunk's weight scale_f^2 kFp8Pre^2 as a float;
// the chunk adds scale_f^2 sum_c (q'_c / scale_f - x8_c)^2 = sum_c (q'_c - scale_f x8_c)^2,
// the 16 squares formed and summed in half2 (two 8-term sums) and weighted in FP32.
template <int RK>
__device__ __forceinline__ float chunk_dist(uint4 raw, const float* qv, int f, float acc) {
    if constexpr (RK == kRowF32) {
        const float4 o = make_float4(__uint_as_float(raw.x), __uint_as_float(raw.y),
                                     __uint_as_float(raw.z), __uint_as_float(raw.w));
        const float4 q = reinterpret_cast<const float4*>(qv)[f];
        return sq4(o, q, acc);
    } else if constexpr (RK == kRowBF16) {
        const float4 q0 = reinterpret_cast<const float4*>(qv)[2 * f];
        const float4 q1 = reinterpret_cast<const float4*>(qv)[2 * f + 1];
        const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
        const float2 a0 = __bfloat1622float2(b[0]);
        const float2 a1 = __bfloat1622float2(b[1]);
        const float2 a2 = __bfloat1622float2(b[2]);
        const float2 a3 = __bfloat1622float2(b[3]);
        acc = sq4(make_float4(a0.x, a0.y, a1.x, a1.y), q0, acc);
        return sq4(make_float4(a2.x, a2.y, a3.x, a3.y), q1, acc);
    } else {
        // chunk f's 48 bytes of the query: 16 halves, then its float weight (the 48-byte
        // stride puts the G lanes of a row, reading consecutive chunks, on different banks)
        const unsigned char* qc = reinterpret_cast<const unsigned char*>(qv) + 48 * f;
        const uint4 qa = *reinterpret_cast<const uint4*>(qc);
        const uint4 qb = *reinterpret_cast<const uint4*>(qc + 16);
        const float w = *reinterpret_cast<const float*>(qc + 32);
        const uint32_t qp[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
        const __half2 neg_pre = __float2half2_rn(-1.f / kFp8Pre);
        __half2 s2 = __float2half2_rn(0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const __half2 x2(__nv_cvt_fp8x2_to_halfraw2(
                    __nv_fp8x2_storage_t((w4[u] >> (16 * h)) & 0xffffu), __NV_E4M3));
                __half2 q2;
                memcpy(&q2, &qp[2 * u + h], 4);
                const __half2 dd = __hfma2(x2, neg_pre, q2);   // (q_c - x_c) / kFp8Pre
                s2 = __hfma2(dd, dd, s2);
            }
        }
        const float2 sf = __half22float2(s2);
        return fmaf(w, sf.x + sf.y, acc);
    }
}

// Squared distances of up to CPW*U queued candidates to the query, G lanes per row.
// Lane-group leaders (gl == 0) end with the full sums; val/cid tell which are real.
template <int G, int RK>
__device__ __forceinline__ void gather_distances(const unsigned char* base, size_t row_bytes,
                                                 int nch, const float* qv, const uint32_t* buf,
                                                 int b0, int m, float (&acc)[2], uint32_t (&cid)[2],
                                                 bool (&val)[2], int gid, int gl, uint64_t pol) {
    constexpr int CPW = 32 / G;
    constexpr int U = 2;
    constexpr int CH = 2;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * CPW + gid;
        val[u] = idx < m;
        cid[u] = val[u] ? buf[idx] : 0u;
        acc[u] = 0.f;
    }
    for (int f0 = 0; f0 < nch; f0 += G * CH) {
        uint4 raw[U][CH];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                const int f = f0 + ch * G + gl;
                raw[u][ch] = (val[u] && f < nch)
                                 ? ldg_stream_u4(base + size_t(cid[u]) * row_bytes + size_t(f) * 16, pol)
                                 : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                const int f = f0 + ch * G + gl;
                if (f < nch) acc[u] = chunk_dist<RK>(raw[u][ch], qv, f, acc[u]);
            }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int off = G / 2; off; off >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], off);
    }
}

// Exclusive scan of two values over the block; tmp holds 2 * NW entries.
template <int NW = kRrWarps>   // warps of the block
__device__ __forceinline__ uint2 block_excl_scan2(uint32_t a, uint32_t b, uint32_t* tmp, uint2& total,
                                                  int lane, int warp) {
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t ta = __shfl_up_sync(kFull, ia, off), tb = __shfl_up_sync(kFull, ib, off);
        if (lane >= off) { ia += ta; ib += tb; }
    }
    if (lane == 31) { tmp[warp] = ia; tmp[NW + warp] = ib; }
    __syncthreads();
    uint32_t pa = 0, pb = 0, sa = 0, sb = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t xa = tmp[w], xb = tmp[NW + w];
        pa += w < warp ? xa : 0u;
        pb += w < warp ? xb : 0u;
        sa += xa;
        sb += xb;
    }
    __syncthreads();
    total = make_uint2(sa, sb);
    return make_uint2(pa + ia - a, pb + ib - b);
}

constexpr int kCellBatch = 512;    // probed cells staged per walk
constexpr int kRunPad = 36;        // boundary entries past the last staged run (>= 33)
constexpr int kBufCap = 4096;      // candidate ids buffered per re-rank round (>= 8 * kRrThreads)
constexpr int kListCap = 4096;     // ids that reached a level >= 2 during counting
constexpr int kWalkUnroll = 8;     // id loads in flight per lane while counting (<= 32)
constexpr int kLevelShift = 27;    // list entry: id relative to the CTA range | level << 27
constexpr uint32_t kPastEnd = 0x80000000u;   // walk lane past the end (relative ids < 12 * 2^15 < 2^26)

// Compact the runs (start, len) held one per thread into the staged form described below:
// the non-empty ones in thread order. Block-wide; ends with a barrier.
template <int NW = kRrWarps>   // warps of the block
__device__ __forceinline__ uint2 stage_runs(uint32_t start, uint32_t len, uint32_t* rbase, uint32_t* cpre,
                                            uint32_t* s_tmp, int tid, int lane, int warp) {
    uint2 tot;
    const uint2 ex = block_excl_scan2<NW>(len, len != 0u ? 1u : 0u, s_tmp, tot, lane, warp);
    if (len != 0u) {
        cpre[ex.y] = ex.x;
        rbase[ex.y] = start - ex.x;
    }
    if (tid <= 32) cpre[tot.y + uint32_t(tid)] = tid == 0 ? tot.x : 0xffffffffu;
    __syncthreads();
    return tot;
}

// Stage the non-empty id runs of probed cells [cb0, cb0 + nb) of query q that fall in slabs
// [slab_lo, slab_hi), in cell order. Element e of the concatenation lies in run r with
// cpre[r] <= e < cpre[r + 1]; its id-array index is rbase[r] + e (uint32 arithmetic:
// the id array holds fewer than 2^32 entries). cpre[nr] = total and cpre[nr + 1 .. nr + 32] = 0xffffffff. Returns
// (total, nr). Block-wide; ends with a barrier.
template <int NW = kRrWarps>   // warps of the block
__device__ __forceinline__ uint2 stage_cells(const RerankParams& P, int64_t q, const int* s_pre,
                                             int cb0, int nb, int slab_lo, int slab_hi,
                                             uint32_t* rbase, uint32_t* cpre,
                                             uint32_t* s_tmp, int tid, int lane, int warp,
                                             uint64_t keep) {
    const int Ns = P.Ns, K = P.K;
    const int sstride = P.n_slabs + 1;
    uint32_t len = 0, start = 0;
    if (tid < nb) {
        const int g = cb0 + tid;
        int i = 0;
        while (g >= s_pre[i + 1]) ++i;
        const int cell = P.cells[(q * Ns + i) * K + (g - s_pre[i])];
        const uint32_t* sp = P.split + (size_t(i) * K + cell) * sstride;
        const uint32_t b = ldg_keep_u32(sp + slab_lo, keep), e = ldg_keep_u32(sp + slab_hi, keep);
        start = b;   // absolute position in the id array
        len = e - b;
    }
    return stage_runs<NW>(start, len, rbase, cpre, s_tmp, tid, lane, warp);
}

// Cell whose run holds element `key` of the concatenation (largest c with cpre[c] <= key).
__device__ __forceinline__ int find_cell(const uint32_t* cpre, int nb, uint32_t key) {
    int lo_c = 0, hi_c = nb - 1;
    while (lo_c < hi_c) {
        const int mid = (lo_c + hi_c + 1) >> 1;
        if (cpre[mid] <= key) lo_c = mid;
        else hi_c = mid - 1;
    }
    return lo_c;
}

// k-way merge of `nl` sorted lists (list j at ld/li + j*stride, each of length kk) into the
// first kk entries of (od, oi), by one full warp: lane j holds the head of list j, and each
// round moves the smallest (dist, id) head (ties by lane) to the output. nl <= 32.
__device__ __forceinline__ void warp_merge(const float* ld, const uint32_t* li, int stride,
                                           int nl, int kk, float* od, uint32_t* oi, int lane) {
    int p = 0;
    for (int o = 0; o < kk; ++o) {
        float v = __int_as_float(0x7f800000);
        uint32_t vi = kNoId;
        if (lane < nl && p < kk) {
            v = ld[lane * stride + p];
            vi = li[lane * stride + p];
        }
        float bv = v;
        uint32_t bi = vi;
        int bl = lane;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const float ov = __shfl_xor_sync(kFull, bv, off);
            const uint32_t oi2 = __shfl_xor_sync(kFull, bi, off);
            const int ol = __shfl_xor_sync(kFull, bl, off);
            if (lt_pair(ov, oi2, bv, bi) || (ov == bv && oi2 == bi && ol < bl)) {
                bv = ov;
                bi = oi2;
                bl = ol;
            }
        }
        if (lane == bl) ++p;
        if (lane == 0) {
            od[o] = bv;
            oi[o] = bi;
        }
    }
}

// Warp-aggregated append: lanes with `take` get consecutive slots after one atomicAdd on
// *counter by the warp; returns the lane's slot (undefined where !take). All lanes call it.
__device__ __forceinline__ uint32_t warp_append_slot(bool take, uint32_t* counter, int lane) {
    const unsigned bal = __ballot_sync(kFull, take);
    uint32_t base = 0;
    if (bal) {
        const int leader = __ffs(bal) - 1;
        if (lane == leader) base = atomicAdd(counter, uint32_t(__popc(bal)));
        base = __shfl_sync(kFull, base, leader);
    }
    return base + __popc(bal & ((1u << lane) - 1u));
}

// s_pre[i] = number of probed cells of query q in subspaces < i (one warp, all lanes).
__device__ __forceinline__ void load_cell_prefix(const RerankParams& P, int64_t q, int* s_pre, int lane) {
    int v = lane < P.Ns ? P.ncells[q * P.Ns + lane] : 0;
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const int t = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += t;
    }
    if (lane < P.Ns) s_pre[lane + 1] = v;
    if (lane == 0) s_pre[0] = 0;
}

// Shared-memory state of the counting phase of one (query, id range) unit.
struct CountSmem {
    uint32_t* cnt;                 // 4-bit SC counters of the range
    uint32_t* lst;                 // kListCap level entries
    uint32_t* rbase;               // staged runs: id-array index minus the run's prefix
    uint32_t* cpre;                // staged run boundaries (kCellBatch + kRunPad)
    uint32_t* ge;                  // [16] ids with SC >= j
    int* s_pre;                    // prefix of probed cells per subspace
    uint32_t* s_tmp;               // block-scan scratch
    uint32_t* s_listn;             // entries appended to lst
};

// Count the collisions of query q in ids [lo, hi) (slabs [slab_lo, slab_hi)) into sm.cnt,
// fill ge[1..N_s] and the level list. SC[id] += 1 for every id of every probed cell; the
// nibble's old value v says the id just reached level v + 1. Ids reaching a level >= 2 are
// appended to the list sm.lst with that level, so every id with SC >= j >= 2 is there
// exactly once tagged j; ge[1] is the number of events minus the level >= 2 events (an id
// with SC = c contributes c events, c - 1 of which reach a level >= 2). *sm.s_listn (zero on
// entry) ends as the number of appends; more than kListCap means the list overflowed, and
// then ge[2..] were counted from the counters. Returns true on overflow. Block-wide; all
// threads return after a barrier with s_pre set by the caller.
// Walk one staged batch (total elements in nr non-empty runs) of the range starting at id
// lo: counters, list appends and *sm.s_listn. The concatenated runs are walked in rounds of
// kWalkUnroll windows of 32 consecutive elements, round g by warp g mod NW, with all
// loads of a round in flight. Lane u finds the run holding the first element of window u
// (binary search); in a window, lane j reads the j-th next run boundary, the boundaries
// inside the window form a bit mask, and a lane's run is the window's first run plus the
// mask bits at or below it (runs are non-empty, so at most 32 boundaries fall in a window).
// Every window is executed in full: lanes past the end load a valid id-array entry and add
// 0 to counter word 0. WU windows per round (WU id loads in flight per lane). Warp-level; no
// barrier.
template <int NW = kRrWarps, int WU = kWalkUnroll>   // warps of the block, windows per round
__device__ __forceinline__ void walk_batch(const RerankParams& P, int64_t lo, uint32_t total, uint32_t nr,
                                           const CountSmem& sm, uint64_t pol_keep, int lane, int warp) {
    static_assert(WU >= 1 && WU <= 32, "one lane finds the run of each window of a round");
    const uint32_t lane_le = (2u << lane) - 1u;  // lanes 0..lane
    const uint32_t last_idx = uint32_t(P.n_ids) - 1u;
    constexpr uint32_t kRound = 32u * WU;
    const uint32_t nrounds = (total + kRound - 1) / kRound;
    for (uint32_t g = uint32_t(warp); g < nrounds; g += NW) {   // warp-uniform
        const uint32_t e = g * kRound;
        const uint32_t key = min(e + 32u * uint32_t(lane % WU), total - 1u);
        const uint32_t cwl = uint32_t(find_cell(sm.cpre, int(nr), key));
        uint32_t idv[WU];
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            const uint32_t E = e + 32u * uint32_t(u);
            const uint32_t cw = __shfl_sync(kFull, cwl, u);
            const uint32_t pb = sm.cpre[cw + 1u + uint32_t(lane)] - E;   // >= 1 inside
            const uint32_t mask = __reduce_or_sync(kFull, shl_clamped(1u, pb));   // 0 for pb >= 32
            const uint32_t r = min(cw + __popc(mask & lane_le), nr - 1u);
            const uint32_t xr = sm.rbase[r] + E + uint32_t(lane);
            (void)TACO_CHECK(P.status, E + uint32_t(lane) >= total || xr <= last_idx, kStatusCluster);
            const uint32_t x = min(xr, last_idx);
            const uint32_t v = ldg_keep_u32(P.ids + x, pol_keep);
            idv[u] = E + uint32_t(lane) < total ? v - uint32_t(lo) : kPastEnd;
        }
        // all counter atomics first (independent), then the ids that reached level >= 2
        // go to the list: one reservation per round, offsets by ballot. A lane past the end
        // (kPastEnd) gets nibble shift 32 and word 0: it adds 0 and reads level 0.
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            const uint32_t id = idv[u];
            const uint32_t sh = ((id << 2) & 28u) | (id >> 26);
            const uint32_t old = atomicAdd(&sm.cnt[(id & ~kPastEnd) >> 3], shl_clamped(1u, sh));
            const uint32_t v = shr_clamped(old, sh) & 15u;
            idv[u] = v != 0u ? (id | ((v + 1u) << kLevelShift)) : 0u;
        }
        unsigned bal[WU];
        uint32_t napp = 0;
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            bal[u] = __ballot_sync(kFull, idv[u] != 0u);
            napp += __popc(bal[u]);
        }
        uint32_t at = 0;
        if (lane == 0 && napp) at = atomicAdd(sm.s_listn, napp);
        at = __shfl_sync(kFull, at, 0);
#pragma unroll
        for (int u = 0; u < WU; ++u) {
            const uint32_t a = at + __popc(bal[u] & (lane_le >> 1));
            if (idv[u] != 0u && a < uint32_t(kListCap)) sm.lst[a] = idv[u];
            at += __popc(bal[u]);
        }
    }
}

// The level list overflowed: ge[2..N_s] from the counters themselves (SWAR compare of the
// eight nibbles of a word against each level), and ge[1] loses the level >= 2 events.
// Block-wide over the counter words; no barrier.
template <int NW = kRrWarps>   // warps of the block
__device__ __forceinline__ void levels_from_counters(int Ns, int words, const CountSmem& sm, int tid, int lane) {
    uint32_t gel[TACO_MAX_SUBSPACES];
#pragma unroll
    for (int j = 0; j < TACO_MAX_SUBSPACES; ++j) gel[j] = 0;
    for (int w = tid; w < words; w += (NW * 32)) {
        const uint32_t x = sm.cnt[w];
        if (x == 0u) continue;
        const uint32_t ev = x & 0x0f0f0f0fu, od = (x >> 4) & 0x0f0f0f0fu;
#pragma unroll
        for (int j = 2; j <= TACO_MAX_SUBSPACES; ++j) {
            if (j <= Ns) {
                const uint32_t add = (0x80u - uint32_t(j)) * 0x01010101u;
                gel[j - 1] += __popc((ev + add) & 0x80808080u) + __popc((od + add) & 0x80808080u);
            }
        }
    }
    uint32_t events = 0;   // level >= 2 events of this warp's words
#pragma unroll
    for (int j = 2; j <= TACO_MAX_SUBSPACES; ++j) {
        if (j <= Ns) {
            const uint32_t v = __reduce_add_sync(kFull, gel[j - 1]);
            events += v;
            if (lane == 0 && v) atomicAdd(&sm.ge[j], v);
        }
    }
    if (lane == 0 && events) atomicSub(&sm.ge[1], events);
}

// After the walks of a range (and a barrier): ge[2..N_s] from the list, or from the
// counters if the list overflowed; ge[1] loses the level >= 2 events. Returns true on
// overflow. Block-wide; ends with a barrier.
template <int NW = kRrWarps>   // warps of the block
__device__ __forceinline__ bool finish_levels(const RerankParams& P, int words, const CountSmem& sm,
                                              int tid, int lane, int warp) {
    const uint32_t nlist = *sm.s_listn;
    const bool overflow = nlist > uint32_t(kListCap);
    if (!overflow) {
        // lanes holding the same level form one group, whose lowest lane adds its size
        const uint32_t lane_lt = (1u << lane) - 1u;
        for (uint32_t e0 = uint32_t(warp) * 32u; e0 < nlist; e0 += (NW * 32)) {
            const uint32_t e = e0 + uint32_t(lane);
            const uint32_t level = e < nlist ? sm.lst[e] >> kLevelShift : 0u;
            const unsigned grp = __match_any_sync(kFull, level);
            if (level != 0u && (grp & lane_lt) == 0u) atomicAdd(&sm.ge[level], uint32_t(__popc(grp)));
        }
        if (tid == 0 && nlist) atomicSub(&sm.ge[1], nlist);
    } else {
        levels_from_counters<NW>(P.Ns, words, sm, tid, lane);
    }
    __syncthreads();
    return overflow;
}

// FINISH = false: return after the last walk, without a barrier and without the level
// counts (the caller counts them); the return value is then meaningless.
template <int NW = kRrWarps, int WU = kWalkUnroll, bool FINISH = true>
__device__ __forceinline__ bool count_phase(const RerankParams& P, int64_t q, int slab_lo, int slab_hi,
                                            int64_t lo, int words, const CountSmem& sm, uint64_t pol_keep,
                                            int tid, int lane, int warp) {
    const int total_cells = sm.s_pre[P.Ns];
    const int nbatch = (total_cells + kCellBatch - 1) / kCellBatch;
    for (int bt = 0; bt < nbatch; ++bt) {
        const int cb0 = bt * kCellBatch;
        const int nb = min(kCellBatch, total_cells - cb0);
        const uint2 st = stage_cells<NW>(P, q, sm.s_pre, cb0, nb, slab_lo, slab_hi, sm.rbase,
                                     sm.cpre, sm.s_tmp, tid, lane, warp, pol_keep);
        if (tid == 0 && st.x) atomicAdd(&sm.ge[1], st.x);   // minus the level >= 2 events later
        walk_batch<NW, WU>(P, lo, st.x, st.y, sm, pol_keep, lane, warp);
        if (bt + 1 < nbatch) __syncthreads();   // staging is reused by the next batch
    }
    if (!FINISH) return false;
    __syncthreads();
    return finish_levels<NW>(P, words, sm, tid, lane, warp);
}

// Debug: the SC of every touched id of the range (untouched ids stay at the caller's zero).
template <int NW = kRrWarps, int PER = 8, int CB = 4>   // warps of the block, counters a word, bits
__device__ __forceinline__ void debug_sc(const RerankParams& P, int64_t q, int64_t lo, int64_t hi,
                                        int words, const uint32_t* cnt, int tid) {
    constexpr uint32_t kMask = (1u << CB) - 1u;
    for (int w = tid; w < words; w += (NW * 32)) {
        const uint32_t x = cnt[w];
        if (!x) continue;
        const int64_t id0 = lo + int64_t(w) * PER;
        for (int j = 0; j < PER && id0 + j < hi; ++j)
            if ((x >> (CB * j)) & kMask) P.dbg_sc[q * P.n + id0 + j] = uint8_t((x >> (CB * j)) & kMask);
    }
}

// G lanes per candidate, R registers per lane of top list, BF16 rows or FP32 rows.
// Persistent: the clusters of the grid take queries blockIdx.y, blockIdx.y + gridDim.y, ...
template <int G, int R, bool BF16>
__global__ void __launch_bounds__(kRrThreads, (R <= 4 ? 2 : 1))
count_select_rerank_kernel(const RerankParams P) {
    constexpr int CPW = 32 / G;   // candidates per warp pass
    constexpr int U = 2;          // passes in flight
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = int(cluster.block_rank());
    const int ncta = int(cluster.num_blocks());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);                          // counters
    float* qv = reinterpret_cast<float*>(smem + P.region_a);                     // d_pad
    uint32_t* buf = reinterpret_cast<uint32_t*>(qv + P.d_pad);                   // buf_cap
    uint32_t* lst = buf + P.buf_cap;                                             // kListCap
    uint32_t* rbase = lst + kListCap;                                            // kCellBatch
    uint32_t* cpre = rbase + kCellBatch;                                         // kCellBatch+kRunPad
    uint32_t* ge2 = cpre + kCellBatch + kRunPad;                                 // [2][16]
    __shared__ int s_pre[TACO_MAX_SUBSPACES + 1];
    __shared__ int s_last;
    __shared__ uint32_t s_tmp[2 * kRrWarps];
    __shared__ uint32_t s_wcnt[2][kRrWarps];
    __shared__ uint32_t s_allge2[2][16 * 16];   // [parity][cta][level], filled by every CTA
    __shared__ uint32_t s_bufn, s_app;
    __shared__ uint32_t s_gs[TACO_MAX_SUBSPACES + 1];

    const int Ns = P.Ns;
    const int slab_lo = cta * P.slabs_per_cta;
    const int slab_hi = min(slab_lo + P.slabs_per_cta, P.n_slabs);
    const int64_t lo = int64_t(slab_lo) << kSlabLog2;
    const int64_t hi = min(int64_t(slab_hi) << kSlabLog2, P.n);
    const int words = hi > lo ? int((hi - lo + 7) >> 3) : 0;
    const int gid = lane / G, gl = lane % G;
    const int nch = P.d_pad / RowChunk<BF16>::kElems;
    const size_t row_bytes = size_t(P.d_pad) * (BF16 ? 2 : 4);
    const unsigned char* rows = BF16 ? reinterpret_cast<const unsigned char*>(P.data_bf16)
                                     : reinterpret_cast<const unsigned char*>(P.data);
    const int kk = P.kk;
    const uint64_t pol_keep = l2_policy_keep(), pol_stream = l2_policy_stream();
    CountSmem csm;
    csm.cnt = cnt;
    csm.lst = lst;
    csm.rbase = rbase;
    csm.cpre = cpre;
    csm.s_pre = s_pre;
    csm.s_tmp = s_tmp;
    csm.s_listn = &s_app;

    // counters start at zero; every query leaves them at zero again
    for (int w = tid; w < P.counter_words; w += kRrThreads) cnt[w] = 0u;
    if (tid < 32) ge2[tid] = 0u;

    int par = 0;
    for (int64_t q = blockIdx.y; q < P.nq; q += gridDim.y, par ^= 1) {
        if (P.qmask && !P.qmask[q]) continue;   // same decision in every CTA of the cluster
        const QueryParamsDev qp = P.params ? P.params[q] : P.defaults;
        // this query's list length: its k or shortlist (lists are allotted the batch's
        // longest, kk; a query's answer is the first qp.kk of its merged list, and each
        // warp's first qp.kk entries hold its qp.kk nearest)
        const int kq = min(qp.kk, kk);
        uint32_t* ge = ge2 + 16 * par;
        uint32_t* s_allge = s_allge2[par];
        csm.ge = ge;
        __syncthreads();   // the previous query's readers of qv / s_pre / lists are done
        for (int j = tid; j < P.d_pad; j += kRrThreads)
            qv[j] = j < P.d ? P.queries[q * P.d + j] : 0.f;
        if (tid < 16) ge[tid] = 0u;
        if (warp == 0) load_cell_prefix(P, q, s_pre, lane);
        if (tid == 0) {
            s_app = 0u;
            s_bufn = 0u;
        }
        __syncthreads();

        // ---- 1. count the collisions of the probed cells' ids in this CTA's range
        const bool overflow = count_phase(P, q, slab_lo, slab_hi, lo, words, csm, pol_keep, tid, lane, warp);
        // push this CTA's level counts into row `cta` of every CTA's table
        if (tid < ncta * Ns) {
            const int r = tid / Ns, j = tid - r * Ns + 1;
            cluster.map_shared_rank(s_allge, r)[cta * 16 + j] = ge[j];
        }
        cluster.sync();

        // ---- 2. Alg. 5 on the cluster-wide collision_num (same result in every CTA) ----
        if (tid < Ns) {
            uint32_t v = 0;
            for (int r = 0; r < ncta; ++r) v += s_allge[r * 16 + tid + 1];
            s_gs[tid + 1] = v;
        }
        __syncthreads();
        if (tid == 0) {
            long long gs[TACO_MAX_SUBSPACES + 2];
            gs[0] = P.n;
            for (int j = 1; j <= Ns; ++j) gs[j] = s_gs[j];
            gs[Ns + 1] = 0;
            int last = Ns;
            long long cand = 0;
            for (int j = Ns; j >= 0; --j) {
                const long long h = gs[j] - gs[j + 1];
                cand += h;
                const bool go = qp.select_rule == TACO_SELECT_LITERAL ? (h <= qp.rerank_target - cand)
                                                                     : (cand <= qp.rerank_target);
                if (go) --last;
                else break;
            }
            s_last = last;
            if (cta == 0) {
                if (P.dbg_hist)
                    for (int j = 0; j <= Ns; ++j) P.dbg_hist[q * (Ns + 1) + j] = gs[j] - gs[j + 1];
                if (P.dbg_last) P.dbg_last[q] = last;
                if (P.dbg_cand) P.dbg_cand[q] = cand;
            }
        }
        __syncthreads();
        const int last = s_last;

        // ---- 3. candidates of this CTA -> warp top lists --------------------------------
        WarpTop<R> top;
        top.init();
        float kth_d = __int_as_float(0x7f800000);
        uint32_t kth_i = kNoId;
        auto rerank_buffer = [&](int m) {
            for (int b0 = warp * CPW * U; b0 < m; b0 += kRrWarps * CPW * U) {
                float acc[U];
                uint32_t cid[U];
                bool val[U];
                gather_distances<G, BF16>(rows, row_bytes, nch, qv, buf, b0, m, acc, cid, val, gid, gl,
                                          pol_stream);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool better = val[u] && gl == 0 && lt_pair(acc[u], cid[u], kth_d, kth_i);
                    unsigned bal = __ballot_sync(kFull, better);
                    while (bal) {
                        const int src = __ffs(bal) - 1;
                        bal &= bal - 1;
                        const float x = __shfl_sync(kFull, acc[u], src);
                        const uint32_t xi = __shfl_sync(kFull, cid[u], src);
                        if (lt_pair(x, xi, kth_d, kth_i)) {
                            top.insert(x, xi, kq, lane);
                            top.kth(kq, kth_d, kth_i);
                        }
                    }
                }
            }
        };
        const uint32_t mine = last >= 1 ? s_allge[cta * 16 + last] : 0u;   // ids with SC >= last
        if (P.dbg_sc && last >= 1) {
            debug_sc(P, q, lo, hi, words, cnt, tid);
            __syncthreads();   // every counter is read before any is cleared below
        }
        if (last >= 2 && !overflow && mine <= uint32_t(P.buf_cap)) {
            // the candidates are the list entries tagged `last`
            {
                const uint32_t nlist = s_app;   // <= kListCap: no overflow
                for (uint32_t e0 = uint32_t(warp) * 32u; e0 < nlist; e0 += kRrThreads) {
                    const uint32_t e = e0 + uint32_t(lane);
                    const uint32_t x = e < nlist ? lst[e] : 0u;
                    const bool take = e < nlist && int(x >> kLevelShift) == last;
                    const uint32_t at = warp_append_slot(take, &s_bufn, lane);
                    if (take && TACO_CHECK(P.status, at < uint32_t(P.buf_cap), kStatusCluster))
                        buf[at] = uint32_t(lo) + (x & ((1u << kLevelShift) - 1u));
                }
            }
            // clear the counters for the next query
            uint4* c4 = reinterpret_cast<uint4*>(cnt);
            for (int w = tid; w < (words + 3) / 4; w += kRrThreads) c4[w] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            rerank_buffer(int(s_bufn));
        } else if (last >= 1) {
            // SC >= 1 (or an overflowing list): scan every counter word in tiles of
            // kRrThreads words (at most 8 * kRrThreads ids each), clearing it; the buffer is
            // re-ranked and emptied before a tile that would not fit
            uint32_t bufn = 0;
            int wpar = 0;
            const uint32_t add = (0x80u - uint32_t(last)) * 0x01010101u;
            for (int t0 = 0; t0 < words; t0 += kRrThreads) {
                const int w = t0 + tid;
                uint32_t m8 = 0;
                const int64_t id0 = lo + (int64_t(w) << 3);
                if (w < words) {
                    const uint32_t x = cnt[w];
                    if (x) {
                        cnt[w] = 0u;
                        const uint32_t he = ((x & 0x0f0f0f0fu) + add) & 0x80808080u;
                        const uint32_t ho = (((x >> 4) & 0x0f0f0f0fu) + add) & 0x80808080u;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            m8 |= ((he >> (8 * b + 7)) & 1u) << (2 * b);
                            m8 |= ((ho >> (8 * b + 7)) & 1u) << (2 * b + 1);
                        }
                    }
                }
                const uint32_t cnum = __popc(m8);
                uint32_t incl = cnum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off) incl += v;
                }
                if (lane == 31) s_wcnt[wpar][warp] = incl;
                __syncthreads();
                uint32_t wbase = 0, step_total = 0;
#pragma unroll
                for (int ww = 0; ww < kRrWarps; ++ww) {
                    const uint32_t x = s_wcnt[wpar][ww];
                    wbase += ww < warp ? x : 0u;
                    step_total += x;
                }
                if (bufn + step_total > uint32_t(P.buf_cap)) {
                    rerank_buffer(int(bufn));   // entries were written before the barrier above
                    __syncthreads();
                    bufn = 0;
                }
                uint32_t at = bufn + wbase + incl - cnum;
                while (m8) {
                    const int j = __ffs(m8) - 1;
                    m8 &= m8 - 1;
                    if (TACO_CHECK(P.status, at < uint32_t(P.buf_cap), kStatusCluster)) buf[at] = uint32_t(id0 + j);
                    ++at;
                }
                bufn += step_total;
                wpar ^= 1;
            }
            __syncthreads();
            rerank_buffer(int(bufn));
        } else {
            // Alg. 5 kept every level: all ids of this CTA's range are candidates.
            if (P.dbg_sc) {
                for (int w = tid; w < words; w += kRrThreads) {
                    const uint32_t x = cnt[w];
                    for (int j = 0; j < 8 && lo + 8 * w + j < hi; ++j)
                        P.dbg_sc[q * P.n + lo + 8 * w + j] = uint8_t((x >> (4 * j)) & 15u);
                }
            }
            for (int64_t b = lo; b < hi; b += P.buf_cap) {
                const int m = int(hi - b < int64_t(P.buf_cap) ? hi - b : int64_t(P.buf_cap));
                __syncthreads();
                for (int t = tid; t < m; t += kRrThreads) buf[t] = uint32_t(b + t);
                __syncthreads();
                rerank_buffer(m);
            }
            __syncthreads();
            for (int w = tid; w < words; w += kRrThreads) cnt[w] = 0u;
        }

        // ---- 4. every warp's best kk go to global memory; a per-query kernel merges them
        {
            const size_t row = ((size_t(q) * ncta + cta) * kRrWarps + warp) * kk;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = r * 32 + lane;
                if (e < kk && TACO_CHECK(P.status, row + e < P.list_rows * size_t(kk), kStatusCluster)) {
                    P.lists_d[row + e] = top.d[r];
                    P.lists_i[row + e] = top.i[r];
                }
            }
        }
    }
    cluster.sync();   // no CTA leaves while another may still write its level table
}

// ---------------------------------------------------------------------------------------
// Two-pass form. Pass 1 (count_lists_kernel, taco_count.cuh) counts the collisions of each
// (query, id range) unit and writes the unit's level counts and, for every level j >= 2 an id
// reaches, an entry (id relative to the range | j << 27) to the unit's arena slot. Pass 2
// (select_rerank_kernel, taco_select.cuh): one CTA per query sums the level counts of its
// ranges, applies Alg. 5, keeps the arena entries tagged last_collision and re-ranks them.
// Queries whose threshold falls below 2, or whose entries did not fit, are flagged for a
// fallback.
// ---------------------------------------------------------------------------------------

template <int G, int R, bool BF16>
cudaError_t launch_rerank_t(const RerankParams& P, int cluster, int64_t nq, size_t smem,
                            cudaStream_t st) {
    auto kern = count_select_rerank_kernel<G, R, BF16>;
    // persistent grid: as many clusters as can be resident at once (cached per shape)
    static thread_local size_t cached_smem = 0;
    static thread_local int cached_cluster = 0, cached_active = 0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return g_launch_step = "an earlier unchecked call", e;
    if (cached_smem != smem || cached_cluster != cluster) {
        e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
        if (e != cudaSuccess) return g_launch_step = "cudaFuncSetAttribute", e;
        if (cluster > 8) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return g_launch_step = "cudaFuncSetAttribute (cluster size)", e;
        }
        cudaLaunchConfig_t occ = {};
        occ.gridDim = dim3(unsigned(cluster), 1, 1);
        occ.blockDim = dim3(kRrThreads, 1, 1);
        occ.dynamicSmemBytes = smem;
        cudaLaunchAttribute oa[1];
        oa[0].id = cudaLaunchAttributeClusterDimension;
        oa[0].val.clusterDim.x = unsigned(cluster);
        oa[0].val.clusterDim.y = 1;
        oa[0].val.clusterDim.z = 1;
        occ.attrs = oa;
        occ.numAttrs = 1;
        int active = 0;
        e = cudaOccupancyMaxActiveClusters(&active, kern, &occ);
        if (e != cudaSuccess) return g_launch_step = "cudaOccupancyMaxActiveClusters", e;
        if (active < 1) return g_launch_step = "occupancy (no cluster fits)", cudaErrorInvalidConfiguration;
        cached_smem = smem;
        cached_cluster = cluster;
        cached_active = active;
    }
    const int64_t gy = nq < cached_active ? nq : cached_active;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cluster), unsigned(gy), 1);
    cfg.blockDim = dim3(kRrThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, P);
    if (e != cudaSuccess) {
        static thread_local char what[160];
        snprintf(what, sizeof(what), "cudaLaunchKernelEx (cluster %d, grid %d x %lld, %zu B shared, %d active)",
                 cluster, cluster, (long long)gy, smem, cached_active);
        g_launch_step = what;
    }
    return e;
}

// One translation unit per (row type, R) instantiates the four G variants.
#define TACO_DECLARE_RERANK(B, R)                                                            \
    cudaError_t launch_rerank_b##B##_r##R(int G, const RerankParams& P, int cluster, int64_t nq, \
                                          size_t smem, cudaStream_t st);
TACO_DECLARE_RERANK(0, 1)
TACO_DECLARE_RERANK(0, 4)
TACO_DECLARE_RERANK(0, 16)
TACO_DECLARE_RERANK(1, 1)
TACO_DECLARE_RERANK(1, 4)
TACO_DECLARE_RERANK(1, 16)
#undef TACO_DECLARE_RERANK
// The select / re-rank pass (taco_select.cuh) per row kind (FP8 rows have this pass only;
// fallback queries re-rank with FP32 rows).
cudaError_t launch_select_b0(int G, const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st);
cudaError_t launch_select_b1(int G, const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st);
cudaError_t launch_select_b2(int G, const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st);

}  // namespace taco

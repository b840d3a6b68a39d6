// Select / re-rank pass of the two-pass search (Alg. 5, Alg. 6 step 9): one CTA per query
// sums the level counts of the query's id ranges, applies Alg. 5 (the threshold
// last_collision over collision_num), takes the listed ids with SC >= last_collision as the
// candidates C and returns the k nearest of them by exact distance. In fallback mode the same
// kernel answers the flagged queries from the cell codes (see below).
//
// The candidates are buffered; a full buffer is flushed in two steps: every warp streams its
// share of the buffered rows (G lanes a row, 16-byte loads) and writes their squared
// distances to shared memory, with no dependency between rows, so each warp keeps its loads
// in flight; then the block keeps the nearest of the buffer and of the list kept so far by a
// radix select on the distance bits and a bitonic sort. With BF16 or FP8 rows the kept list
// is a shortlist that is re-ranked with the FP32 rows before the results are written.
#pragma once

#include "taco_rerank.cuh"

namespace taco {

constexpr int kSrThreads = 256;
constexpr int kSrWarps = kSrThreads / 32;
constexpr int kSrBuf = 4096;   // candidate ids per re-rank round
constexpr int kSelHist = 2048;   // bins of one radix pass of the selection (8 a thread)
// rows a lane group gathers at once in the streaming pass, and the CTAs per SM the kernel is
// compiled for (its register budget), per row kind
template <int RK> constexpr int kGatherRows = RK == kRowBF16 ? 2 : 4;
template <int RK> constexpr int kSelectBlocksPerSm = RK == kRowF32 ? 4 : 3;
constexpr int kEntryLoads = 4;   // arena entries a thread loads per tile of the candidate pass

// Squared distances of U queued candidates per lane group (G lanes a row, rows buf[b0 + u *
// (32 / G) + group]): every 16-byte chunk load of the U rows is issued before any arithmetic
// (chunks past G * CH per lane are loaded in further rounds). Lane-group leaders (gl == 0)
// end with the sums; val / cid tell which are real.
template <int G, int RK, int U, int CH>
__device__ __forceinline__ void gather_rows(const unsigned char* base, size_t row_bytes, int nch, const float* qv,
                                            const uint32_t* buf, int b0, int m, float (&acc)[U],
                                            uint32_t (&cid)[U], bool (&val)[U], int gid, int gl, uint64_t pol) {
    constexpr int CPW = 32 / G;
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

// The kq nearest of the M (squared distance, id) pairs cd / ci go to Md / Mi[0, min(M, kq)),
// sorted by (distance, id), and (inf, kNoId) fills Md / Mi up to kkc; *s_cur = min(M, kq).
// Distances are non-negative, so their bit patterns order like their values: three radix
// passes over the bits (11, 11 and 10 bits) find the kq-th smallest distance T; the pairs below
// T are kept, and of the pairs equal to T those with the smallest ids. Ids are distinct.
// Block-wide (kSrThreads threads); ends with a barrier.
static __device__ __noinline__ void keep_nearest(const float* cd, const uint32_t* ci, int M, int kq, int kkc,
                                          float* Md, uint32_t* Mi, uint32_t* hist, uint32_t* s_cur,
                                          uint32_t* s_n, uint32_t* s_eq, uint32_t* s_bin,
                                          uint32_t* s_before, uint32_t* s_tmp, int tid, int lane,
                                          int warp, int* status) {
    const int take = min(M, kq);
    if (M > kq) {
        uint32_t prefix = 0, need = uint32_t(kq);
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
            const uint32_t bins = pass == 2 ? 0x3ffu : 0x7ffu;
            const uint32_t above = pass == 0 ? 0u : (pass == 1 ? 0xffe00000u : 0xfffffc00u);
            for (int t = tid; t < kSelHist; t += kSrThreads) hist[t] = 0u;
            __syncthreads();
            for (int i = tid; i < M; i += kSrThreads) {
                const uint32_t b = __float_as_uint(cd[i]);
                if ((b & above) == prefix) atomicAdd(&hist[(b >> shift) & bins], 1u);
            }
            __syncthreads();
            // the bin where the running count reaches need
            constexpr int kPer = kSelHist / kSrThreads;
            uint32_t loc = 0;
#pragma unroll
            for (int j = 0; j < kPer; ++j) loc += hist[tid * kPer + j];
            uint32_t incl = loc;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, incl, off);
                if (lane >= off) incl += v;
            }
            if (lane == 31) s_tmp[warp] = incl;
            __syncthreads();
            uint32_t before = incl - loc;
            for (int w = 0; w < warp; ++w) before += s_tmp[w];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const uint32_t h = hist[tid * kPer + j];
                if (before < need && need <= before + h) {
                    *s_bin = uint32_t(tid * kPer + j);
                    *s_before = before;
                }
                before += h;
            }
            __syncthreads();
            prefix |= *s_bin << shift;
            need -= *s_before;
        }
        // prefix = T; `need` of the pairs equal to T are kept
        if (tid == 0) {
            *s_n = 0u;
            *s_eq = 0u;
        }
        __syncthreads();
        for (int i = tid; i < M; i += kSrThreads) {
            const uint32_t b = __float_as_uint(cd[i]);
            if (b < prefix) {
                const uint32_t s = atomicAdd(s_n, 1u);
                if (!TACO_CHECK(status, s < uint32_t(kkc), kStatusSelect)) continue;
                Md[s] = cd[i];
                Mi[s] = ci[i];
            } else if (b == prefix) {
                atomicAdd(s_eq, 1u);
            }
        }
        __syncthreads();
        const uint32_t neq = *s_eq;
        for (int i = tid; i < M; i += kSrThreads) {
            if (__float_as_uint(cd[i]) != prefix) continue;
            bool keep = true;
            if (neq > need) {   // rank among the equal pairs by id
                uint32_t r = 0;
                for (int j = 0; j < M; ++j) r += __float_as_uint(cd[j]) == prefix && ci[j] < ci[i];
                keep = r < need;
            }
            if (keep) {
                const uint32_t s = atomicAdd(s_n, 1u);
                if (!TACO_CHECK(status, s < uint32_t(kkc), kStatusSelect)) continue;
                Md[s] = cd[i];
                Mi[s] = ci[i];
            }
        }
    } else {
        for (int i = tid; i < M; i += kSrThreads) {
            Md[i] = cd[i];
            Mi[i] = ci[i];
        }
    }
    int p2 = 1;
    while (p2 < take) p2 <<= 1;
    for (int t = take + tid; t < kkc; t += kSrThreads) {
        Md[t] = __int_as_float(0x7f800000);
        Mi[t] = kNoId;
    }
    __syncthreads();
    for (int k2 = 2; k2 <= p2; k2 <<= 1) {
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < p2; t += kSrThreads) {
                const int o = t ^ j;
                if (o > t) {
                    const float a = Md[t], b = Md[o];
                    const uint32_t ia = Mi[t], ib = Mi[o];
                    if (lt_pair(b, ib, a, ia) == ((t & k2) == 0)) {
                        Md[t] = b;
                        Mi[t] = ib;
                        Md[o] = a;
                        Mi[o] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) *s_cur = uint32_t(take);
    __syncthreads();
}

// Dynamic shared memory of select_rerank_kernel: lists of kkc entries, the query row, the
// candidate buffer with room for a kept list, the selection histogram, the FP8 query pairs,
// and the mode's extra: the ranges' list offsets (two-pass form) or the probed-cell bitmaps
// and a batch of cell runs (codes fallback).
inline size_t select_smem_bytes(int kkc, int d_pad, int dp8_or_0, int n_ranges, int Ns, int K, bool fallback) {
    size_t b = size_t(4) * kkc * 4 + size_t(d_pad) * 4 + size_t(kSrBuf + TACO_MAX_K) * 8 + size_t(kSelHist) * 4 +
               size_t(dp8_or_0) * 8;
    if (fallback) return b + size_t(Ns) * ((K + 31) / 32) * 4 + size_t(3 * kSrThreads + 1) * 4;
    return b + size_t(2 * n_ranges + 1) * 4;
}


template <int G, int RK>
__global__ void __launch_bounds__(kSrThreads, kSelectBlocksPerSm<RK>)
select_rerank_kernel(const RerankParams P) {
    constexpr int CPW = 32 / G;
    constexpr int U = 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    const int kkc = P.kkc;
    float* Md = reinterpret_cast<float*>(smem);                         // [kkc] the query's list
    uint32_t* Mi = reinterpret_cast<uint32_t*>(Md + kkc);
    float* Xd = reinterpret_cast<float*>(Mi + kkc);                     // [kkc] exact (BF16, FP8)
    uint32_t* Xi = reinterpret_cast<uint32_t*>(Xd + kkc);
    float* qv = reinterpret_cast<float*>(Xi + kkc);                     // d_pad
    float* cd = qv + P.d_pad;                                           // [kSrBuf + TACO_MAX_K]
    uint32_t* ci = reinterpret_cast<uint32_t*>(cd + kSrBuf + TACO_MAX_K);   // candidate ids, same
    uint32_t* hist = ci + kSrBuf + TACO_MAX_K;                          // [kSelHist]
    float* qf = reinterpret_cast<float*>(hist + kSelHist);              // FP8: 48 B a chunk (of 8 dp8)
    // codes fallback: probed-cell bitmaps [Ns][K / 32] and one batch of cells' runs
    uint32_t* fbm = reinterpret_cast<uint32_t*>(qf + (RK == kRowFP8 ? 2 * P.dp8 : 0));
    uint32_t* fpre = fbm + P.Ns * ((P.K + 31) / 32);                    // [kSrThreads + 1]
    uint32_t* fst = fpre + kSrThreads + 1;                              // [kSrThreads]
    uint32_t* fsub = fst + kSrThreads;                                  // [kSrThreads]
    __shared__ int s_fpre[TACO_MAX_SUBSPACES + 1];
    __shared__ uint32_t s_gs[TACO_MAX_SUBSPACES + 2];
    __shared__ int s_last;
    __shared__ uint32_t s_bufn;
    __shared__ uint32_t s_flag;
    __shared__ uint32_t s_tmp2[2 * kSrWarps];
    __shared__ uint32_t s_cur, s_n, s_eq, s_bin, s_before;
    const int Ns = P.Ns, nr = P.n_ranges, kk = P.kk;
    const int gid = lane / G, gl = lane % G;
    constexpr bool kFP8 = RK == kRowFP8;
    // 16-byte chunks of a row that hold coordinates (FP8 rows are padded to whole lines)
    const int nch = kFP8 ? ((P.fp8_space ? P.d : P.Dp) + 15) / 16 : P.d_pad / RowChunk<RK>::kElems;
    const size_t row_bytes = kFP8 ? size_t(P.dp8) : size_t(P.d_pad) * (RK == kRowBF16 ? 2 : 4);
    const unsigned char* rows = RK == kRowBF16 ? reinterpret_cast<const unsigned char*>(P.data_bf16)
                                : kFP8         ? P.data_fp8
                                               : reinterpret_cast<const unsigned char*>(P.data);
    const float* qd = kFP8 ? qf : qv;   // what the candidate distances compare against
    const uint64_t pol_stream = l2_policy_stream();
    __shared__ int64_t s_next;
    // two-pass form: queries handed out by a counter; codes fallback: a fixed stride
    for (int64_t q = blockIdx.x; q < P.nq;
         q = P.fb_mode ? q + gridDim.x : next_query(P.work + 1, &s_next)) {
        const QueryParamsDev qp = P.params ? P.params[q] : P.defaults;
        __syncthreads();
        for (int j = tid; j < P.d_pad; j += kSrThreads) qv[j] = j < P.d ? P.queries[q * P.d + j] : 0.f;
        if constexpr (kFP8) {
            // the query in the FP8 rows' space (the transformed query q', zero past N_s * s,
            // or the centred query q - o_bar, zero past d), per dimension c as
            // x_c / scale_c / kFp8Pre in half precision, clamped to kFp8Clamp / kFp8Pre (a
            // query coordinate beyond 4x the points' largest keeps the half-precision sums of
            // a chunk finite), and per 16-dimension chunk its scale^2 * kFp8Pre^2
            // (48 bytes per 16-dimension chunk: 16 halves, the weight, 12 bytes unused)
            const int cols = P.fp8_space ? P.d : P.Dp;
            unsigned char* qc = reinterpret_cast<unsigned char*>(qf);
            for (int j = tid; j < P.dp8; j += kSrThreads) {
                float x = 0.f;
                if (j < cols) x = P.fp8_space ? P.queries[q * P.d + j] - P.obar[j] : P.qt[q * P.Dp + j];
                const float xs = fminf(fmaxf(x * P.fp8_scale[P.dp8 + j], -kFp8Clamp), kFp8Clamp);
                reinterpret_cast<__half*>(qc + 48 * (j >> 4))[j & 15] =
                    __float2half_rn(j < cols ? xs * (1.f / kFp8Pre) : 0.f);
                if ((j & 15) == 0) {
                    const float sc = P.fp8_scale[j];
                    *reinterpret_cast<float*>(qc + 48 * (j >> 4) + 32) = sc * sc * (kFp8Pre * kFp8Pre);
                }
            }
        }
        if (tid <= TACO_MAX_SUBSPACES + 1) s_gs[tid] = 0u;
        if (tid == 0) {
            s_bufn = 0u;
            s_flag = P.qflag[q];
            if (P.fb_mode) s_last = P.qlast[q];
        }
        __syncthreads();
        if (P.fb_mode && !s_flag) continue;   // the fallback answers flagged queries only
        if (!P.fb_mode) {
        // Alg. 5 over the summed level counts of the query's ranges (with shards: over the
        // counts summed across all shards, so every shard finds the same threshold)
        if (tid < Ns) {
            uint64_t v = 0;
            if (P.ghist) {
                v = uint64_t(P.ghist[q * (Ns + 1) + tid + 1]);
            } else {
                for (int r = 0; r < nr; ++r) v += P.unit_ge[(q * nr + r) * 16 + tid + 1];
            }
            s_gs[tid + 1] = uint32_t(v);   // <= n < 2^32
        }
        __syncthreads();
        if (tid == 0) {
            long long gs[TACO_MAX_SUBSPACES + 2];
            gs[0] = P.ghist ? P.ghist[q * (Ns + 1)] : P.n;
            for (int j = 1; j <= Ns; ++j) gs[j] = (long long)s_gs[j];
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
            if (P.dbg_hist)
                for (int j = 0; j <= Ns; ++j) P.dbg_hist[q * (Ns + 1) + j] = gs[j] - gs[j + 1];
            if (P.dbg_last) P.dbg_last[q] = last;
            if (P.dbg_cand) P.dbg_cand[q] = cand;
            if (last < 2) {
                s_flag = 1u;
                P.qflag[q] = 1u;   // candidates below level 2 are not in the lists
            }
            if (s_flag && P.qlast) P.qlast[q] = last;
        }
        __syncthreads();
        if (s_flag) continue;   // answered by the fallback
        }   // !fb_mode
        const int last = s_last;
        // this query's list length (see the cluster kernel): each warp keeps its qp.kk nearest
        const int kq = min(qp.kk, kk);
        // Candidates are buffered (ids in ci); a full buffer is flushed: (A) every warp
        // streams its share of the buffered rows and writes their squared distances to cd,
        // with no dependency between rows, then (B) the block keeps the kq nearest of the
        // buffer and of the list kept so far (Md / Mi, s_cur entries) by a radix select on
        // the distance bits (ties by id) and a bitonic sort.
        if (tid == 0) s_cur = 0u;
        auto flush = [&](int m) {   // block-wide; ends with a barrier
#ifdef TACO_CHECKED
            for (int i = tid; i < m; i += kSrThreads)   // every candidate is a point of D
                if (!TACO_CHECK(P.status, ci[i] < uint32_t(P.n), kStatusSelect)) ci[i] = 0u;
            __syncthreads();
#endif
            constexpr int UG = kGatherRows<RK>;
            for (int b0 = warp * CPW * UG; b0 < m; b0 += kSrWarps * CPW * UG) {
                float acc[UG];
                uint32_t cid[UG];
                bool val[UG];
                gather_rows<G, RK, UG, 2>(rows, row_bytes, nch, qd, ci, b0, m, acc, cid, val, gid, gl, pol_stream);
#pragma unroll
                for (int uu = 0; uu < UG; ++uu)
                    if (val[uu] && gl == 0) cd[b0 + uu * CPW + gid] = acc[uu];
            }
            const int cur = int(s_cur);
            for (int t = tid; t < cur; t += kSrThreads) {   // the list so far joins the buffer
                cd[m + t] = Md[t];
                ci[m + t] = Mi[t];
            }
            __syncthreads();
            keep_nearest(cd, ci, m + cur, kq, kkc, Md, Mi, hist, &s_cur, &s_n, &s_eq, &s_bin, &s_before,
                         s_tmp2, tid, lane, warp, P.status);
        };
        // flush the candidate buffer if a tile of kSrThreads more might not fit (block-wide)
        auto make_room = [&](uint32_t tile = uint32_t(kSrThreads)) {
            if (s_bufn + tile > uint32_t(kSrBuf)) {
                __syncthreads();
                flush(int(s_bufn));
                if (tid == 0) s_bufn = 0u;
                __syncthreads();
            }
        };
        if (P.fb_mode) {
            // codes fallback: SC(id) = #subspaces i with code_i(id) probed (Def. 6), from the
            // cell codes and per-subspace bitmaps of the probed cells; every probed id is
            // taken once (in the first subspace that probed it) if SC >= last; last <= 0
            // takes every point (Alg. 5 reaching level 0)
            // (a shard: the ids of its ranges only, slabs [fb_slab0, fb_slab1))
            const int fb_slab0 = P.shard_r0 * P.slabs_per_cta;
            const int fb_slab1 = min(P.shard_r1 * P.slabs_per_cta, P.n_slabs);
            const int64_t fb_id1 = min(int64_t(fb_slab1) << kSlabLog2, P.n);
            if (last <= 0) {
                for (int64_t t0 = int64_t(fb_slab0) << kSlabLog2; t0 < fb_id1; t0 += kSrThreads) {
                    make_room();
                    const int64_t id = t0 + tid;
                    const bool take = id < fb_id1;
                    const uint32_t at = warp_append_slot(take, &s_bufn, lane);
                    if (take && TACO_CHECK(P.status, at < uint32_t(kSrBuf), kStatusSelect)) ci[at] = uint32_t(id);
                    __syncthreads();
                }
            } else {
                const int Kw = (P.K + 31) / 32;
                if (warp == 0) load_cell_prefix(P, q, s_fpre, lane);
                for (int w = tid; w < Ns * Kw; w += kSrThreads) fbm[w] = 0u;
                __syncthreads();
                const int total_cells = s_fpre[Ns];
                for (int t = tid; t < total_cells; t += kSrThreads) {
                    int i = 0;
                    while (t >= s_fpre[i + 1]) ++i;
                    const int c = P.cells[(q * Ns + i) * P.K + (t - s_fpre[i])];
                    atomicOr(&fbm[i * Kw + (c >> 5)], 1u << (c & 31));
                }
                __syncthreads();
                const int sstride = P.n_slabs + 1;
                for (int cb0 = 0; cb0 < total_cells; cb0 += kSrThreads) {
                    // this batch's cells: their full id runs, prefix of their lengths
                    uint32_t len = 0;
                    const int g = cb0 + tid;
                    if (g < total_cells) {
                        int i = 0;
                        while (g >= s_fpre[i + 1]) ++i;
                        const int c = P.cells[(q * Ns + i) * P.K + (g - s_fpre[i])];
                        const uint32_t* sp = P.split + (size_t(i) * P.K + c) * sstride;
                        fst[tid] = sp[fb_slab0];
                        fsub[tid] = uint32_t(i);
                        len = sp[fb_slab1] - sp[fb_slab0];
                    }
                    uint2 tot;
                    const uint2 ex = block_excl_scan2<kSrWarps>(len, 0u, s_tmp2, tot, lane, warp);
                    fpre[tid] = ex.x;
                    if (tid == 0) fpre[kSrThreads] = tot.x;
                    __syncthreads();
                    const int nb = min(kSrThreads, total_cells - cb0);
                    for (uint32_t e0 = 0; e0 < tot.x; e0 += kSrThreads) {
                        make_room();
                        const uint32_t e = e0 + uint32_t(tid);
                        bool take = false;
                        uint32_t id = 0;
                        if (e < tot.x) {
                            int lo_c = 0, hi_c = nb - 1;   // the cell holding element e
                            while (lo_c < hi_c) {
                                const int mid = (lo_c + hi_c + 1) >> 1;
                                if (fpre[mid] <= e) lo_c = mid;
                                else hi_c = mid - 1;
                            }
                            const uint32_t pos = fst[lo_c] + (e - fpre[lo_c]);
                            id = TACO_CHECK(P.status, pos < uint64_t(P.n_ids), kStatusSelect) ? P.ids[pos] : 0u;
                            if (!TACO_CHECK(P.status, id < uint32_t(P.n), kStatusSelect)) id = 0u;
                            const int own = int(fsub[lo_c]);
                            int sc = 0;
                            bool dup = false;
                            for (int i = 0; i < Ns; ++i) {
                                const uint32_t c = P.codes[size_t(i) * P.n + id];
                                const bool p = (fbm[i * Kw + (c >> 5)] >> (c & 31)) & 1u;
                                sc += p;
                                dup |= p && i < own;
                            }
                            take = !dup && sc >= last;
                        }
                        const uint32_t at = warp_append_slot(take, &s_bufn, lane);
                        if (take && TACO_CHECK(P.status, at < uint32_t(kSrBuf), kStatusSelect)) ci[at] = id;
                        __syncthreads();
                    }
                }
            }
        } else {
        // candidates: the entries tagged last of all the query's ranges (range r's entries are
        // upre[r] .. upre[r + 1] - 1 of one sequence; an id with SC = s >= 2 has one entry per
        // level 2 .. s, so exactly the ids with SC >= last have one tagged last), in tiles of
        // kEntryLoads x kSrThreads entries (each thread's loads of a tile are independent); the
        // buffer is re-ranked and emptied before a tile that would not fit
        // (a shard takes the units of its ranges [shard_r0, shard_r1) only; local index r)
        const int nsr = P.shard_r1 - P.shard_r0;
        uint32_t* upre = fbm;             // [nsr + 1] (the fallback's bitmaps are not in use)
        uint32_t* uoff = upre + nsr + 1;  // [nsr]
        uint32_t nent = 0;
        for (int r0 = 0; r0 < nsr; r0 += kSrThreads) {
            const int r = r0 + tid;
            uint32_t len = 0;
            if (r < nsr) {
                len = P.unit_len[q * nr + P.shard_r0 + r];
                uoff[r] = P.unit_off[q * nr + P.shard_r0 + r];
            }
            uint2 tot;
            const uint2 ex = block_excl_scan2<kSrWarps>(len, 0u, s_tmp2, tot, lane, warp);
            if (r < nsr) upre[r] = nent + ex.x;
            nent += tot.x;
        }
        if (tid == 0) upre[nsr] = nent;
        __syncthreads();
        constexpr uint32_t kTile = uint32_t(kEntryLoads) * kSrThreads;
        for (uint32_t t0 = 0; t0 < nent; t0 += kTile) {
            make_room(kTile);
            uint32_t x[kEntryLoads], rlo[kEntryLoads];
#pragma unroll
            for (int j = 0; j < kEntryLoads; ++j) {
                const uint32_t t = t0 + uint32_t(j * kSrThreads + tid);
                x[j] = 0u;
                rlo[j] = 0xffffffffu;   // no entry
                if (t < nent) {
                    int lo_r = 0, hi_r = nsr - 1;   // the range holding entry t
                    while (lo_r < hi_r) {
                        const int mid = (lo_r + hi_r + 1) >> 1;
                        if (upre[mid] <= t) lo_r = mid;
                        else hi_r = mid - 1;
                    }
                    const size_t ap = size_t(uoff[lo_r]) + (t - upre[lo_r]);
                    x[j] = TACO_CHECK(P.status, ap < P.arena_words, kStatusSelect) ? P.arena[ap] : 0u;
                    rlo[j] = uint32_t(int64_t(P.shard_r0 + lo_r) * P.slabs_per_cta << kSlabLog2);
                }
            }
#pragma unroll
            for (int j = 0; j < kEntryLoads; ++j) {
                const bool take = rlo[j] != 0xffffffffu && int(x[j] >> kLevelShift) == last;
                const uint32_t at = warp_append_slot(take, &s_bufn, lane);
                if (take && TACO_CHECK(P.status, at < uint32_t(kSrBuf), kStatusSelect))
                    ci[at] = rlo[j] + (x[j] & ((1u << kLevelShift) - 1u));
            }
            __syncthreads();
        }
        }
        __syncthreads();
        flush(int(s_bufn));
        // Md / Mi: the query's nearest kq (its k, or its shortlist), sorted by (distance, id),
        // padded with (inf, kNoId) where it has fewer candidates
        if constexpr (RK != kRowF32) {
            // exact FP32 distances of the shortlist (its real entries gathered like the
            // candidate rows, G lanes a row), then rank sort by (distance, id)
            const int nreal = min(int(s_cur), kq);
            const unsigned char* rows32 = reinterpret_cast<const unsigned char*>(P.data);
            for (int b0 = warp * CPW * U; b0 < nreal; b0 += kSrWarps * CPW * U) {
                float acc[U];
                uint32_t cid[U];
                bool val[U];
                gather_distances<G, kRowF32>(rows32, size_t(P.d_pad) * 4, P.d_pad / 4, qv, Mi, b0, nreal, acc, cid,
                                             val, gid, gl, pol_stream);
#pragma unroll
                for (int uu = 0; uu < U; ++uu)
                    if (val[uu] && gl == 0) {
                        Xd[b0 + uu * CPW + gid] = acc[uu];
                        Xi[b0 + uu * CPW + gid] = cid[uu];
                    }
            }
            for (int e = nreal + tid; e < kq; e += kSrThreads) {
                Xd[e] = __int_as_float(0x7f800000);
                Xi[e] = kNoId;
            }
            __syncthreads();
            for (int e = tid; e < kq; e += kSrThreads) {
                const float x = Xd[e];
                const uint32_t xid = Xi[e];
                int rank = 0;
                for (int f = 0; f < kq; ++f)
                    rank += lt_pair(Xd[f], Xi[f], x, xid) || (Xd[f] == x && Xi[f] == xid && f < e);
                Md[rank] = x;
                Mi[rank] = xid;
            }
            __syncthreads();
        }
        for (int t = tid; t < P.k_stride; t += kSrThreads) {
            const bool ok = t < qp.k && t < kq && Mi[t] != kNoId;
            P.out_ids[q * P.k_stride + t] = ok ? int64_t(Mi[t]) : int64_t(-1);
            P.out_dists[q * P.k_stride + t] = ok ? sqrtf(Md[t]) : __int_as_float(0x7f800000);
        }
    }
}

template <int G, int RK>
cudaError_t launch_select_rerank_t(const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st) {
    auto kern = select_rerank_kernel<G, RK>;
    // two cached shapes per instance: the two-pass form and the codes fallback
    static thread_local size_t cached_smem_v[2] = {0, 0};
    static thread_local int cached_blocks_v[2] = {0, 0};
    const int slot = P.fb_mode ? 1 : 0;
    size_t& cached_smem = cached_smem_v[slot];
    int& cached_blocks = cached_blocks_v[slot];
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return g_launch_step = "an earlier unchecked call", e;
    if (cached_smem != smem) {
        e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
        if (e != cudaSuccess) return g_launch_step = "cudaFuncSetAttribute", e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSrThreads, smem);
        if (e != cudaSuccess) return g_launch_step = "cudaOccupancyMaxActiveBlocksPerMultiprocessor", e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (per_sm * sms < 1) return g_launch_step = "occupancy (no block fits)", cudaErrorInvalidConfiguration;
        cached_blocks = per_sm * sms;
        cached_smem = smem;
    }
    const int64_t blocks = nq < cached_blocks ? nq : cached_blocks;
    kern<<<unsigned(blocks), kSrThreads, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) g_launch_step = "launch";
    return e;
}


}  // namespace taco

// Fused collision counting (Alg. 6 step 7, Def. 6), query-aware candidate selection
// (Alg. 5) and exact re-rank (Alg. 6 step 9) for one query per thread-block cluster.
//
// Layout: the n point ids are split into slabs of 2^15. CTA r of a query's cluster owns a
// contiguous range of slabs and holds one 4-bit SC counter per owned id in shared memory
// (N_s <= 15). Cell id lists are ascending, so the ids of a probed cell that fall in the
// CTA's range form one contiguous run; a per-cell table of slab boundaries gives the run.
//   1. count:  every warp takes probed cells; lanes read the run's ids (coalesced) and add
//              1 to the id's nibble with a shared-memory atomic.
//   2. levels: each CTA counts its ids with SC >= j for every j (SWAR over nibbles); the
//              cluster sums these through distributed shared memory, giving collision_num
//              over all n points, and every CTA evaluates Alg. 5 to the same threshold.
//   3. re-rank: warps scan their counter words, queue the ids whose SC reaches the
//              threshold, gather the rows (G lanes per row, 16-byte loads) and keep a
//              warp-wide sorted top list in registers (insertion by ballot + shuffle).
//   4. merge:  warp lists -> CTA list (warp 0, k-way merge) -> cluster list in CTA 0 via
//              distributed shared memory. With BF16 rows the merged list is a shortlist
//              that CTA 0 re-ranks with FP32 rows before writing the top k.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "taco_internal.h"

namespace taco {
namespace cg = cooperative_groups;

constexpr int kRrThreads = 512;
constexpr int kRrWarps = kRrThreads / 32;
constexpr int kQueueCap = 256;   // one scan step: 32 words x 8 ids
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoId = 0xffffffffu;

struct RerankParams {
    const float* queries;   // [nq][d]
    const float* data;      // [n][d_pad]
    const __nv_bfloat16* data_bf16;  // [n][d_pad]
    const uint32_t* ids;    // [Ns][n]
    const uint32_t* split;  // [Ns][K][n_slabs+1]
    const uint16_t* cells;  // [nq][Ns][K]
    const int32_t* ncells;  // [nq][Ns]
    const QueryParamsDev* params;
    QueryParamsDev defaults;
    int64_t n;
    int d, d_pad, Ns, K, n_slabs, slabs_per_cta;
    int counter_words;      // slabs_per_cta * kSlabWords
    int kk;                 // list length (<= 32*R)
    int kkc;                // power of two >= kk
    size_t region_a;        // bytes of the counter / merge region
    int64_t* out_ids;
    float* out_dists;
    int k_stride;
    uint8_t* dbg_sc;
    int64_t* dbg_hist;
    int32_t* dbg_last;
    int64_t* dbg_cand;
};

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

// k-way merge of `nl` sorted lists (list j at (ld + j*stride, li + j*stride), each of
// length kk) into the first kk entries of (od, oi). Called by one full warp; nl <= 32.
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

// Same merge, reading list j from CTA j of the cluster (distributed shared memory).
__device__ __forceinline__ void cluster_merge(cg::cluster_group& cluster, float* ld,
                                              uint32_t* li, int nl, int kk, float* od,
                                              uint32_t* oi, int lane) {
    const float* rd = ld;
    const uint32_t* ri = li;
    if (lane < nl) {
        rd = cluster.map_shared_rank(ld, lane);
        ri = cluster.map_shared_rank(li, lane);
    }
    int p = 0;
    for (int o = 0; o < kk; ++o) {
        float v = __int_as_float(0x7f800000);
        uint32_t vi = kNoId;
        if (lane < nl && p < kk) {
            v = rd[p];
            vi = ri[p];
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

// Row chunk = 16 bytes: 4 floats or 8 bf16.
template <bool BF16>
struct RowChunk {
    static constexpr int kElems = BF16 ? 8 : 4;
};

__device__ __forceinline__ uint4 ldg_nc_u4(const void* p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

template <bool BF16>
__device__ __forceinline__ float chunk_dist(uint4 raw, const float* qv, int f, float acc) {
    if constexpr (!BF16) {
        const float4 o = make_float4(__uint_as_float(raw.x), __uint_as_float(raw.y),
                                     __uint_as_float(raw.z), __uint_as_float(raw.w));
        const float4 q = reinterpret_cast<const float4*>(qv)[f];
        return sq4(o, q, acc);
    } else {
        const float4 q0 = reinterpret_cast<const float4*>(qv)[2 * f];
        const float4 q1 = reinterpret_cast<const float4*>(qv)[2 * f + 1];
        const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
        const float2 a0 = __bfloat1622float2(b[0]);
        const float2 a1 = __bfloat1622float2(b[1]);
        const float2 a2 = __bfloat1622float2(b[2]);
        const float2 a3 = __bfloat1622float2(b[3]);
        acc = sq4(make_float4(a0.x, a0.y, a1.x, a1.y), q0, acc);
        return sq4(make_float4(a2.x, a2.y, a3.x, a3.y), q1, acc);
    }
}

// G lanes per candidate, R registers per lane of top list, BF16 rows or FP32 rows.
template <int G, int R, bool BF16>
__global__ void __launch_bounds__(kRrThreads, (R <= 4 ? 2 : 1))
count_select_rerank_kernel(const RerankParams P) {
    constexpr int CPW = 32 / G;   // candidates per warp pass
    constexpr int U = 2;          // passes in flight
    constexpr int CH = 4;         // 16-byte chunks per lane per row pass
    cg::cluster_group cluster = cg::this_cluster();
    const int cta = int(cluster.block_rank());
    const int ncta = int(cluster.num_blocks());
    const int64_t q = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);
    float* qv = reinterpret_cast<float*>(smem + P.region_a);
    uint32_t* queue = reinterpret_cast<uint32_t*>(qv + P.d_pad);
    uint32_t* ge = queue + kRrWarps * kQueueCap;   // [16]
    __shared__ int s_pre[TACO_MAX_SUBSPACES + 1];
    __shared__ int s_last;

    const QueryParamsDev qp = P.params ? P.params[q] : P.defaults;
    const int Ns = P.Ns, K = P.K;
    const int slab_lo = cta * P.slabs_per_cta;
    const int slab_hi = min(slab_lo + P.slabs_per_cta, P.n_slabs);
    const int64_t lo = int64_t(slab_lo) << kSlabLog2;
    const int64_t hi = min(int64_t(slab_hi) << kSlabLog2, P.n);
    const int words = hi > lo ? int((hi - lo + 7) >> 3) : 0;

    // ---- 0. clear counters, stage the query --------------------------------------------
    for (int w = tid; w < P.counter_words; w += kRrThreads) cnt[w] = 0u;
    for (int j = tid; j < P.d_pad; j += kRrThreads)
        qv[j] = j < P.d ? P.queries[q * P.d + j] : 0.f;
    if (tid < 16) ge[tid] = 0u;
    if (tid == 0) {
        int acc = 0;
        s_pre[0] = 0;
        for (int i = 0; i < Ns; ++i) {
            acc += P.ncells[q * Ns + i];
            s_pre[i + 1] = acc;
        }
    }
    __syncthreads();

    // ---- 1. count collisions of the probed cells' ids in this CTA's range ---------------
    const int total_cells = s_pre[Ns];
    const int sstride = P.n_slabs + 1;
    for (int t = warp; t < total_cells; t += kRrWarps) {
        int i = 0;
        while (t >= s_pre[i + 1]) ++i;
        const int cell = P.cells[(q * Ns + i) * K + (t - s_pre[i])];
        const uint32_t* sp = P.split + (size_t(i) * K + cell) * sstride;
        const uint32_t beg = __ldg(sp + slab_lo), end = __ldg(sp + slab_hi);
        const uint32_t* idp = P.ids + size_t(i) * P.n;
        for (uint32_t p = beg + lane; p < end; p += 32) {
            const uint32_t id = __ldg(idp + p) - uint32_t(lo);
            atomicAdd(&cnt[id >> 3], 1u << ((id & 7u) << 2));
        }
    }
    __syncthreads();

    // ---- 2. SC levels: ge[j] = #ids of this CTA with SC >= j ---------------------------
    {
        uint32_t gel[TACO_MAX_SUBSPACES];
#pragma unroll
        for (int j = 0; j < TACO_MAX_SUBSPACES; ++j) gel[j] = 0;
        for (int w = tid; w < words; w += kRrThreads) {
            const uint32_t x = cnt[w];
            if (x == 0u) continue;
            const uint32_t ev = x & 0x0f0f0f0fu, od = (x >> 4) & 0x0f0f0f0fu;
#pragma unroll
            for (int j = 1; j <= TACO_MAX_SUBSPACES; ++j) {
                if (j <= Ns) {
                    const uint32_t add = (0x80u - uint32_t(j)) * 0x01010101u;
                    gel[j - 1] += __popc((ev + add) & 0x80808080u) + __popc((od + add) & 0x80808080u);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TACO_MAX_SUBSPACES; ++j) {
            if (j < Ns) {
                uint32_t v = gel[j];
#pragma unroll
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
                if (lane == 0 && v) atomicAdd(&ge[j + 1], v);
            }
        }
    }
    cluster.sync();

    // ---- 3. Alg. 5 on the cluster-wide collision_num (same result in every CTA) --------
    if (tid == 0) {
        long long gs[TACO_MAX_SUBSPACES + 2];
        for (int j = 0; j <= Ns + 1; ++j) gs[j] = 0;
        for (int r = 0; r < ncta; ++r) {
            const uint32_t* rg = cluster.map_shared_rank(ge, r);
            for (int j = 1; j <= Ns; ++j) gs[j] += rg[j];
        }
        gs[0] = P.n;
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

    // ---- 4. gather the candidates of this CTA and keep the warp's best kk ---------------
    WarpTop<R> top;
    top.init();
    const int kk = P.kk;
    float kth_d = __int_as_float(0x7f800000);
    uint32_t kth_i = kNoId;
    uint32_t* wq = queue + warp * kQueueCap;
    const int gid = lane / G, gl = lane % G;
    const int nch = P.d_pad / RowChunk<BF16>::kElems;
    const size_t row_bytes = size_t(P.d_pad) * (BF16 ? 2 : 4);
    const unsigned char* base = BF16 ? reinterpret_cast<const unsigned char*>(P.data_bf16)
                                     : reinterpret_cast<const unsigned char*>(P.data);
    for (int wb = warp * 32; wb < words; wb += kRrWarps * 32) {
        const int w = wb + lane;
        uint32_t m8 = 0;
        const int64_t id0 = lo + (int64_t(w) << 3);
        if (w < words) {
            const uint32_t x = cnt[w];
            if (last <= 0) {
                m8 = 0xffu;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (int((x >> (4 * j)) & 15u) >= last) m8 |= 1u << j;
            }
            const int64_t rem = hi - id0;
            if (rem < 8) m8 &= (1u << rem) - 1u;
            if (P.dbg_sc) {
                for (int j = 0; j < 8 && j < rem; ++j)
                    P.dbg_sc[q * P.n + id0 + j] = uint8_t((x >> (4 * j)) & 15u);
            }
        }
        const int c = __popc(m8);
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += v;
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        int at = incl - c;
        while (m8) {
            const int b = __ffs(m8) - 1;
            m8 &= m8 - 1;
            wq[at++] = uint32_t(id0 + b);
        }
        __syncwarp();
        for (int b0 = 0; b0 < tot; b0 += CPW * U) {
            float acc[U];
            uint32_t cid[U];
            bool val[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = b0 + u * CPW + gid;
                val[u] = idx < tot;
                cid[u] = val[u] ? wq[idx] : 0u;
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
                                         ? ldg_nc_u4(base + size_t(cid[u]) * row_bytes + size_t(f) * 16)
                                         : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int ch = 0; ch < CH; ++ch) {
                        const int f = f0 + ch * G + gl;
                        if (f < nch) acc[u] = chunk_dist<BF16>(raw[u][ch], qv, f, acc[u]);
                    }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int off = G / 2; off; off >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], off);
            }
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
                        top.insert(x, xi, kk, lane);
                        top.kth(kk, kth_d, kth_i);
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();   // counters are dead from here on: region A becomes the merge area

    // ---- 5. merge: warps -> CTA -> cluster --------------------------------------------
    const int kkc = P.kkc;
    float* Ld = reinterpret_cast<float*>(smem);
    uint32_t* Li = reinterpret_cast<uint32_t*>(Ld + kRrWarps * kkc);
    float* CLd = reinterpret_cast<float*>(Li + kRrWarps * kkc);
    uint32_t* CLi = reinterpret_cast<uint32_t*>(CLd + kkc);
    float* GLd = reinterpret_cast<float*>(CLi + kkc);
    uint32_t* GLi = reinterpret_cast<uint32_t*>(GLd + kkc);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < kk) {
            Ld[warp * kkc + e] = top.d[r];
            Li[warp * kkc + e] = top.i[r];
        }
    }
    __syncthreads();
    if (warp == 0) warp_merge(Ld, Li, kkc, kRrWarps, kk, CLd, CLi, lane);
    cluster.sync();
    if (cta == 0) {
        if (warp == 0) cluster_merge(cluster, CLd, CLi, ncta, kk, GLd, GLi, lane);
        __syncthreads();
        if constexpr (BF16) {
            // exact FP32 re-rank of the shortlist, then sort it by (dist, id)
            const int nf4 = P.d_pad / 4;
            for (int e = warp; e < kkc; e += kRrWarps) {
                const uint32_t id = e < kk ? GLi[e] : kNoId;
                float acc = 0.f;
                if (id != kNoId) {
                    const float4* row = reinterpret_cast<const float4*>(P.data + size_t(id) * P.d_pad);
                    const float4* q4 = reinterpret_cast<const float4*>(qv);
                    for (int f = lane; f < nf4; f += 32) acc = sq4(__ldg(row + f), q4[f], acc);
                }
#pragma unroll
                for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
                if (lane == 0) {
                    GLd[e] = id != kNoId ? acc : __int_as_float(0x7f800000);
                    GLi[e] = id;
                }
            }
            __syncthreads();
            for (int k2 = 2; k2 <= kkc; k2 <<= 1) {
                for (int j = k2 >> 1; j > 0; j >>= 1) {
                    for (int t = tid; t < kkc; t += kRrThreads) {
                        const int o = t ^ j;
                        if (o > t) {
                            const float a = GLd[t], b = GLd[o];
                            const uint32_t ia = GLi[t], ib = GLi[o];
                            const bool asc = (t & k2) == 0;
                            if (lt_pair(b, ib, a, ia) == asc) {
                                GLd[t] = b;
                                GLd[o] = a;
                                GLi[t] = ib;
                                GLi[o] = ia;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        for (int t = tid; t < P.k_stride; t += kRrThreads) {
            const bool ok = t < qp.k && t < kk && GLi[t] != kNoId;
            P.out_ids[q * P.k_stride + t] = ok ? int64_t(GLi[t]) : int64_t(-1);
            P.out_dists[q * P.k_stride + t] = ok ? sqrtf(GLd[t]) : __int_as_float(0x7f800000);
        }
    }
    cluster.sync();   // keep every CTA's shared memory alive until CTA 0 has read it
}

template <int G, int R, bool BF16>
cudaError_t launch_rerank_t(const RerankParams& P, int cluster, int64_t nq, size_t smem,
                            cudaStream_t st) {
    auto kern = count_select_rerank_kernel<G, R, BF16>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cluster), unsigned(nq), 1);
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
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
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

}  // namespace taco

// Query path orchestration and the cell-probe kernel (Alg. 6 steps 3-6 with Alg. 4).
//
// Alg. 4 pops IMI cells in ascending order of d1[r] + d2[c] and stops as soon as the
// retrieved sizes reach the budget; the popped set is therefore the shortest prefix of
// the key-sorted cells whose sizes sum to >= B (the paper notes that its heap and the
// linear activation array of SuCo return the same cells). The GPU computes that prefix
// directly: one CTA per (query, subspace) builds the K keys (FP32 sum bits << 32 | cell id,
// a total order that breaks equal sums by r then c), finds the bucket of a size-weighted
// histogram over the key range where the running size crosses B, sorts only that bucket,
// and walks it to the exact threshold key T. Cells with key <= T are the probed set.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include <algorithm>
#include <cstdint>

#include "taco_internal.h"
#include "taco_count.cuh"
#include "taco_rerank.cuh"
#include "taco_select.cuh"

namespace taco {

constexpr int kSelThreads = 256;
constexpr int kSelBins = 2048;
constexpr int kSelBinsPerThread = kSelBins / kSelThreads;

__device__ __forceinline__ unsigned long long cell_key(const float* d1, const float* d2, int sk,
                                                       int cell) {
    const int r = cell / sk, c = cell - r * sk;
    const float sum = d1[r] + d2[c];
    return (static_cast<unsigned long long>(__float_as_uint(sum)) << 32) | unsigned(cell);
}

__global__ void __launch_bounds__(kSelThreads)
probe_cells_kernel(const float* __restrict__ qt, int Dp, const float* __restrict__ cent,
                   const float* __restrict__ hd,
                   int Ns, int s, int h1, int sk, const uint32_t* __restrict__ sizes, int64_t n,
                   QueryParamsDev defaults, const QueryParamsDev* __restrict__ params,
                   int list_cap, uint16_t* __restrict__ cells_out,
                   int32_t* __restrict__ ncells_out, int64_t* __restrict__ retrieved_out,
                   int redo_only) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int i = blockIdx.x;
    const int64_t q = blockIdx.y;
    if (redo_only && ncells_out[size_t(q) * Ns + i] >= 0) return;   // the walk settled it
    const int K = sk * sk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long* list = reinterpret_cast<unsigned long long*>(sm);  // list_cap
    uint32_t* hist = reinterpret_cast<uint32_t*>(list + list_cap);         // kSelBins
    float* d1 = reinterpret_cast<float*>(hist + kSelBins);                  // sk
    float* d2 = d1 + sk;                                                    // sk
    __shared__ uint32_t s_min, s_max;
    __shared__ int s_bucket, s_m, s_cnt;
    __shared__ unsigned long long s_pre, s_T, s_ret;
    __shared__ uint32_t s_wsum[kSelThreads / 32];

    const QueryParamsDev qp = params ? params[q] : defaults;
    const int64_t budget = qp.budget;

    // Alg. 6 steps 4-5: squared distances of the two half-queries to their centroids
    const float* qi = qt + q * Dp + size_t(i) * s;
    for (int t = tid; t < 2 * sk; t += kSelThreads) {
        const int h = t >= sk;
        const int c = h ? t - sk : t;
        const int off = h ? h1 : 0, len = h ? s - h1 : h1;
        const float* cc = cent + (size_t(i) * sk + c) * s + off;
        float acc = 0.f;
        if (hd) {   // from the separate centroid block
            acc = hd[(size_t(q) * Ns + i) * 2 * sk + t];
        } else {
            for (int j = 0; j < len; ++j) {
                const float df = qi[off + j] - cc[j];
                acc = fmaf(df, df, acc);
            }
        }
        (h ? d2 : d1)[c] = acc;
    }
    for (int t = tid; t < kSelBins; t += kSelThreads) hist[t] = 0u;
    if (tid == 0) {
        s_min = 0xffffffffu;
        s_max = 0u;
        s_m = 0;
        s_cnt = 0;
        s_ret = 0ull;
        s_T = ~0ull;
        s_bucket = -1;
        s_pre = 0ull;
    }
    __syncthreads();
    const uint32_t* sz = sizes + size_t(i) * K;

    if (budget <= n) {
        // key range (the sums are >= +0, so their bit patterns order like the values)
        uint32_t mn = 0xffffffffu, mx = 0u;
        for (int cell = tid; cell < K; cell += kSelThreads) {
            const uint32_t b = uint32_t(cell_key(d1, d2, sk, cell) >> 32);
            mn = min(mn, b);
            mx = max(mx, b);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
        if (lane == 0) {
            atomicMin(&s_min, mn);
            atomicMax(&s_max, mx);
        }
        __syncthreads();
        const uint32_t minb = s_min, range = s_max - s_min;
        const int bits = range ? 32 - __clz(range) : 0;
        const int shift = bits > 11 ? bits - 11 : 0;
        // size-weighted histogram of the high key bits
        for (int cell = tid; cell < K; cell += kSelThreads) {
            const uint32_t w = sz[cell];
            if (w) {
                const uint32_t b = uint32_t(cell_key(d1, d2, sk, cell) >> 32);
                atomicAdd(&hist[(b - minb) >> shift], w);
            }
        }
        __syncthreads();
        // block scan over the bins; find the bin where the running size first reaches B
        unsigned long long loc = 0;
#pragma unroll
        for (int j = 0; j < kSelBinsPerThread; ++j) loc += hist[tid * kSelBinsPerThread + j];
        unsigned long long incl = loc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) s_wsum[warp] = uint32_t(incl);
        __syncthreads();
        unsigned long long wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        unsigned long long pre = wpre + incl - loc;
        for (int j = 0; j < kSelBinsPerThread; ++j) {
            const uint32_t hb = hist[tid * kSelBinsPerThread + j];
            if (pre < (unsigned long long)budget && (unsigned long long)budget <= pre + hb) {
                s_bucket = tid * kSelBinsPerThread + j;
                s_pre = pre;
            }
            pre += hb;
        }
        __syncthreads();
        // cells of that bin (with any size: empty cells keep their place in the order)
        const int bucket = s_bucket;
        for (int cell = tid; cell < K; cell += kSelThreads) {
            const unsigned long long key = cell_key(d1, d2, sk, cell);
            if (int((uint32_t(key >> 32) - minb) >> shift) == bucket) list[atomicAdd(&s_m, 1)] = key;
        }
        __syncthreads();
        const int m = s_m;
        int p2 = 1;
        while (p2 < m) p2 <<= 1;
        for (int t = m + tid; t < p2; t += kSelThreads) list[t] = ~0ull;
        __syncthreads();
        for (int k2 = 2; k2 <= p2; k2 <<= 1) {
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < p2; t += kSelThreads) {
                    const int o = t ^ j;
                    if (o > t) {
                        const unsigned long long a = list[t], b = list[o];
                        if ((a > b) == ((t & k2) == 0)) {
                            list[t] = b;
                            list[o] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // walk the sorted bin until the running size reaches B
        if (warp == 0) {
            unsigned long long cum = s_pre;
            for (int b0 = 0; b0 < m; b0 += 32) {
                const int idx = b0 + lane;
                const unsigned long long key = idx < m ? list[idx] : ~0ull;
                unsigned long long w = idx < m ? sz[uint32_t(key)] : 0ull;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned long long v = __shfl_up_sync(0xffffffffu, w, off);
                    if (lane >= off) w += v;
                }
                const bool hit = idx < m && cum + w >= (unsigned long long)budget;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (bal) {
                    if (lane == __ffs(bal) - 1) s_T = key;
                    break;
                }
                cum += __shfl_sync(0xffffffffu, w, 31);
            }
        }
        __syncthreads();
    }
    // the probed set: every cell whose key is <= T
    const unsigned long long T = s_T;
    const size_t qi_off = (size_t(q) * Ns + i);
    unsigned long long ret = 0;
    for (int base = 0; base < K; base += kSelThreads) {
        const int cell = base + tid;
        bool take = false;
        if (cell < K) take = cell_key(d1, d2, sk, cell) <= T;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        int wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&s_cnt, __popc(bal));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (take) {
            cells_out[qi_off * K + wbase + __popc(bal & ((1u << lane) - 1u))] = uint16_t(cell);
            ret += sz[cell];
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) ret += __shfl_xor_sync(0xffffffffu, ret, off);
    if (lane == 0 && ret) atomicAdd(&s_ret, ret);
    __syncthreads();
    if (tid == 0) {
        ncells_out[qi_off] = s_cnt;
        retrieved_out[qi_off] = (long long)s_ret;
    }
}

// Alg. 4 by merging sorted rows, one warp per (query, subspace). The second-half distances
// d2 are sorted once; lane l owns the rows r = l + 32 e (first-half centroids), each with a
// pointer into the sorted d2, so a row's next cell is its smallest unvisited key. A pop takes
// the minimum over the row heads of (FP32 key bits, cell) (two warp min-reductions), which
// visits the cells in the order of probe_cells_kernel's keys as long as no two cells share
// a key; sizes are checked every kWalkBatch pops and the prefix stops at the cell where the
// running size first reaches B. If another cell has exactly the key of that cell (its place
// is then decided by the cell index among equal keys), or more than kWalkMaxPops pops are
// needed, ncells is set to -1 and the histogram kernel redoes this (query, subspace).
constexpr int kWalkThreads = 256;
constexpr int kWalkBatch = 16;      // pops between size checks (<= 32)
constexpr int kWalkMaxPops = 1024;

template <int E>   // rows per lane: sqrtK <= 32 E, E in {1, 2, 4}
__global__ void __launch_bounds__(kWalkThreads)
probe_cells_walk_kernel(const float* __restrict__ qt, int Dp, const float* __restrict__ cent,
                   const float* __restrict__ hd,
                        int Ns, int s, int h1, int sk, const uint32_t* __restrict__ sizes,
                        int64_t n, QueryParamsDev defaults, const QueryParamsDev* __restrict__ params,
                        int64_t ntasks, uint16_t* __restrict__ cells_out,
                        int32_t* __restrict__ ncells_out, int64_t* __restrict__ retrieved_out) {
    constexpr int W = kWalkThreads / 32;
    constexpr int N = 32 * E;
    __shared__ uint32_t s_bv[W][N];   // sorted d2 (FP32 bits)
    __shared__ uint32_t s_bc[W][N];   // their second-half centroid indices
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = sk * sk;
    for (int64_t task = int64_t(blockIdx.x) * W + warp; task < ntasks; task += int64_t(gridDim.x) * W) {
        const int64_t q = task / Ns;
        const int i = int(task - q * Ns);
        const QueryParamsDev qp = params ? params[q] : defaults;
        const int64_t budget = qp.budget;
        uint16_t* out = cells_out + size_t(task) * K;
        if (budget > n) {   // every cell
            for (int c = lane; c < K; c += 32) out[c] = uint16_t(c);
            if (lane == 0) {
                ncells_out[task] = K;
                retrieved_out[task] = n;
            }
            continue;
        }
        // Alg. 6 steps 4-5: squared distances of the two half-queries to their centroids
        const float* qi = qt + q * Dp + size_t(i) * s;
        float a[E];
        uint32_t bk[E], bc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int t = lane + 32 * e;
            float d1 = __int_as_float(0x7f800000), d2 = d1;
            if (t < sk && hd) {   // from the separate centroid block
                d1 = hd[(size_t(q) * Ns + i) * 2 * sk + t];
                d2 = hd[(size_t(q) * Ns + i) * 2 * sk + sk + t];
            } else if (t < sk) {
                const float* cc = cent + (size_t(i) * sk + t) * s;
                float acc = 0.f;
                for (int j = 0; j < h1; ++j) {
                    const float df = qi[j] - cc[j];
                    acc = fmaf(df, df, acc);
                }
                d1 = acc;
                acc = 0.f;
                for (int j = 0; j < s - h1; ++j) {
                    const float df = qi[h1 + j] - cc[h1 + j];
                    acc = fmaf(df, df, acc);
                }
                d2 = acc;
            }
            a[e] = d1;
            bk[e] = t < sk ? __float_as_uint(d2) : 0xffffffffu;
            bc[e] = uint32_t(t);
        }
        // bitonic sort of (bk, bc) ascending over the N slots, slot = 32 e + lane
#pragma unroll
        for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                if (j >= 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int f = e ^ (j >> 5);
                        if (f > e) {
                            const bool up = ((32 * e + lane) & k) == 0;
                            const bool gt = bk[e] > bk[f] || (bk[e] == bk[f] && bc[e] > bc[f]);
                            if (gt == up) {
                                const uint32_t tk = bk[e], tc = bc[e];
                                bk[e] = bk[f];
                                bc[e] = bc[f];
                                bk[f] = tk;
                                bc[f] = tc;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const uint32_t ok = __shfl_xor_sync(kFull, bk[e], j);
                        const uint32_t oc = __shfl_xor_sync(kFull, bc[e], j);
                        const bool up = ((32 * e + lane) & k) == 0;
                        const bool lower = (lane & j) == 0;
                        const bool own_lt = bk[e] < ok || (bk[e] == ok && bc[e] < oc);
                        const bool keep_own = (lower == up) ? own_lt : !own_lt;
                        if (!keep_own) {
                            bk[e] = ok;
                            bc[e] = oc;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            s_bv[warp][32 * e + lane] = bk[e];
            s_bc[warp][32 * e + lane] = bc[e];
        }
        __syncwarp();
        // row heads (key bits, cell); exhausted or absent rows hold 0xffffffff
        uint32_t hs[E], hc[E];
        int jp[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int r = lane + 32 * e;
            jp[e] = 0;
            hs[e] = 0xffffffffu;
            hc[e] = 0xffffffffu;
            if (r < sk) {
                hs[e] = __float_as_uint(a[e] + __uint_as_float(s_bv[warp][0]));
                hc[e] = uint32_t(r * sk) + s_bc[warp][0];
            }
        }
        uint32_t ls = hs[0], lc = hc[0];
#pragma unroll
        for (int e = 1; e < E; ++e)
            if (hs[e] < ls || (hs[e] == ls && hc[e] < lc)) { ls = hs[e]; lc = hc[e]; }
        const uint32_t* sz = sizes + size_t(i) * K;
        unsigned long long cum = 0;
        uint32_t prev_last = 0, rec_s = 0, rec_c = 0;
        bool has_prev = false;
        int nout = 0, pops = 0, status = 0;   // status: 1 settled, 2 redo
        while (status == 0) {
            int np = 0;
            for (; np < kWalkBatch; ++np) {
                const uint32_t ms = __reduce_min_sync(kFull, ls);
                if (ms == 0xffffffffu) break;   // every cell visited
                const uint32_t mc = __reduce_min_sync(kFull, ls == ms ? lc : 0xffffffffu);
                if (lane == np) {
                    rec_s = ms;
                    rec_c = mc;
                }
                if (ls == ms && lc == mc) {   // this lane's row advances
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (hc[e] == mc) {
                            const int jn = ++jp[e];
                            if (jn < sk) {
                                hs[e] = __float_as_uint(a[e] + __uint_as_float(s_bv[warp][jn]));
                                hc[e] = uint32_t((lane + 32 * e) * sk) + s_bc[warp][jn];
                            } else {
                                hs[e] = 0xffffffffu;
                                hc[e] = 0xffffffffu;
                            }
                        }
                    }
                    ls = hs[0];
                    lc = hc[0];
#pragma unroll
                    for (int e = 1; e < E; ++e)
                        if (hs[e] < ls || (hs[e] == ls && hc[e] < lc)) { ls = hs[e]; lc = hc[e]; }
                }
            }
            pops += np;
            // running size over this batch's pops
            unsigned long long w = lane < np ? sz[rec_c] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long v = __shfl_up_sync(kFull, w, off);
                if (lane >= off) w += v;
            }
            const unsigned hit = __ballot_sync(kFull, lane < np && cum + w >= (unsigned long long)budget);
            if (hit) {
                const int x = __ffs(hit) - 1;
                const uint32_t S = __shfl_sync(kFull, rec_s, x);
                const bool tie = __ballot_sync(kFull, lane < np && lane != x && rec_s == S) != 0u ||
                                 (has_prev && prev_last == S) ||
                                 __reduce_min_sync(kFull, ls) == S;
                if (tie) {
                    status = 2;
                } else {
                    if (lane <= x) out[nout + lane] = uint16_t(rec_c);
                    nout += x + 1;
                    cum += __shfl_sync(kFull, w, x);
                    status = 1;
                }
                break;
            }
            if (np > 0) {
                if (lane < np) out[nout + lane] = uint16_t(rec_c);
                nout += np;
                cum += __shfl_sync(kFull, w, np - 1);
                prev_last = __shfl_sync(kFull, rec_s, np - 1);
                has_prev = true;
            }
            if (np < kWalkBatch) status = 1;                 // every cell visited
            else if (pops >= kWalkMaxPops) status = 2;
        }
        if (lane == 0) {
            ncells_out[task] = status == 2 ? -1 : nout;
            retrieved_out[task] = (long long)cum;
        }
        __syncwarp();   // s_bv / s_bc are rewritten by the next task
    }
}

// Same selection as probe_cells_kernel for K <= 256 * CPT cells, keeping each thread's CPT
// keys and sizes in registers: the key range comes from the extremes of d1 and d2 (FP32
// addition is monotone, so min1 + min2 and max1 + max2 bound every key), and the histogram,
// bucket collection and output passes reuse the registers instead of recomputing keys.
template <int CPT>
__global__ void __launch_bounds__(kSelThreads)
probe_cells_reg_kernel(const float* __restrict__ qt, int Dp, const float* __restrict__ cent,
                   const float* __restrict__ hd,
                       int Ns, int s, int h1, int sk, const uint32_t* __restrict__ sizes,
                       int64_t n, QueryParamsDev defaults, const QueryParamsDev* __restrict__ params,
                       int list_cap, uint16_t* __restrict__ cells_out,
                       int32_t* __restrict__ ncells_out, int64_t* __restrict__ retrieved_out,
                       int redo_only) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int i = blockIdx.x;
    const int64_t q = blockIdx.y;
    if (redo_only && ncells_out[size_t(q) * Ns + i] >= 0) return;   // the walk settled it
    const int K = sk * sk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long* list = reinterpret_cast<unsigned long long*>(sm);  // list_cap
    uint32_t* hist = reinterpret_cast<uint32_t*>(list + list_cap);         // kSelBins
    float* d1 = reinterpret_cast<float*>(hist + kSelBins);                  // sk
    float* d2 = d1 + sk;                                                    // sk
    __shared__ uint32_t s_min, s_max;
    __shared__ int s_bucket, s_m, s_cnt;
    __shared__ unsigned long long s_pre, s_T, s_ret;
    __shared__ uint32_t s_wsum[kSelThreads / 32];

    const QueryParamsDev qp = params ? params[q] : defaults;
    const int64_t budget = qp.budget;
    const uint32_t* sz = sizes + size_t(i) * K;
    uint32_t kw[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {   // sizes first: their loads overlap the distance math
        const int cell = tid + kSelThreads * u;
        kw[u] = cell < K ? __ldg(sz + cell) : 0u;
    }
    // Alg. 6 steps 4-5: squared distances of the two half-queries to their centroids
    const float* qi = qt + q * Dp + size_t(i) * s;
    for (int t = tid; t < 2 * sk; t += kSelThreads) {
        const int h = t >= sk;
        const int c = h ? t - sk : t;
        const int off = h ? h1 : 0, len = h ? s - h1 : h1;
        const float* cc = cent + (size_t(i) * sk + c) * s + off;
        float acc = 0.f;
        if (hd) {   // from the separate centroid block
            acc = hd[(size_t(q) * Ns + i) * 2 * sk + t];
        } else {
            for (int j = 0; j < len; ++j) {
                const float df = qi[off + j] - cc[j];
                acc = fmaf(df, df, acc);
            }
        }
        (h ? d2 : d1)[c] = acc;
    }
    for (int t = tid; t < kSelBins; t += kSelThreads) hist[t] = 0u;
    if (tid == 0) {
        s_m = 0;
        s_cnt = 0;
        s_ret = 0ull;
        s_T = ~0ull;
        s_bucket = -1;
        s_pre = 0ull;
    }
    __syncthreads();
    if (warp == 0) {
        float mn1 = 3.4e38f, mx1 = 0.f, mn2 = 3.4e38f, mx2 = 0.f;
        for (int t = lane; t < sk; t += 32) {
            mn1 = fminf(mn1, d1[t]);
            mx1 = fmaxf(mx1, d1[t]);
            mn2 = fminf(mn2, d2[t]);
            mx2 = fmaxf(mx2, d2[t]);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, off));
            mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, off));
            mn2 = fminf(mn2, __shfl_xor_sync(0xffffffffu, mn2, off));
            mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, off));
        }
        if (lane == 0) {
            s_min = __float_as_uint(mn1 + mn2);
            s_max = __float_as_uint(mx1 + mx2);
        }
    }
    uint32_t kb[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const int cell = tid + kSelThreads * u;
        kb[u] = 0xffffffffu;
        if (cell < K) {
            const int r = cell / sk, c = cell - r * sk;
            kb[u] = __float_as_uint(d1[r] + d2[c]);
        }
    }
    __syncthreads();
    if (budget <= n) {
        const uint32_t minb = s_min, range = s_max - s_min;
        const int bits = range ? 32 - __clz(range) : 0;
        const int shift = bits > 11 ? bits - 11 : 0;
#pragma unroll
        for (int u = 0; u < CPT; ++u)
            if (kw[u]) atomicAdd(&hist[(kb[u] - minb) >> shift], kw[u]);
        __syncthreads();
        unsigned long long loc = 0;
#pragma unroll
        for (int j = 0; j < kSelBinsPerThread; ++j) loc += hist[tid * kSelBinsPerThread + j];
        unsigned long long incl = loc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) s_wsum[warp] = uint32_t(incl);
        __syncthreads();
        unsigned long long wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        unsigned long long pre = wpre + incl - loc;
        for (int j = 0; j < kSelBinsPerThread; ++j) {
            const uint32_t hb = hist[tid * kSelBinsPerThread + j];
            if (pre < (unsigned long long)budget && (unsigned long long)budget <= pre + hb) {
                s_bucket = tid * kSelBinsPerThread + j;
                s_pre = pre;
            }
            pre += hb;
        }
        __syncthreads();
        const int bucket = s_bucket;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int cell = tid + kSelThreads * u;
            if (cell < K && int((kb[u] - minb) >> shift) == bucket)
                list[atomicAdd(&s_m, 1)] = (static_cast<unsigned long long>(kb[u]) << 32) | unsigned(cell);
        }
        __syncthreads();
        const int m = s_m;
        int p2 = 1;
        while (p2 < m) p2 <<= 1;
        for (int t = m + tid; t < p2; t += kSelThreads) list[t] = ~0ull;
        __syncthreads();
        for (int k2 = 2; k2 <= p2; k2 <<= 1) {
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < p2; t += kSelThreads) {
                    const int o = t ^ j;
                    if (o > t) {
                        const unsigned long long a = list[t], b = list[o];
                        if ((a > b) == ((t & k2) == 0)) {
                            list[t] = b;
                            list[o] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (warp == 0) {
            unsigned long long cum = s_pre;
            for (int b0 = 0; b0 < m; b0 += 32) {
                const int idx = b0 + lane;
                const unsigned long long key = idx < m ? list[idx] : ~0ull;
                unsigned long long w = idx < m ? sz[uint32_t(key)] : 0ull;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned long long v = __shfl_up_sync(0xffffffffu, w, off);
                    if (lane >= off) w += v;
                }
                const bool hit = idx < m && cum + w >= (unsigned long long)budget;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (bal) {
                    if (lane == __ffs(bal) - 1) s_T = key;
                    break;
                }
                cum += __shfl_sync(0xffffffffu, w, 31);
            }
        }
        __syncthreads();
    }
    const unsigned long long T = s_T;
    const size_t qi_off = (size_t(q) * Ns + i);
    unsigned long long ret = 0;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const int cell = tid + kSelThreads * u;
        const bool take = cell < K &&
                          ((static_cast<unsigned long long>(kb[u]) << 32) | unsigned(cell)) <= T;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        int wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&s_cnt, __popc(bal));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (take) {
            cells_out[qi_off * K + wbase + __popc(bal & ((1u << lane) - 1u))] = uint16_t(cell);
            ret += kw[u];
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) ret += __shfl_xor_sync(0xffffffffu, ret, off);
    if (lane == 0 && ret) atomicAdd(&s_ret, ret);
    __syncthreads();
    if (tid == 0) {
        ncells_out[qi_off] = s_cnt;
        retrieved_out[qi_off] = (long long)s_ret;
    }
}

// Debug output of Alg. 4: flags[pair][cell] = 1 for the cells the probe step wrote for that
// (query, subspace) pair, whichever probe kernel settled it; one warp per pair. The flags
// were zeroed by the caller.
__global__ void __launch_bounds__(256)
expand_probed_kernel(const uint16_t* __restrict__ cells, const int32_t* __restrict__ ncells, int K,
                     int64_t pairs, uint8_t* __restrict__ flags) {
    const int64_t p = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    if (p >= pairs) return;
    const int m = ncells[p];
    for (int t = threadIdx.x & 31; t < m; t += 32) flags[size_t(p) * K + cells[size_t(p) * K + t]] = 1;
}

// Shared memory of one warp of final_merge_kernel: the lists and merge buffers, rounded up
// to 16 bytes, then the query row (d_pad floats; d_pad is a multiple of 8).
__host__ __device__ __forceinline__ size_t merge_head_bytes(int ncta, int kkc) {
    return (size_t(ncta) * kkc * 8 + size_t(4) * kkc * 4 + 15) & ~size_t(15);
}
__host__ __device__ __forceinline__ size_t merge_warp_bytes(int ncta, int kkc, int d_pad) {
    return merge_head_bytes(ncta, kkc) + size_t(d_pad) * 4;
}

// Per query, one warp merges the top lists of every warp of the cluster (Alg. 6 step 9:
// the k nearest candidates) and writes the result: first the kRrWarps lists of each CTA,
// then the cluster's CTA lists. For BF16 rows the merged list is a shortlist: the warp
// recomputes its distances from the FP32 rows and sorts them by (distance, id) first.
template <bool BF16>
__global__ void __launch_bounds__(256)
final_merge_kernel(const float* __restrict__ lists_d, const uint32_t* __restrict__ lists_i,
                   int ncta, int kk, int kkc, const float* __restrict__ queries, int d, int d_pad,
                   const float* __restrict__ data, QueryParamsDev defaults,
                   const QueryParamsDev* __restrict__ params, int64_t nq,
                   int64_t* __restrict__ out_ids, float* __restrict__ out_dists, int k_stride,
                   const uint32_t* __restrict__ qmask) {
    extern __shared__ __align__(16) unsigned char fm[];
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = int64_t(blockIdx.x) * nw + warp;
    if (q >= nq) return;
    if (qmask && !qmask[q]) return;
    float* cd = reinterpret_cast<float*>(fm + warp * merge_warp_bytes(ncta, kkc, d_pad));   // [ncta][kkc]
    uint32_t* ci = reinterpret_cast<uint32_t*>(cd + ncta * kkc);  // [ncta][kkc]
    float* od = reinterpret_cast<float*>(ci + ncta * kkc);
    uint32_t* oi = reinterpret_cast<uint32_t*>(od + kkc);
    float* xd = reinterpret_cast<float*>(oi + kkc);
    uint32_t* xi = reinterpret_cast<uint32_t*>(xd + kkc);
    // the query row is read as float4: it starts on a 16-byte boundary
    float* qv = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(cd) + merge_head_bytes(ncta, kkc));
    const QueryParamsDev qp = params ? params[q] : defaults;
    for (int r = 0; r < ncta; ++r) {
        const size_t row = (size_t(q) * ncta + r) * kRrWarps * kk;
        warp_merge(lists_d + row, lists_i + row, kk, kRrWarps, kk, cd + r * kkc, ci + r * kkc, lane);
    }
    __syncwarp();
    warp_merge(cd, ci, kkc, ncta, kk, od, oi, lane);
    __syncwarp();
    // the query's own shortlist: the first qp.kk of the merged list (lists are as long as
    // the batch's longest; a shorter shortlist is a prefix of them)
    const int kq = min(qp.kk, kk);
    if constexpr (BF16) {
        for (int j = lane; j < d_pad; j += 32) qv[j] = j < d ? queries[q * d + j] : 0.f;
        __syncwarp();
        const int nf4 = d_pad / 4;
        const float4* q4 = reinterpret_cast<const float4*>(qv);
        for (int e0 = 0; e0 < kq; e0 += 4) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int f = lane; f < nf4; f += 32) {
                float4 r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u;
                    const uint32_t id = e < kq ? oi[e] : kNoId;
                    r[u] = id != kNoId ? __ldg(reinterpret_cast<const float4*>(data + size_t(id) * d_pad) + f)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = sq4(r[u], q4[f], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int off = 16; off; off >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], off);
                const int e = e0 + u;
                if (lane == 0 && e < kq) {
                    xd[e] = oi[e] != kNoId ? acc[u] : __int_as_float(0x7f800000);
                    xi[e] = oi[e];
                }
            }
        }
        __syncwarp();
        // rank sort (ties between padding entries by position)
        for (int e = lane; e < kq; e += 32) {
            const float x = xd[e];
            const uint32_t xid = xi[e];
            int rank = 0;
            for (int f = 0; f < kq; ++f)
                rank += lt_pair(xd[f], xi[f], x, xid) || (xd[f] == x && xi[f] == xid && f < e);
            od[rank] = x;
            oi[rank] = xid;
        }
        __syncwarp();
    }
    for (int t = lane; t < k_stride; t += 32) {
        const bool ok = t < qp.k && t < kq && oi[t] != kNoId;
        out_ids[q * k_stride + t] = ok ? int64_t(oi[t]) : int64_t(-1);
        out_dists[q * k_stride + t] = ok ? sqrtf(od[t]) : __int_as_float(0x7f800000);
    }
}

// Level counts of one id-range shard: hist[q][0] = the shard's points, hist[q][j] = its ids
// with SC >= j (the sum of its units' counts), j = 1..N_s. One thread per (query, level).
__global__ void shard_hist_kernel(const uint32_t* __restrict__ unit_ge, int64_t nq, int nr, int r0, int r1,
                                  int Ns, int64_t points, int64_t* __restrict__ hist) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= nq * (Ns + 1)) return;
    const int64_t q = t / (Ns + 1);
    const int j = int(t - q * (Ns + 1));
    int64_t v = points;
    if (j > 0) {
        v = 0;
        for (int r = r0; r < r1; ++r) v += unit_ge[(q * nr + r) * 16 + j];
    }
    hist[t] = v;
}

cudaError_t launch_shard_hist(const uint32_t* unit_ge, int64_t nq, int nr, int r0, int r1, int Ns, int64_t points,
                              int64_t* hist, cudaStream_t st) {
    const int64_t n = nq * (Ns + 1);
    if (n == 0) return cudaSuccess;
    shard_hist_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(unit_ge, nq, nr, r0, r1, Ns, points, hist);
    return cudaGetLastError();
}

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// The most counter slabs one CTA of the cluster kernel holds: its dynamic shared memory is
// the counters plus the query row, the candidate buffer, the level list and the staging
// arrays (the launch's byte count), and its static shared memory stays under 4 KB; all of it
// must fit the 227 KB a CTA can opt into.
static int cluster_spc_max(const taco_index* ix) {
    const size_t beyond = size_t(ix->d_pad) * 4 + size_t(kBufCap) * 4 + size_t(kListCap) * 4 +
                          size_t(kCellBatch) * 4 + size_t(kCellBatch + kRunPad) * 4 + 32 * 4 + 4096;
    const size_t limit = size_t(227) * 1024;
    return limit > beyond ? int((limit - beyond) / kSlabBytes) : 0;
}

// Cluster size and slabs per CTA for an index (called once at index creation).
int configure_search(taco_index* ix) {
    ix->n_slabs = int((ix->n + kSlabIds - 1) / kSlabIds);
    const int spc_max = std::min(12, cluster_spc_max(ix));
    // Aim for 4 slabs (64 KB of counters) per CTA so two clusters' CTAs share an SM.
    int spc = 4;
    int cluster = (ix->n_slabs + spc - 1) / spc;
    if (cluster > 8) {
        // grow the per-CTA range before going past the portable cluster size
        spc = (ix->n_slabs + 7) / 8;
        cluster = (ix->n_slabs + spc - 1) / spc;
    }
    if (spc > spc_max) {
        spc = (ix->n_slabs + 15) / 16;
        cluster = (ix->n_slabs + spc - 1) / spc;
    }
    // the two-pass counting's default layout: the widest ranges a CTA's shared memory holds
    // (12 slabs of 4-bit counters, 15 of 3-bit where N_s <= 7), one 512-thread CTA per SM;
    // on the 1M x 128 and 10M x 96 workloads this beat narrower ranges with two CTAs per SM
    ix->tp_spc = ix->tp_spc0 = std::min(ix->Ns <= 7 ? 15 : 12, ix->n_slabs);
    ix->tp_ranges = ix->tp_ranges0 = (ix->n_slabs + ix->tp_spc - 1) / ix->tp_spc;
    if (spc > spc_max || cluster > 16) {
        // no cluster holds a query's counters: flagged queries take the codes fallback
        ix->cluster = 0;
        ix->slabs_per_cta = 0;
        return TACO_OK;
    }
    if (cluster < 1) cluster = 1;
    if (spc > ix->n_slabs) spc = ix->n_slabs;
    ix->cluster = cluster;
    ix->slabs_per_cta = spc;
    return TACO_OK;
}

static int pick_g(int nchunks) {
    // lanes per row so that each lane issues about 2 sixteen-byte loads per row
    int g = 4;
    while (g < 32 && g * 2 < nchunks) g <<= 1;
    return g;
}

static cudaEvent_t prof_event(Profiler& pr) {
    if (pr.used == pr.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pr.pool.push_back(e);
    }
    return pr.pool[pr.used++];
}

cudaError_t ensure_dynamic_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{func, dev}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int prof_begin(taco_index* ix, int slot, cudaStream_t st, cudaEvent_t* b, cudaEvent_t* e) {
    (void)slot;
    *b = *e = nullptr;
    if (!ix || !ix->prof.enabled) return TACO_OK;
    *b = prof_event(ix->prof);
    *e = prof_event(ix->prof);
    if (!*b || !*e) return fail(TACO_ECUDA, "cudaEventCreate failed");
    TACO_CUDA(cudaEventRecord(*b, st));
    return TACO_OK;
}

int prof_end(taco_index* ix, int slot, cudaStream_t st, cudaEvent_t b, cudaEvent_t e) {
    if (!b) return TACO_OK;
    TACO_CUDA(cudaEventRecord(e, st));
    ix->prof.pending.push_back({slot, {b, e}});
    return TACO_OK;
}

// prof_end for an event pair around `kernels` launches of one slot (the slot's launch count
// grows by that many; taco_profile_read takes the count from bits 8 and up of the entry).
static int prof_end_n(taco_index* ix, int slot, int kernels, cudaStream_t st, cudaEvent_t b, cudaEvent_t e) {
    return prof_end(ix, slot | (kernels << 8), st, b, e);
}

// The select / re-rank kernel for a row kind (0 FP32, 1 BF16, 2 FP8) with G lanes per row.
static cudaError_t launch_select(int rk, int G, const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st) {
    return rk == 2 ? launch_select_b2(G, P, nq, smem, st)
                   : (rk == 1 ? launch_select_b1(G, P, nq, smem, st) : launch_select_b0(G, P, nq, smem, st));
}

int run_search_chunk(const SearchLaunch& L, cudaStream_t st) {
    taco_index* ix = const_cast<taco_index*>(L.ix);
    taco_index* pix = L.skip_profile ? nullptr : ix;   // profiling target (none: no events)
    cudaEvent_t pb, pe;
    const int K = ix->K;
    // (phase 2 of a shard: the transform, probe and counts of phase 1 are in the workspace)
    if (L.phase != 2) {
    // 1. transform (Alg. 6 step 1)
    if (int rc = prof_begin(pix, 0, st, &pb, &pe)) return rc;
    TACO_CUDA(launch_project(L.queries, L.nq, ix->d, ix->d, ix->d_obar, ix->d_B, ix->Dp, L.qt, st));
    if (int rc = prof_end(pix, 0, st, pb, pe)) return rc;
    if (L.dbg.query_t)
        TACO_CUDA(cudaMemcpyAsync(L.dbg.query_t, L.qt, size_t(L.nq) * ix->Dp * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));
    // 1b. the query x centroid block on the tensor cores (probe_precision BF16)
    const float* hd = nullptr;
    if (L.centroid_tc) {
        if (int rc = prof_begin(pix, 6, st, &pb, &pe)) return rc;
        TACO_CUDA(launch_centroid_dist(ix, L.qt, L.nq, L.centroid_tc, L.hd, st));
        if (int rc = prof_end(pix, 6, st, pb, pe)) return rc;
        hd = L.hd;
    }
    // 2. per (query, subspace) probed cells (Alg. 6 steps 3-6, Alg. 4)
    {
        const int cap = next_pow2(K);
        const size_t smem = size_t(cap) * 8 + kSelBins * 4 + size_t(2) * ix->sk * 4;
        static thread_local bool attr_set = false;
        if (smem > 48 * 1024 && !attr_set) {
            TACO_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(probe_cells_kernel), 200 * 1024));
            attr_set = true;
        }
        // the register variant handles K <= 4096, whose list needs at most 48 KB

        dim3 grid(unsigned(ix->Ns), unsigned(L.nq));
        if (int rc = prof_begin(pix, 1, st, &pb, &pe)) return rc;
        // the row-merge walk settles small budgets; the histogram kernel redoes what it flags
        // (and does everything when the budget needs many pops). Debug outputs change nothing
        // here: the probed-cell flags are expanded afterwards from the cells this step wrote.
        bool walk = ix->sk <= 128 && ix->tp_walk != 0;
        if (walk && ix->tp_walk < 0 && L.params == nullptr &&
            double(L.defaults.budget) * double(K) > 0.5 * kWalkMaxPops * double(ix->n))
            walk = false;
        if (walk) {
            const int64_t ntasks = L.nq * ix->Ns;
            const unsigned blocks = unsigned((ntasks + kWalkThreads / 32 - 1) / (kWalkThreads / 32));
#define TACO_PROBE_WALK(E)                                                                        \
    probe_cells_walk_kernel<E><<<blocks, kWalkThreads, 0, st>>>(                                  \
        L.qt, ix->Dp, ix->d_cent, hd, ix->Ns, ix->s, ix->h1, ix->sk, ix->d_sizes, ix->n, L.defaults, \
        L.params, ntasks, L.cells, L.ncells, L.retrieved)
            if (ix->sk <= 32) TACO_PROBE_WALK(1);
            else if (ix->sk <= 64) TACO_PROBE_WALK(2);
            else TACO_PROBE_WALK(4);
#undef TACO_PROBE_WALK
            TACO_CUDA(cudaGetLastError());
        }
        const int redo = walk ? 1 : 0;
        const int cpt = (K + kSelThreads - 1) / kSelThreads;
#define TACO_PROBE_REG(N)                                                                         \
    probe_cells_reg_kernel<N><<<grid, kSelThreads, smem, st>>>(                                   \
        L.qt, ix->Dp, ix->d_cent, hd, ix->Ns, ix->s, ix->h1, ix->sk, ix->d_sizes, ix->n, L.defaults, \
        L.params, cap, L.cells, L.ncells, L.retrieved, redo)
        if (cpt <= 1) TACO_PROBE_REG(1);
        else if (cpt <= 2) TACO_PROBE_REG(2);
        else if (cpt <= 4) TACO_PROBE_REG(4);
        else if (cpt <= 8) TACO_PROBE_REG(8);
        else if (cpt <= 16) TACO_PROBE_REG(16);
        else
            probe_cells_kernel<<<grid, kSelThreads, smem, st>>>(
                L.qt, ix->Dp, ix->d_cent, hd, ix->Ns, ix->s, ix->h1, ix->sk, ix->d_sizes, ix->n,
                L.defaults, L.params, cap, L.cells, L.ncells, L.retrieved, redo);
#undef TACO_PROBE_REG
        TACO_CUDA(cudaGetLastError());
        if (int rc = prof_end_n(pix, 1, walk ? 2 : 1, st, pb, pe)) return rc;   // walk + histogram kernel
        if (L.dbg.probed) {
            TACO_CUDA(cudaMemsetAsync(L.dbg.probed, 0, size_t(L.nq) * ix->Ns * K, st));
            const int64_t pairs = L.nq * ix->Ns;
            expand_probed_kernel<<<unsigned((pairs + 7) / 8), 256, 0, st>>>(L.cells, L.ncells, K, pairs,
                                                                         L.dbg.probed);
            TACO_CUDA(cudaGetLastError());
        }
        if (L.dbg.retrieved_num)
            TACO_CUDA(cudaMemcpyAsync(L.dbg.retrieved_num, L.retrieved,
                                      size_t(L.nq) * ix->Ns * sizeof(int64_t),
                                      cudaMemcpyDeviceToDevice, st));
    }
    }   // phase != 2
    // 3. count, select, re-rank (Alg. 6 steps 7-9, Alg. 5)
    {
        // FP8 rows serve the select / re-rank pass; queries on the fallback cluster path
        // re-rank with FP32 rows
        const bool fp8 = L.precision == TACO_PREC_FP8;
        const bool bf16 = L.precision == TACO_PREC_BF16;
        RerankParams P = {};
        P.queries = L.queries;
        P.data = ix->d_data;
        P.data_bf16 = ix->d_data_bf16;
        P.data_fp8 = ix->d_data_fp8;
        P.fp8_scale = ix->d_fp8_scale;
        P.qt = L.qt;
        P.Dp = ix->Dp;
        P.dp8 = ix->dp8;
        P.obar = ix->d_obar;
        P.fp8_space = ix->fp8_space;
        P.ids = ix->d_ids;
        P.split = ix->d_split;
        P.n_ids = ix->n_ids;
        P.status = ix->d_status;
        P.list_rows = size_t(L.nq) * ix->cluster * kListsPerCta;
        P.cells = L.cells;
        P.ncells = L.ncells;
        P.params = L.params;
        P.defaults = L.defaults;
        P.n = ix->n;
        P.d = ix->d;
        P.d_pad = ix->d_pad;
        P.Ns = ix->Ns;
        P.K = K;
        P.n_slabs = ix->n_slabs;
        P.slabs_per_cta = ix->slabs_per_cta;
        P.counter_words = ix->slabs_per_cta * kSlabWords;
        P.kk = L.kk_max;
        P.kkc = next_pow2(L.kk_max);
        P.nq = L.nq;
        P.region_a = (size_t(P.counter_words) * 4 + 15) & ~size_t(15);
        P.lists_d = L.lists_d;
        P.lists_i = L.lists_i;
        P.out_ids = L.out_ids;
        P.out_dists = L.out_dists;
        P.k_stride = L.k_stride;
        P.dbg_sc = L.dbg.sc;
        P.dbg_hist = L.dbg.collision_num;
        P.dbg_last = L.dbg.last_collision;
        P.dbg_cand = L.dbg.candidate_num;
        P.buf_cap = kBufCap;
        P.n_ranges = ix->cluster;
        if (L.dbg.sc) TACO_CUDA(cudaMemsetAsync(L.dbg.sc, 0, size_t(L.nq) * ix->n, st));
        const int R = L.kk_max <= 32 ? 1 : (L.kk_max <= 128 ? 4 : 16);
        const int G = pick_g(ix->d_pad / (bf16 ? 8 : 4));
        const int rk = fp8 ? 2 : (bf16 ? 1 : 0);
        // lanes per row of the select pass (tuned, else from the chunks a row holds)
        const int Gs = ix->tp_lanes[rk] ? ix->tp_lanes[rk]
                                        : (fp8 ? pick_g(((ix->fp8_space ? ix->d : ix->Dp) + 15) / 16) : G);
        const bool two_pass = L.unit_ge != nullptr;
        if (two_pass) {
            // the two-pass range layout (tuned): tp_spc slabs of counters per range
            // (4-bit counters up to 12 slabs, 3-bit counters for 13-15 slabs, N_s <= 7)
            const int cb = ix->tp_spc > 12 ? 3 : 4;
            P.slabs_per_cta = ix->tp_spc;
            P.counter_words = (counter_words_for(int64_t(ix->tp_spc) * kSlabIds, cb) + 3) & ~3;
            P.region_a = size_t(P.counter_words) * 4 + 32 * 4;   // + the walk's 32 spare words
            P.n_ranges = ix->tp_ranges;
            P.arena_per_unit = uint32_t(kArenaPerSlab) * uint32_t(ix->tp_spc);
            P.arena_words = size_t(L.nq) * ix->tp_ranges * P.arena_per_unit;
            P.unit_ge = L.unit_ge;
            P.unit_off = L.unit_off;
            P.unit_len = L.unit_len;
            P.arena = L.arena;
            P.qflag = L.qflag;
            P.qlast = L.qlast;
            P.work = L.qflag + L.nq;   // the two query counters follow the flags
            P.shard_r0 = L.shard_r1 > 0 ? L.shard_r0 : 0;
            P.shard_r1 = L.shard_r1 > 0 ? L.shard_r1 : ix->tp_ranges;
            P.ghist = L.phase == 2 ? L.ghist : nullptr;
            if (L.phase != 2)
                TACO_CUDA(cudaMemsetAsync(L.qflag, 0, size_t(L.nq + 2) * sizeof(uint32_t), st));
            // pass 1: counting per (query, id range) unit; 256, 512 or 1024 threads per CTA and
            // 2, 4 or 8 chunk windows per walk round (tuned)
            struct CountVariant {
                int nw, wu, cb;
                void (*fn)(const RerankParams);
            };
            static const CountVariant kVariants[] = {
                {8, 2, 4, count_lists_kernel<8, 2, 4>},   {8, 4, 4, count_lists_kernel<8, 4, 4>},
                {16, 2, 4, count_lists_kernel<16, 2, 4>}, {16, 4, 4, count_lists_kernel<16, 4, 4>},
                {16, 8, 4, count_lists_kernel<16, 8, 4>}, {32, 2, 4, count_lists_kernel<32, 2, 4>},
                {32, 4, 4, count_lists_kernel<32, 4, 4>}, {8, 2, 3, count_lists_kernel<8, 2, 3>},
                {8, 4, 3, count_lists_kernel<8, 4, 3>},   {16, 2, 3, count_lists_kernel<16, 2, 3>},
                {16, 4, 3, count_lists_kernel<16, 4, 3>}, {16, 8, 3, count_lists_kernel<16, 8, 3>},
                {32, 2, 3, count_lists_kernel<32, 2, 3>}, {32, 4, 3, count_lists_kernel<32, 4, 3>}};
            constexpr int kNumVariants = int(sizeof(kVariants) / sizeof(kVariants[0]));
            int c1 = cb == 4 ? 3 : 10;   // 16 x 4 unless the tuned pair exists
            for (int v = 0; v < kNumVariants; ++v)
                if (kVariants[v].nw == ix->tp_count_warps && kVariants[v].wu == ix->tp_walk_unroll &&
                    kVariants[v].cb == cb)
                    c1 = v;
            const int nw1 = kVariants[c1].nw;
            auto k1 = kVariants[c1].fn;
            const size_t smem1 = P.region_a + count_lists_extra();
            static thread_local size_t c1_smem[kNumVariants] = {};
            static thread_local int c1_blocks[kNumVariants] = {};
            if (c1_smem[c1] != smem1) {
                TACO_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(k1), smem1));
                int per_sm = 0, sms = 0;
                TACO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, nw1 * 32, smem1));
                TACO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
                if (per_sm < 1) return fail(TACO_ECAPACITY, "count_lists_kernel does not fit an SM");
                c1_blocks[c1] = per_sm * sms;
                c1_smem[c1] = smem1;
            }
            // a batch smaller than the resident CTAs splits each query's ranges into runs
            // (work items) so that more CTAs count it
            const int own = P.shard_r1 - P.shard_r0;   // ranges this launch counts
            P.range_parts = 1;
            if (L.nq < c1_blocks[c1]) {
                const int want = int(std::min<int64_t>(own, (c1_blocks[c1] + L.nq - 1) / L.nq));
                const int per_part = (own + want - 1) / want;
                P.range_parts = (own + per_part - 1) / per_part;
            }
            if (L.phase != 2) {
                if (int rc = prof_begin(pix, 2, st, &pb, &pe)) return rc;
                k1<<<unsigned(std::min<int64_t>(L.nq * P.range_parts, c1_blocks[c1])), nw1 * 32, smem1, st>>>(P);
                TACO_CUDA(cudaGetLastError());
                if (int rc = prof_end(pix, 2, st, pb, pe)) return rc;
            }
            if (L.phase == 1) {
                // the shard's level counts for the all-shard sum (Alg. 5 needs the whole
                // histogram): [q][0] = the shard's points, [q][j] = its ids with SC >= j
                const int64_t lo = int64_t(P.shard_r0) * ix->tp_spc * kSlabIds;
                const int64_t hi = std::min<int64_t>(int64_t(P.shard_r1) * ix->tp_spc * kSlabIds, ix->n);
                TACO_CUDA(launch_shard_hist(L.unit_ge, L.nq, ix->tp_ranges, P.shard_r0, P.shard_r1, ix->Ns,
                                            hi - lo, L.shard_hist, st));
                return TACO_OK;
            }
            // pass 2: Alg. 5, candidates, re-rank, results
            const size_t smem2 = select_smem_bytes(P.kkc, ix->d_pad, fp8 ? ix->dp8 : 0, P.n_ranges, ix->Ns, K, false);
            if (int rc = prof_begin(pix, 3, st, &pb, &pe)) return rc;
            const cudaError_t e = launch_select(rk, Gs, P, L.nq, smem2, st);
            if (e != cudaSuccess) return cuda_fail(e, "select_rerank launch", __FILE__, __LINE__);
            if (int rc = prof_end(pix, 3, st, pb, pe)) return rc;
            P.qmask = L.qflag;   // the cluster kernel below only answers flagged queries
            P.slabs_per_cta = ix->slabs_per_cta;   // back to the cluster layout
            P.counter_words = ix->slabs_per_cta * kSlabWords;
            P.region_a = (size_t(P.counter_words) * 4 + 15) & ~size_t(15);
            P.n_ranges = ix->cluster;
        }
        if (two_pass && (ix->codes_fallback || L.phase == 2)) {
            // codes fallback for the flagged queries: the select pass again, in fallback mode
            // (a shard always takes it: the cluster kernel counts every id of the index)
            P.fb_mode = 1;
            P.codes = ix->d_codes;
            P.slabs_per_cta = ix->tp_spc;
            P.n_ranges = ix->tp_ranges;
            const size_t smem3 = select_smem_bytes(P.kkc, ix->d_pad, fp8 ? ix->dp8 : 0, P.n_ranges, ix->Ns, K, true);
            if (int rc = prof_begin(pix, 4, st, &pb, &pe)) return rc;
            const cudaError_t e = launch_select(rk, Gs, P, L.nq, smem3, st);
            if (e != cudaSuccess) return cuda_fail(e, "codes fallback launch", __FILE__, __LINE__);
            if (int rc = prof_end(pix, 4, st, pb, pe)) return rc;
            return TACO_OK;
        }
        if (ix->cluster == 0) return fail(TACO_ECAPACITY, "no cluster layout for n = %lld", (long long)ix->n);
        // cluster kernel: every query (single-pass form) or the flagged ones
        const size_t smem = P.region_a + size_t(ix->d_pad) * 4 + size_t(P.buf_cap) * 4 +
                            size_t(kListCap) * 4 + size_t(kCellBatch) * 4 + size_t(kCellBatch + kRunPad) * 4 + 32 * 4;
        cudaError_t e;
        if (int rc = prof_begin(pix, 4, st, &pb, &pe)) return rc;
        if (!bf16) {
            e = R == 1 ? launch_rerank_b0_r1(G, P, ix->cluster, L.nq, smem, st)
                : R == 4 ? launch_rerank_b0_r4(G, P, ix->cluster, L.nq, smem, st)
                         : launch_rerank_b0_r16(G, P, ix->cluster, L.nq, smem, st);
        } else {
            e = R == 1 ? launch_rerank_b1_r1(G, P, ix->cluster, L.nq, smem, st)
                : R == 4 ? launch_rerank_b1_r4(G, P, ix->cluster, L.nq, smem, st)
                         : launch_rerank_b1_r16(G, P, ix->cluster, L.nq, smem, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "count_select_rerank launch", __FILE__, __LINE__);
        if (int rc = prof_end(pix, 4, st, pb, pe)) return rc;
        // merge of the cluster kernel's lists (and BF16 shortlist re-rank)
        const size_t per_warp = merge_warp_bytes(ix->cluster, P.kkc, ix->d_pad);
        int fw = 8;
        while (fw > 1 && size_t(fw) * per_warp > 160 * 1024) fw >>= 1;
        const size_t fsm = size_t(fw) * per_warp;
        auto fk = bf16 ? final_merge_kernel<true> : final_merge_kernel<false>;
        if (fsm > 48 * 1024) TACO_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(fk), fsm));
        if (int rc = prof_begin(pix, 5, st, &pb, &pe)) return rc;
        fk<<<unsigned((L.nq + fw - 1) / fw), fw * 32, fsm, st>>>(
            L.lists_d, L.lists_i, ix->cluster, P.kk, P.kkc, L.queries, ix->d, ix->d_pad, ix->d_data,
            L.defaults, L.params, L.nq, L.out_ids, L.out_dists, L.k_stride, P.qmask);
        TACO_CUDA(cudaGetLastError());
        if (int rc = prof_end(pix, 5, st, pb, pe)) return rc;
    }
    return TACO_OK;
}

}  // namespace taco

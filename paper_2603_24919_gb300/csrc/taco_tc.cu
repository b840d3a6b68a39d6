// Query x centroid distance block of Alg. 6 steps 4-5 on the tcgen05 tensor cores.
//
// For every subspace i and half h the squared distances of the transformed half-queries to
// the sqrt(K) half-centroids form a dense product: dist[q][c] = |q|^2 + |c|^2 - 2 q.c with
// Q_{i,h} [nq x len] and C_{i,h} [sqrt(K) x len]. One CTA (4 warps) takes 128 queries and
// a stage of its 2 N_s (subspace, half) pairs: the centroid operands (BF16, already in the tensor-core
// shared-memory layout, built with the index) arrive by bulk asynchronous copy (cp.async.bulk,
// completion counted on an mbarrier), the threads write the BF16 half-queries, and one
// thread issues the MMAs (kind::f16, M = 128, N = sqrt(K) rounded up to 16, K steps of 16)
// into tensor-memory accumulators and commits them to a second mbarrier, and each warp reads
// its 32 accumulator lanes back (tcgen05.ld) and writes the distances from registers. A CTA
// takes one stage of up to 128 / N pairs (an accumulator of N TMEM columns per pair, so four
// CTAs share an SM's 512 columns): one bulk copy brings the stage's centroid operands, the
// threads stage its query dimensions with coalesced loads, and one commit covers its MMAs.
// Every wait is bounded: on a timeout the kernel records 1 in the index's status word and
// leaves the stage loop.
//
// Operands are BF16 with FP32 accumulation, so this is the precision form of the block; the
// FP32 path computes the same distances on CUDA cores (centroid_dist_simt_kernel and the
// fused code of the probe kernels).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "taco_internal.h"

namespace taco {
namespace {

constexpr int kTcM = 128;        // queries per CTA (MMA M; one TMEM lane per query)
constexpr int kTcThreads = 128;  // 4 warps: warp w reads TMEM lanes 32 w .. 32 w + 31
constexpr uint32_t kTcWaitPolls = 1u << 22;   // bounded mbarrier waits (~0.3 s with backoff)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of a K-major operand without swizzle: 8-row x 16-byte core
// matrices; `lbo` = byte distance between core matrices adjacent along K, `sbo` = between
// core matrices adjacent along M / N; bit 46 = descriptor version of tcgen05.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr & 0x3ffffu) >> 4) | (uint64_t((lbo & 0x3ffffu) >> 4) << 16) |
           (uint64_t((sbo & 0x3ffffu) >> 4) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A (bits 7-9 = 1)
// and B (bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
// Instruction descriptor of kind::f8f6f4 with E4M3 A and B (format code 0 in bits 7-9 and
// 10-12), FP32 accumulator, both K-major.
constexpr uint32_t instr_desc_e4m3(int M, int N) {
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of `parity` to complete; false after kTcWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kTcWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 32) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bulk asynchronous global -> shared copy (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// One MMA of kind::f8f6f4 (K = 32 one-byte elements).
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane (load and wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

struct TcGeom {
    int Ns, s, h1, sk, Dp;
    int N;    // sqrt_k rounded up to 16 (>= 16): MMA N
    int KH;   // longer half rounded up to 16 (BF16) or 32 (E4M3) elements: the operands' K extent
};

// E4M3 (the largest finite magnitude is 448) of x * inv, rounded to nearest even, saturating.
__host__ __device__ __forceinline__ uint8_t to_e4m3(float x) {
    return uint8_t(__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3));
}
__device__ __forceinline__ float e4m3_value(uint32_t byte) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw(__nv_fp8_storage_t(byte), __NV_E4M3);
    return __half2float(__half(h));
}

// FP8 = false: BF16 operands, kind::f16. FP8 = true: E4M3 operands with one scale per
// (query, pair) for A and per pair for B (cscale), kind::f8f6f4; the accumulator holds the
// dot product of the scaled values, so q.c = acc * scale_q * scale_c.
template <bool FP8>
__global__ void __launch_bounds__(kTcThreads, 4)
centroid_dist_tc_kernel(const float* __restrict__ qt, int64_t nq, TcGeom g, int G, const uint8_t* __restrict__ cimg,
                        const float* __restrict__ cnorm, const float* __restrict__ cscale, float* __restrict__ hd,
                        int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kEs = FP8 ? 1u : 2u;                   // bytes per element
    const uint32_t abytes = uint32_t(kTcM) * g.KH * kEs;      // one pair's A: [128 / 8][KH bytes / 16] core matrices
    const uint32_t bbytes = uint32_t(g.N) * g.KH * kEs;       // one pair's B: [N / 8][KH bytes / 16] core matrices
    unsigned char* sA = smem;                                 // G pairs' A
    unsigned char* sB = smem + size_t(G) * abytes;            // G pairs' B
    float* sS = reinterpret_cast<float*>(sB + size_t(G) * bbytes);   // FP8: [G][128] query scales
    float* sQ = sS + (FP8 ? size_t(G) * kTcM : 0);            // [128][W + 1] query dims
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = int64_t(blockIdx.x) * kTcM;
    const int P = 2 * g.Ns;
    uint32_t ncols = 32;
    while (ncols < uint32_t(G * g.N)) ncols <<= 1;           // G * N <= 128 (or one pair of N = 128)
    if (warp == 0) tmem_alloc(&s_tmem, ncols);
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = FP8 ? instr_desc_e4m3(kTcM, g.N) : instr_desc_bf16(kTcM, g.N);
    const int kc = int(g.KH * kEs / 16);                      // core matrices along K
    const uint32_t sbo = uint32_t(kc) * 128u;
    uint32_t phase = 0;
    for (int p0 = int(blockIdx.y) * G; p0 < P; p0 += int(gridDim.y) * G) {   // this CTA's stages
        const int np = min(G, P - p0);
        // the stage's centroid operands: one bulk copy (pairs are contiguous in the image)
        if (tid == 0) {
            mbar_expect_tx(&bar_load, uint32_t(np) * bbytes);
            bulk_g2s(sB, cimg + size_t(p0) * bbytes, uint32_t(np) * bbytes, &bar_load);
        }
        // the stage's query dimensions: one contiguous range [d0, d0 + W) of every row, staged
        // with coalesced loads (a warp per row, 4 rows in flight per warp), row pitch W + 1
        const int pl = p0 + np - 1;
        const int d0 = (p0 >> 1) * g.s + ((p0 & 1) ? g.h1 : 0);
        const int W = (pl >> 1) * g.s + ((pl & 1) ? g.s : g.h1) - d0;
#pragma unroll 8
        for (int m = warp; m < kTcM; m += kTcThreads / 32) {
            const bool ok = q0 + m < nq;
            const float* src = qt + (q0 + m) * g.Dp + d0;
            for (int j = lane; j < W; j += 32) sQ[m * (W + 1) + j] = ok ? src[j] : 0.f;
        }
        __syncthreads();
        // this thread's half-queries (row tid of each pair's A), zero past a half's length:
        // BF16, or E4M3 of x / scale with scale = max |x| / 448 of the row's half
        for (int pp = 0; pp < np; ++pp) {
            const int p = p0 + pp, h = p & 1;
            const int len = h ? g.s - g.h1 : g.h1;
            const int base = (p >> 1) * g.s + (h ? g.h1 : 0) - d0;
            const float* x = sQ + tid * (W + 1) + base;
            unsigned char* dst = sA + size_t(pp) * abytes + (tid >> 3) * kc * 128 + (tid & 7) * 16;
            if constexpr (FP8) {
                float amax = 0.f;
                for (int k = 0; k < len; ++k) amax = fmaxf(amax, fabsf(x[k]));
                const float inv = amax > 0.f ? 448.f / amax : 0.f;
                sS[pp * kTcM + tid] = amax > 0.f ? amax / 448.f : 0.f;
                for (int c16 = 0; c16 < kc; ++c16) {
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int k = c16 * 16 + e;
                        const uint32_t b = k < len ? to_e4m3(x[k] * inv) : 0u;
                        w[e >> 2] |= b << (8 * (e & 3));
                    }
                    *reinterpret_cast<uint4*>(dst + c16 * 128) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else {
                for (int c8 = 0; c8 < kc; ++c8) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const int k = c8 * 8 + e;
                        const __nv_bfloat162 b2 =
                            __floats2bfloat162_rn(k < len ? x[k] : 0.f, k + 1 < len ? x[k + 1] : 0.f);
                        uint32_t u;
                        memcpy(&u, &b2, 4);
                        w[e >> 1] = u;
                    }
                    *reinterpret_cast<uint4*>(dst + c8 * 128) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A visible to the MMA
        __syncthreads();
        int failed = 0;
        if (tid == 0) {
            if (mbar_wait(&bar_load, phase)) {
                tc_fence_after();
                for (int pp = 0; pp < np; ++pp) {
                    const uint32_t aaddr = smem_u32(sA + size_t(pp) * abytes);
                    const uint32_t baddr = smem_u32(sB + size_t(pp) * bbytes);
                    // one MMA per 32 bytes of K (16 BF16 or 32 E4M3 elements)
                    for (int t = 0; t < int(g.KH * kEs / 32); ++t) {
                        const uint64_t da = smem_desc(aaddr + t * 256, 128, sbo);
                        const uint64_t db = smem_desc(baddr + t * 256, 128, sbo);
                        if constexpr (FP8) mma_e4m3(tmem + uint32_t(pp * g.N), da, db, idesc, t > 0 ? 1u : 0u);
                        else mma_bf16(tmem + uint32_t(pp * g.N), da, db, idesc, t > 0 ? 1u : 0u);
                    }
                }
                mma_commit(&bar_mma);
            } else {
                failed = 1;
            }
        }
        if (__syncthreads_or(failed)) {
            if (tid == 0) atomicExch(status, 1);
            break;
        }
        failed = mbar_wait(&bar_mma, phase) ? 0 : 1;
        if (__syncthreads_or(failed)) {
            if (tid == 0) atomicExch(status, 1);
            break;
        }
        tc_fence_after();
        for (int pp = 0; pp < np; ++pp) {
            const int p = p0 + pp, i = p >> 1, h = p & 1;
            // |q|^2 of this row's half-query as the operand holds it, from the A operand itself
            float qn = 0.f, dscale = 1.f;
            const unsigned char* row = sA + size_t(pp) * abytes + (tid >> 3) * kc * 128 + (tid & 7) * 16;
            for (int c8 = 0; c8 < kc; ++c8) {
                const uint4 u = *reinterpret_cast<const uint4*>(row + c8 * 128);
                if constexpr (FP8) {
                    const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float f = e4m3_value((w4[e >> 2] >> (8 * (e & 3))) & 0xffu);
                        qn = fmaf(f, f, qn);
                    }
                } else {
                    const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 f = __bfloat1622float2(b2[e]);
                        qn = fmaf(f.x, f.x, qn);
                        qn = fmaf(f.y, f.y, qn);
                    }
                }
            }
            if constexpr (FP8) {   // back to the unscaled values
                const float sq = sS[pp * kTcM + tid];
                qn *= sq * sq;
                dscale = sq * __ldg(cscale + p);
            }
            const float* cn = cnorm + size_t(p) * g.N;
            const int64_t q = q0 + tid;                       // TMEM lane tid = this query
            float* out = hd + ((q * g.Ns + i) * 2 + h) * g.sk;
            const bool vec = (g.sk & 3) == 0;                 // rows start on 16 bytes
            for (int c0 = 0; c0 < g.N; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(pp * g.N + c0), v);
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = fmaxf(qn + __ldg(cn + c0 + e) - 2.f * (v[e] * dscale), 0.f);
                if (q < nq) {
                    if (vec) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            if (c0 + e < g.sk)
                                *reinterpret_cast<float4*>(out + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (c0 + e < g.sk) out[c0 + e] = v[e];
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // A, B and the accumulators are free for the next stage
        phase ^= 1u;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// The same block in FP32 on CUDA cores, sum of squared differences (one thread per
// (query, pair, centroid)).
__global__ void centroid_dist_simt_kernel(const float* __restrict__ qt, int64_t nq, TcGeom g,
                                          const float* __restrict__ cent, float* __restrict__ hd) {
    const int64_t total = nq * 2 * g.Ns * g.sk;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(t % g.sk);
        const int64_t r = t / g.sk;
        const int h = int(r % 2);
        const int i = int((r / 2) % g.Ns);
        const int64_t q = r / (2 * g.Ns);
        const int off = h ? g.h1 : 0, len = h ? g.s - g.h1 : g.h1;
        const float* qi = qt + q * g.Dp + size_t(i) * g.s + off;
        const float* cc = cent + (size_t(i) * g.sk + c) * g.s + off;
        float acc = 0.f;
        for (int j = 0; j < len; ++j) {
            const float df = qi[j] - cc[j];
            acc = fmaf(df, df, acc);
        }
        hd[t] = acc;
    }
}

TcGeom geom_of(const taco_index* ix, bool fp8 = false) {
    TcGeom g;
    g.Ns = ix->Ns;
    g.s = ix->s;
    g.h1 = ix->h1;
    g.sk = ix->sk;
    g.Dp = ix->Dp;
    g.N = std::max(16, (ix->sk + 15) / 16 * 16);
    const int kq = fp8 ? 32 : 16;   // elements of one MMA's K (32 bytes)
    g.KH = std::max(kq, (std::max(ix->h1, ix->s - ix->h1) + kq - 1) / kq * kq);
    return g;
}

constexpr size_t kTcStageBytes = size_t(54) * 1024;   // operands of one stage (4 CTAs per SM)

// Bytes of one pair in a stage: its A and B operands, its query dimensions (at most the
// longer half) in the staging tile and, for E4M3, its 128 query scales.
size_t tc_pair_bytes(const TcGeom& g, bool fp8) {
    return size_t(kTcM + g.N) * g.KH * (fp8 ? 1 : 2) + size_t(kTcM) * std::max(g.h1, g.s - g.h1) * 4 +
           (fp8 ? size_t(kTcM) * 4 : 0);
}

// Pairs per stage (one stage per CTA): four CTAs share an SM, so a stage's accumulators fit
// 128 of the 512 TMEM columns and its operands a quarter of the shared memory; the many
// small CTAs spread the block over every SM.
int tc_pairs_per_stage(const TcGeom& g, bool fp8) {
    const int by_tmem = std::max(1, 128 / g.N);
    const int by_smem = int(kTcStageBytes / tc_pair_bytes(g, fp8));
    return std::max(1, std::min({by_tmem, by_smem, 2 * g.Ns}));
}

size_t tc_smem_bytes(const TcGeom& g, int G, bool fp8) {
    // the stage's operands, query scales and staging tile (row pitch W + 1 <= G * longer half
    // + 1), and at least a fifth of the SM's shared memory so that at most four CTAs (4 x 128
    // TMEM columns) share an SM
    const size_t ops = size_t(G) * (kTcM + g.N) * g.KH * (fp8 ? 1 : 2) + (fp8 ? size_t(G) * kTcM * 4 : 0);
    const size_t tile = size_t(kTcM) * (size_t(G) * std::max(g.h1, g.s - g.h1) + 1) * 4;
    return std::max<size_t>(ops + tile, 46 * 1024);
}

// Value of an E4M3 byte (sign, 4 exponent bits with bias 7, 3 mantissa bits; exponent 0 is
// subnormal), for the centroid norms built on the host.
float e4m3_host_value(uint8_t b) {
    const int e = (b >> 3) & 15, m = b & 7;
    const float v = e == 0 ? std::ldexp(float(m) / 8.f, -6) : std::ldexp(1.f + float(m) / 8.f, e - 7);
    return (b & 0x80) ? -v : v;
}

}  // namespace

bool centroid_tc_supported(const taco_index* ix) {
    const TcGeom g = geom_of(ix), g8 = geom_of(ix, true);
    return g.N <= 128 && tc_pair_bytes(g, false) + size_t(kTcM) * 4 <= size_t(200) * 1024 &&
           tc_pair_bytes(g8, true) + size_t(kTcM) * 4 <= size_t(200) * 1024;
}

// The centroid operands of both blocks, in the no-swizzle K-major core-matrix layout
// ([2 N_s] pairs of [N / 8][K bytes / 16] core matrices of 8 rows x 16 bytes): BF16 values with
// their squared norms, and E4M3 values of c / scale_p with scale_p = max |c| / 448 over the
// pair's centroids, with the squared norms of the values they stand for (scale_p^2 sum e^2).
int build_centroid_tc(taco_index* ix) {
    if (!centroid_tc_supported(ix)) return TACO_OK;   // the tensor-core blocks are not offered
    const TcGeom g = geom_of(ix), g8 = geom_of(ix, true);
    const int P = 2 * g.Ns, kc = g.KH / 8, kc8 = g8.KH / 16;
    const size_t bbytes = size_t(g.N) * g.KH * 2, bbytes8 = size_t(g8.N) * g8.KH;
    std::vector<uint8_t> img(size_t(P) * bbytes, 0), img8(size_t(P) * bbytes8, 0);
    std::vector<float> norm(size_t(P) * g.N, 0.f), norm8(size_t(P) * g.N, 0.f), scale8(P, 0.f);
    for (int p = 0; p < P; ++p) {
        const int i = p >> 1, h = p & 1;
        const int off = h ? g.h1 : 0, len = h ? g.s - g.h1 : g.h1;
        auto cval = [&](int n, int k) { return float(ix->centroids[(size_t(i) * g.sk + n) * g.s + off + k]); };
        float amax = 0.f;
        for (int n = 0; n < g.sk; ++n)
            for (int k = 0; k < len; ++k) amax = std::max(amax, std::fabs(cval(n, k)));
        const float inv = amax > 0.f ? 448.f / amax : 0.f, sc = amax > 0.f ? amax / 448.f : 0.f;
        scale8[p] = sc;
        for (int n = 0; n < g.sk; ++n) {
            float acc = 0.f, acc8 = 0.f;
            for (int k = 0; k < len; ++k) {
                const float x = cval(n, k);
                const __nv_bfloat16 b = __float2bfloat16_rn(x);
                const float r = __bfloat162float(b);
                acc += r * r;
                uint16_t bits;
                std::memcpy(&bits, &b, 2);
                const size_t at = size_t(p) * bbytes + size_t((n / 8) * kc + k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
                std::memcpy(&img[at], &bits, 2);
                const uint8_t e8 = to_e4m3(x * inv);
                const float r8 = e4m3_host_value(e8);
                acc8 += r8 * r8;
                img8[size_t(p) * bbytes8 + size_t((n / 8) * kc8 + k / 16) * 128 + (n % 8) * 16 + (k % 16)] = e8;
            }
            norm[size_t(p) * g.N + n] = acc;
            norm8[size_t(p) * g.N + n] = acc8 * sc * sc;
        }
    }
    cudaError_t e = cudaMalloc(&ix->d_cent_tc, img.size());
    if (e == cudaSuccess) e = cudaMalloc(&ix->d_cent_tc_norm, norm.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ix->d_cent_tc8, img8.size());
    if (e == cudaSuccess) e = cudaMalloc(&ix->d_cent_tc8_norm, norm8.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ix->d_cent_tc8_scale, scale8.size() * 4);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (tensor-core centroids)", __FILE__, __LINE__);
    ix->device_bytes += int64_t(img.size() + norm.size() * 4 + img8.size() + norm8.size() * 4 + scale8.size() * 4);
    TACO_CUDA(cudaMemcpy(ix->d_cent_tc, img.data(), img.size(), cudaMemcpyHostToDevice));
    TACO_CUDA(cudaMemcpy(ix->d_cent_tc_norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice));
    TACO_CUDA(cudaMemcpy(ix->d_cent_tc8, img8.data(), img8.size(), cudaMemcpyHostToDevice));
    TACO_CUDA(cudaMemcpy(ix->d_cent_tc8_norm, norm8.data(), norm8.size() * 4, cudaMemcpyHostToDevice));
    TACO_CUDA(cudaMemcpy(ix->d_cent_tc8_scale, scale8.data(), scale8.size() * 4, cudaMemcpyHostToDevice));
    return TACO_OK;
}

// mode: 0 FP32 on CUDA cores, 1 BF16 on tcgen05, 2 E4M3 on tcgen05.
cudaError_t launch_centroid_dist(const taco_index* ix, const float* qt, int64_t nq, int mode, float* hd,
                                 cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (mode != 0) {
        const bool fp8 = mode == 2;
        if (!ix->d_cent_tc || (fp8 && !ix->d_cent_tc8)) return cudaErrorNotSupported;
        const TcGeom g = geom_of(ix, fp8);
        const int G = tc_pairs_per_stage(g, fp8);
        const size_t smem = tc_smem_bytes(g, G, fp8);
        auto kern = fp8 ? centroid_dist_tc_kernel<true> : centroid_dist_tc_kernel<false>;
        cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
        if (e != cudaSuccess) return e;
        // one CTA per (128 queries, stage of pairs): the stages of a query tile run on
        // different SMs
        const dim3 grid(unsigned((nq + kTcM - 1) / kTcM), unsigned((2 * g.Ns + G - 1) / G));
        kern<<<grid, kTcThreads, smem, st>>>(qt, nq, g, G, fp8 ? ix->d_cent_tc8 : ix->d_cent_tc,
                                             fp8 ? ix->d_cent_tc8_norm : ix->d_cent_tc_norm, ix->d_cent_tc8_scale, hd,
                                             ix->d_status);
        return cudaGetLastError();
    }
    const TcGeom g = geom_of(ix);
    const int64_t total = nq * 2 * g.Ns * g.sk;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    centroid_dist_simt_kernel<<<unsigned(blocks), 256, 0, st>>>(qt, nq, g, ix->d_cent, hd);
    return cudaGetLastError();
}

}  // namespace taco

// Device kernels of the index build (Alg. 1 steps 2-3 and 6-11, Alg. 3 steps 6-9) and the
// query projection of Alg. 6 step 1, which uses the same transform kernel.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "taco_internal.h"

namespace taco {

// ---------------------------------------------------------------------------------------
// Y[rows][Dp] = (X[rows][d] - o_bar) * B[d][Dp]   (Alg. 1: r = B^T (o - o_bar))
// 64x64 output tile per 256-thread CTA, 4x4 outputs per thread, k-steps of 16.
// ---------------------------------------------------------------------------------------
constexpr int kPT = 64, kPK = 16;

__global__ void __launch_bounds__(256)
project_kernel(const float* __restrict__ X, int64_t rows, int d, int64_t ldx,
               const float* __restrict__ obar, const float* __restrict__ B, int Dp,
               float* __restrict__ Y) {
    __shared__ float As[kPK][kPT + 4];
    __shared__ float Bs[kPK][kPT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t row0 = int64_t(blockIdx.x) * kPT;
    const int col0 = blockIdx.y * kPT;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < d; k0 += kPK) {
        for (int e = threadIdx.x; e < kPT * kPK; e += 256) {
            const int r = e / kPK, kk = e % kPK;
            const int64_t gr = row0 + r;
            const int gk = k0 + kk;
            float v = 0.f;
            if (gr < rows && gk < d) v = X[gr * ldx + gk] - obar[gk];
            As[kk][r] = v;
        }
        for (int e = threadIdx.x; e < kPT * kPK; e += 256) {
            const int kk = e / kPT, c = e % kPT;
            const int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < d && gc < Dp) ? B[int64_t(gk) * Dp + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kPK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                a[t] = As[kk][ty * 4 + t];
                b[t] = Bs[kk][tx * 4 + t];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + ty * 4 + i;
        if (gr >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = col0 + tx * 4 + j;
            if (gc < Dp) Y[gr * Dp + gc] = acc[i][j];
        }
    }
}

cudaError_t launch_project(const float* X, int64_t rows, int d, int64_t ldx, const float* obar,
                           const float* B, int Dp, float* Y, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    dim3 grid(unsigned((rows + kPT - 1) / kPT), unsigned((Dp + kPT - 1) / kPT));
    project_kernel<<<grid, 256, 0, st>>>(X, rows, d, ldx, obar, B, Dp, Y);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Column sums in FP64 (Alg. 1 step 2). Each CTA sums a block of rows.
// ---------------------------------------------------------------------------------------
constexpr int kMeanRows = 4096;

__global__ void col_sum_kernel(const float* __restrict__ X, int64_t n, int d, int ldx,
                               double* __restrict__ sums) {
    const int64_t r0 = int64_t(blockIdx.x) * kMeanRows;
    const int64_t r1 = min(n, r0 + kMeanRows);
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) acc += double(X[r * ldx + c]);
        atomicAdd(&sums[c], acc);
    }
}

cudaError_t launch_col_mean(const float* X, int64_t n, int d, int ldx, double* sums,
                            cudaStream_t st) {
    const unsigned blocks = unsigned((n + kMeanRows - 1) / kMeanRows);
    col_sum_kernel<<<blocks, 256, 0, st>>>(X, n, d, ldx, sums);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Sum of (x - mean)(x - mean)^T in FP64 (Alg. 1 step 3, before the 1/(n-1) factor).
// One CTA per (32x32 tile with ta <= tb, block of rows); 256 threads, 2x2 entries each.
// ---------------------------------------------------------------------------------------
constexpr int kCovTile = 32, kCovRows = 8192, kCovStep = 32;

__global__ void __launch_bounds__(256)
covariance_kernel(const float* __restrict__ X, int64_t n, int d, int ldx,
                  const double* __restrict__ mean, double* __restrict__ cov, int ntiles) {
    // decode the upper-triangular tile pair
    int t = blockIdx.x, ta = 0;
    while (t >= ntiles - ta) {
        t -= ntiles - ta;
        ++ta;
    }
    const int tb = ta + t;
    const int a0 = ta * kCovTile, b0 = tb * kCovTile;
    const int64_t r0 = int64_t(blockIdx.y) * kCovRows;
    const int64_t r1 = min(n, r0 + kCovRows);
    __shared__ double xa[kCovStep][kCovTile + 1];
    __shared__ double xb[kCovStep][kCovTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t r = r0; r < r1; r += kCovStep) {
        for (int e = threadIdx.x; e < kCovStep * kCovTile; e += 256) {
            const int rr = e / kCovTile, cc = e % kCovTile;
            const int64_t gr = r + rr;
            double va = 0.0, vb = 0.0;
            if (gr < r1) {
                if (a0 + cc < d) va = double(X[gr * ldx + a0 + cc]) - mean[a0 + cc];
                if (b0 + cc < d) vb = double(X[gr * ldx + b0 + cc]) - mean[b0 + cc];
            }
            xa[rr][cc] = va;
            xb[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kCovStep; ++rr) {
            const double u0 = xa[rr][ty * 2], u1 = xa[rr][ty * 2 + 1];
            const double v0 = xb[rr][tx * 2], v1 = xb[rr][tx * 2 + 1];
            acc[0][0] = fma(u0, v0, acc[0][0]);
            acc[0][1] = fma(u0, v1, acc[0][1]);
            acc[1][0] = fma(u1, v0, acc[1][0]);
            acc[1][1] = fma(u1, v1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int a = a0 + ty * 2 + i, b = b0 + tx * 2 + j;
            if (a < d && b < d) atomicAdd(&cov[int64_t(a) * d + b], acc[i][j]);
        }
}

cudaError_t launch_covariance(const float* X, int64_t n, int d, int ldx, const double* mean,
                              double* cov, cudaStream_t st) {
    const int ntiles = (d + kCovTile - 1) / kCovTile;
    const int npairs = ntiles * (ntiles + 1) / 2;
    dim3 grid(unsigned(npairs), unsigned((n + kCovRows - 1) / kCovRows));
    covariance_kernel<<<grid, 256, 0, st>>>(X, n, d, ldx, mean, cov, ntiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Lloyd k-means on all 2*N_s half-subspaces at once (Alg. 3 steps 6-8).
// Problem p = 2*i + h works on columns [i*s + off_h, i*s + off_h + len_h) of T.
// ---------------------------------------------------------------------------------------
constexpr int kKmThreads = 256;
constexpr int kKmPoints = 4096;   // points per CTA in the assignment pass

struct KmGeom {
    int Ns, s, h1, sk, Dp, hmax;
};

__device__ __forceinline__ void km_problem(const KmGeom& g, int p, int& col, int& len) {
    const int i = p >> 1, h = p & 1;
    col = i * g.s + (h ? g.h1 : 0);
    len = h ? g.s - g.h1 : g.h1;
}

// Assign every point to its nearest centroid (ties to the lowest id) and accumulate the
// per-centroid sums and counts of this CTA's points.
__global__ void __launch_bounds__(kKmThreads)
kmeans_assign_kernel(const float* __restrict__ T, int64_t n, KmGeom g,
                     const float* __restrict__ cent,   // [2Ns][sk][hmax]
                     uint16_t* __restrict__ assign,    // [2Ns][n]
                     double* __restrict__ sums,        // [2Ns][sk][hmax]
                     unsigned long long* __restrict__ counts,  // [2Ns][sk]
                     int accumulate) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int p = blockIdx.y;
    int col, len;
    km_problem(g, p, col, len);
    float* c_s = reinterpret_cast<float*>(sm);              // sk*hmax
    float* sum_s = c_s + g.sk * g.hmax;                     // sk*hmax (per-CTA partial sums)
    unsigned int* cnt_s = reinterpret_cast<unsigned int*>(sum_s + g.sk * g.hmax);  // sk
    const float* cp = cent + size_t(p) * g.sk * g.hmax;
    for (int e = threadIdx.x; e < g.sk * g.hmax; e += kKmThreads) {
        c_s[e] = cp[e];
        sum_s[e] = 0.f;
    }
    for (int e = threadIdx.x; e < g.sk; e += kKmThreads) cnt_s[e] = 0;
    __syncthreads();
    const int64_t p0 = int64_t(blockIdx.x) * kKmPoints;
    const int64_t p1 = min(n, p0 + kKmPoints);
    for (int64_t pt = p0 + threadIdx.x; pt < p1; pt += kKmThreads) {
        const float* x = T + pt * g.Dp + col;
        float xv[64];
        const int L = len < 64 ? len : 64;
        for (int j = 0; j < L; ++j) xv[j] = x[j];
        float best = 3.4e38f;
        int bi = 0;
        for (int c = 0; c < g.sk; ++c) {
            const float* cc = c_s + c * g.hmax;
            float acc = 0.f;
            for (int j = 0; j < L; ++j) {
                const float df = xv[j] - cc[j];
                acc = fmaf(df, df, acc);
            }
            for (int j = L; j < len; ++j) {
                const float df = x[j] - cc[j];
                acc = fmaf(df, df, acc);
            }
            if (acc < best) {
                best = acc;
                bi = c;
            }
        }
        assign[size_t(p) * n + pt] = uint16_t(bi);
        if (accumulate) {
            for (int j = 0; j < len; ++j) atomicAdd(&sum_s[bi * g.hmax + j], x[j]);
            atomicAdd(&cnt_s[bi], 1u);
        }
    }
    if (!accumulate) return;
    __syncthreads();
    double* sp = sums + size_t(p) * g.sk * g.hmax;
    for (int e = threadIdx.x; e < g.sk * g.hmax; e += kKmThreads) {
        if (sum_s[e] != 0.f) atomicAdd(&sp[e], double(sum_s[e]));
    }
    for (int e = threadIdx.x; e < g.sk; e += kKmThreads) {
        if (cnt_s[e]) atomicAdd(&counts[size_t(p) * g.sk + e], (unsigned long long)cnt_s[e]);
    }
}

// New centroid = mean of its points; an empty cluster keeps its centroid. Clears sums.
__global__ void kmeans_update_kernel(KmGeom g, float* __restrict__ cent,
                                     double* __restrict__ sums,
                                     unsigned long long* __restrict__ counts) {
    const int p = blockIdx.x;
    for (int e = threadIdx.x; e < g.sk * g.hmax; e += blockDim.x) {
        const int c = e / g.hmax;
        const unsigned long long m = counts[size_t(p) * g.sk + c];
        const size_t at = size_t(p) * g.sk * g.hmax + e;
        if (m > 0) cent[at] = float(sums[at] / double(m));
        sums[at] = 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < g.sk; c += blockDim.x) counts[size_t(p) * g.sk + c] = 0;
}

__global__ void kmeans_init_kernel(const float* __restrict__ T, KmGeom g,
                                   const int64_t* __restrict__ rows,  // [2Ns][sk]
                                   float* __restrict__ cent) {
    const int p = blockIdx.x;
    int col, len;
    km_problem(g, p, col, len);
    for (int e = threadIdx.x; e < g.sk * g.hmax; e += blockDim.x) {
        const int c = e / g.hmax, j = e % g.hmax;
        const int64_t r = rows[size_t(p) * g.sk + c];
        cent[size_t(p) * g.sk * g.hmax + e] = j < len ? T[r * g.Dp + col + j] : 0.f;
    }
}

__global__ void kmeans_codes_kernel(const uint16_t* __restrict__ assign, int64_t n, int Ns,
                                    int sk, uint16_t* __restrict__ codes) {
    const int i = blockIdx.y;
    for (int64_t pt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; pt < n;
         pt += int64_t(gridDim.x) * blockDim.x) {
        const int r = assign[size_t(2 * i) * n + pt];
        const int c = assign[size_t(2 * i + 1) * n + pt];
        codes[size_t(i) * n + pt] = uint16_t(r * sk + c);
    }
}

// Centroids gathered into the index layout [Ns][sk][s].
__global__ void kmeans_export_kernel(const float* __restrict__ cent, KmGeom g,
                                     float* __restrict__ out) {
    const int i = blockIdx.x;
    for (int e = threadIdx.x; e < g.sk * g.s; e += blockDim.x) {
        const int c = e / g.s, j = e % g.s;
        const int h = j >= g.h1;
        const int jj = h ? j - g.h1 : j;
        out[size_t(i) * g.sk * g.s + e] = cent[(size_t(2 * i + h) * g.sk + c) * g.hmax + jj];
    }
}

cudaError_t launch_kmeans(const float* T, int64_t n, int Dp, int Ns, int s, int h1, int sk,
                          int iters, const int64_t* init_rows_host, float* cent_out,
                          uint16_t* codes_out, cudaStream_t st) {
    KmGeom g{Ns, s, h1, sk, Dp, s - h1};
    const int P = 2 * Ns;
    float* cent = nullptr;
    double* sums = nullptr;
    unsigned long long* counts = nullptr;
    uint16_t* assign = nullptr;
    int64_t* rows = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t ncent = size_t(P) * sk * g.hmax;
    auto cleanup = [&]() {
        cudaFree(cent);
        cudaFree(sums);
        cudaFree(counts);
        cudaFree(assign);
        cudaFree(rows);
    };
#define KM_TRY(x)          \
    do {                   \
        e = (x);           \
        if (e != cudaSuccess) { \
            cleanup();     \
            return e;      \
        }                  \
    } while (0)
    KM_TRY(cudaMalloc(&cent, ncent * sizeof(float)));
    KM_TRY(cudaMalloc(&sums, ncent * sizeof(double)));
    KM_TRY(cudaMalloc(&counts, size_t(P) * sk * sizeof(unsigned long long)));
    KM_TRY(cudaMalloc(&assign, size_t(P) * n * sizeof(uint16_t)));
    KM_TRY(cudaMalloc(&rows, size_t(P) * sk * sizeof(int64_t)));
    KM_TRY(cudaMemcpyAsync(rows, init_rows_host, size_t(P) * sk * sizeof(int64_t),
                           cudaMemcpyHostToDevice, st));
    KM_TRY(cudaMemsetAsync(sums, 0, ncent * sizeof(double), st));
    KM_TRY(cudaMemsetAsync(counts, 0, size_t(P) * sk * sizeof(unsigned long long), st));
    kmeans_init_kernel<<<P, 256, 0, st>>>(T, g, rows, cent);
    KM_TRY(cudaGetLastError());
    const size_t smem = 2 * size_t(sk) * g.hmax * sizeof(float) + size_t(sk) * sizeof(unsigned);
    if (smem > 48 * 1024)
        KM_TRY(cudaFuncSetAttribute(kmeans_assign_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    dim3 grid(unsigned((n + kKmPoints - 1) / kKmPoints), unsigned(P));
    for (int it = 0; it < iters; ++it) {
        kmeans_assign_kernel<<<grid, kKmThreads, smem, st>>>(T, n, g, cent, assign, sums,
                                                              counts, 1);
        KM_TRY(cudaGetLastError());
        kmeans_update_kernel<<<P, 256, 0, st>>>(g, cent, sums, counts);
        KM_TRY(cudaGetLastError());
    }
    kmeans_assign_kernel<<<grid, kKmThreads, smem, st>>>(T, n, g, cent, assign, sums, counts, 0);
    KM_TRY(cudaGetLastError());
    dim3 cg(unsigned(std::min<int64_t>((n + 255) / 256, 4096)), unsigned(Ns));
    kmeans_codes_kernel<<<cg, 256, 0, st>>>(assign, n, Ns, sk, codes_out);
    KM_TRY(cudaGetLastError());
    kmeans_export_kernel<<<Ns, 256, 0, st>>>(cent, g, cent_out);
    KM_TRY(cudaGetLastError());
    KM_TRY(cudaStreamSynchronize(st));
    cleanup();
    return cudaSuccess;
#undef KM_TRY
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               size_t count) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += size_t(gridDim.x) * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, size_t count, cudaStream_t st) {
    const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 64);
    to_bf16_kernel<<<unsigned(blocks), 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

__global__ void center_kernel(const float* __restrict__ X, int64_t rows, int d, int64_t ldx,
                              const float* __restrict__ obar, float* __restrict__ Y) {
    const size_t total = size_t(rows) * d;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const size_t r = i / size_t(d);
        const int c = int(i - r * size_t(d));
        Y[i] = X[r * ldx + c] - obar[c];
    }
}

cudaError_t launch_center(const float* X, int64_t rows, int d, int64_t ldx, const float* obar, float* Y,
                          cudaStream_t st) {
    const size_t count = size_t(rows) * d;
    const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 64);
    if (blocks < 1) return cudaSuccess;
    center_kernel<<<unsigned(blocks), 256, 0, st>>>(X, rows, d, ldx, obar, Y);
    return cudaGetLastError();
}

// Column-wise max |Y| (FP8 scales). Non-negative floats order like their bit patterns.
__global__ void absmax_cols_kernel(const float* __restrict__ Y, int64_t rows, int Dp,
                                   unsigned* __restrict__ maxbits) {
    for (int c = threadIdx.x; c < Dp; c += blockDim.x) {
        float m = 0.f;
        for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) m = fmaxf(m, fabsf(Y[r * Dp + c]));
        atomicMax(&maxbits[c], __float_as_uint(m));
    }
}

cudaError_t launch_absmax_cols(const float* Y, int64_t rows, int Dp, unsigned* maxbits,
                               cudaStream_t st) {
    const int threads = Dp < 1024 ? ((Dp + 31) / 32) * 32 : 1024;
    const int64_t blocks = std::min<int64_t>(rows, 152 * 16);
    if (blocks < 1) return cudaSuccess;
    absmax_cols_kernel<<<unsigned(blocks), threads, 0, st>>>(Y, rows, Dp, maxbits);
    return cudaGetLastError();
}

// e4m3 rows, round to nearest with saturation to the finite range.
__global__ void quantize_fp8_kernel(const float* __restrict__ Y, int64_t rows, int Dp, int dp8,
                                    const float* __restrict__ inv_scale, uint8_t* __restrict__ out) {
    const size_t total = size_t(rows) * dp8;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += size_t(gridDim.x) * blockDim.x) {
        const size_t r = i / size_t(dp8);
        const int c = int(i - r * size_t(dp8));
        uint8_t v = 0;
        if (c < Dp) v = __nv_cvt_float_to_fp8(Y[r * Dp + c] * inv_scale[c], __NV_SATFINITE, __NV_E4M3);
        out[i] = v;
    }
}

cudaError_t launch_quantize_fp8(const float* Y, int64_t rows, int Dp, int dp8,
                                const float* inv_scale, uint8_t* out, cudaStream_t st) {
    const size_t count = size_t(rows) * dp8;
    const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 64);
    if (blocks < 1) return cudaSuccess;
    quantize_fp8_kernel<<<unsigned(blocks), 256, 0, st>>>(Y, rows, Dp, dp8, inv_scale, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Cell lists of Alg. 3 (IMI[cell].append(j) for j = 0..n-1, so ids ascend in every cell),
// built on the device as a stable counting sort of the point ids by cell code, one slab of
// 2^15 ids at a time: per (subspace, slab) the cells' counts, then per cell the running
// position of each slab in the cell's list (which is the slab table), then a stable scatter
// of every slab in id order. Each cell's list starts on a multiple of 4 ids and is padded
// with kIdPad (the caller fills the array with it first).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512)
lists_count_kernel(const uint16_t* __restrict__ codes, int64_t n, int K, int n_slabs,
                   uint32_t* __restrict__ counts) {
    extern __shared__ uint32_t h[];
    const int t = blockIdx.x, i = blockIdx.y;
    for (int c = threadIdx.x; c < K; c += blockDim.x) h[c] = 0u;
    __syncthreads();
    const int64_t lo = int64_t(t) << kSlabLog2, hi = min(lo + kSlabIds, n);
    const uint16_t* ci = codes + size_t(i) * n;
    for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) atomicAdd(&h[ci[p]], 1u);
    __syncthreads();
    uint32_t* out = counts + (size_t(i) * n_slabs + t) * K;
    for (int c = threadIdx.x; c < K; c += blockDim.x) out[c] = h[c];
}

// sizes[j] = sum over slabs of counts, j = i * K + c (one thread per cell).
__global__ void lists_size_kernel(const uint32_t* __restrict__ counts, int K, int n_slabs, int Ns,
                                  uint32_t* __restrict__ sizes) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= int64_t(Ns) * K) return;
    const int i = int(j / K), c = int(j - int64_t(i) * K);
    uint32_t s = 0;
    for (int t = 0; t < n_slabs; ++t) s += counts[(size_t(i) * n_slabs + t) * K + c];
    sizes[j] = s;
}

// start[j] = sum over j' < j of the padded sizes (sizes rounded up to 4), start[m] = total;
// one block, each thread a contiguous segment of the m cells.
__global__ void __launch_bounds__(1024)
lists_start_kernel(const uint32_t* __restrict__ sizes, int64_t m, uint32_t* __restrict__ start) {
    __shared__ uint32_t part[1024];
    const int tid = threadIdx.x;
    const int64_t seg = (m + 1023) / 1024;
    const int64_t a = min(m, int64_t(tid) * seg), b = min(m, a + seg);
    uint32_t s = 0;
    for (int64_t j = a; j < b; ++j) s += (sizes[j] + 3u) & ~3u;
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // inclusive scan of the segment sums
        const uint32_t v = tid >= off ? part[tid - off] : 0u;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint32_t run = part[tid] - s;
    for (int64_t j = a; j < b; ++j) {
        start[j] = run;
        run += (sizes[j] + 3u) & ~3u;
    }
    if (tid == 1023) start[m] = part[1023];
}

// Per cell, the position in the id array where each slab's ids begin: split[j][t], and the
// end of the cell's ids split[j][n_slabs]; counts is overwritten with the same positions
// (the scatter's starting points). One thread per cell.
__global__ void lists_split_kernel(uint32_t* __restrict__ counts, const uint32_t* __restrict__ start, int K,
                                   int n_slabs, int Ns, uint32_t* __restrict__ split) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= int64_t(Ns) * K) return;
    const int i = int(j / K), c = int(j - int64_t(i) * K);
    uint32_t run = start[j];
    uint32_t* sp = split + size_t(j) * (n_slabs + 1);
    for (int t = 0; t < n_slabs; ++t) {
        uint32_t& ct = counts[(size_t(i) * n_slabs + t) * K + c];
        const uint32_t v = ct;
        sp[t] = run;
        ct = run;
        run += v;
    }
    sp[n_slabs] = run;
}

// Stable scatter of slab t of subspace i: one warp walks the slab's ids in order, 32 at a
// time; lanes with equal codes are ranked by lane (ids ascend with the lane) and the group's
// lowest lane advances the cell's position.
__global__ void __launch_bounds__(32)
lists_scatter_kernel(const uint16_t* __restrict__ codes, int64_t n, int K, int n_slabs,
                     const uint32_t* __restrict__ pos0, uint32_t* __restrict__ ids) {
    extern __shared__ uint32_t pos[];
    const int t = blockIdx.x, i = blockIdx.y, lane = threadIdx.x;
    const uint32_t* src = pos0 + (size_t(i) * n_slabs + t) * K;
    for (int c = lane; c < K; c += 32) pos[c] = src[c];
    __syncwarp();
    const int64_t lo = int64_t(t) << kSlabLog2, hi = min(lo + kSlabIds, n);
    const uint16_t* ci = codes + size_t(i) * n;
    const uint32_t lane_lt = (1u << lane) - 1u;
    for (int64_t p0 = lo; p0 < hi; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool ok = p < hi;
        const uint32_t c = ok ? uint32_t(ci[p]) : 0x10000u + uint32_t(lane);   // past the end: alone
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        if (ok) {
            const uint32_t at = pos[c] + __popc(grp & lane_lt);
            ids[at] = uint32_t(p);
        }
        __syncwarp();
        if (ok && (grp & lane_lt) == 0u) pos[c] += __popc(grp);
        __syncwarp();
    }
}

int64_t lists_scratch_words(int64_t n, int Ns, int K) {
    const int64_t n_slabs = (n + kSlabIds - 1) / kSlabIds;
    return int64_t(Ns) * n_slabs * K + int64_t(Ns) * K + 1;
}

cudaError_t launch_build_lists(const uint16_t* codes, int64_t n, int Ns, int K, uint32_t* scratch,
                               uint32_t* sizes, uint32_t* start, uint32_t* split, uint32_t* ids,
                               cudaStream_t st) {
    const int n_slabs = int((n + kSlabIds - 1) / kSlabIds);
    uint32_t* counts = scratch;   // [Ns][n_slabs][K]
    const size_t smem = size_t(K) * 4;
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(lists_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(lists_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    const dim3 grid{unsigned(n_slabs), unsigned(Ns), 1u};
    lists_count_kernel<<<grid, 512, smem, st>>>(codes, n, K, n_slabs, counts);
    const int64_t m = int64_t(Ns) * K;
    const unsigned cb = unsigned((m + 255) / 256);
    lists_size_kernel<<<cb, 256, 0, st>>>(counts, K, n_slabs, Ns, sizes);
    lists_start_kernel<<<1, 1024, 0, st>>>(sizes, m, start);
    lists_split_kernel<<<cb, 256, 0, st>>>(counts, start, K, n_slabs, Ns, split);
    lists_scatter_kernel<<<grid, 32, smem, st>>>(codes, n, K, n_slabs, counts, ids);
    return cudaGetLastError();
}

}  // namespace taco

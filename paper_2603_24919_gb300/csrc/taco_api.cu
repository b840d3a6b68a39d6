// C ABI entry points (include/taco.h): index build and import (Alg. 1-3), search (Alg. 6),
// export, persistence.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "taco_internal.h"

using namespace taco;

int taco::ensure_device_codes(taco_index* ix) {
    if (ix->d_codes) return TACO_OK;
    uint16_t* d = nullptr;
    TACO_CUDA(cudaMalloc(&d, ix->codes.size() * sizeof(uint16_t)));
    const cudaError_t e = cudaMemcpy(d, ix->codes.data(), ix->codes.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cell codes upload", __FILE__, __LINE__);
    }
    ix->d_codes = d;
    ix->device_bytes += int64_t(ix->codes.size() * sizeof(uint16_t));
    return TACO_OK;
}

namespace {

template <typename T>
int dev_alloc(T** p, size_t count, int64_t* acct) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    if (acct) *acct += int64_t(count * sizeof(T));
    return TACO_OK;
}

#define TRY(x)                   \
    do {                         \
        int rc_ = (x);           \
        if (rc_ != TACO_OK) return rc_; \
    } while (0)

void free_device(taco_index* ix) {
    cudaFree(ix->d_data);
    cudaFree(ix->d_data_bf16);
    cudaFree(ix->d_data_fp8);
    cudaFree(ix->d_fp8_scale);
    cudaFree(ix->d_cent_tc);
    cudaFree(ix->d_cent_tc_norm);
    cudaFree(ix->d_cent_tc8);
    cudaFree(ix->d_cent_tc8_norm);
    cudaFree(ix->d_cent_tc8_scale);
    cudaFree(ix->d_status);
    cudaFree(ix->d_codes);
    cudaFree(ix->d_obar);
    cudaFree(ix->d_B);
    cudaFree(ix->d_cent);
    cudaFree(ix->d_sizes);
    cudaFree(ix->d_ids);
    cudaFree(ix->d_split);
    cudaFree(ix->ws.base);
    if (ix->ws.host_pinned) cudaFreeHost(ix->ws.host_pinned);
}

struct IndexDeleter {
    void operator()(taco_index* ix) const {
        if (ix) {
            for (cudaEvent_t e : ix->prof.pool) cudaEventDestroy(e);
            free_device(ix);
            delete ix;
        }
    }
};
using IndexPtr = std::unique_ptr<taco_index, IndexDeleter>;

int check_geometry(int64_t n, int d, int Ns, int s, int sk) {
    if (n < 1 || n > int64_t(0x7fffffff)) return fail(TACO_EINVAL, "n = %lld out of range", (long long)n);
    if (d < 1 || d > 65536) return fail(TACO_EINVAL, "d = %d out of range", d);
    if (Ns < 1 || Ns > TACO_MAX_SUBSPACES)
        return fail(TACO_EINVAL, "n_subspaces = %d must be in [1, %d]", Ns, TACO_MAX_SUBSPACES);
    if (s < 2) return fail(TACO_EINVAL, "sub_dim = %d must be >= 2", s);
    if (int64_t(Ns) * s > d) return fail(TACO_EINVAL, "n_subspaces * sub_dim > d");
    if (sk < 1 || sk > TACO_MAX_SQRT_K)
        return fail(TACO_EINVAL, "sqrt_k = %d must be in [1, %d]", sk, TACO_MAX_SQRT_K);
    // the padded cell lists of all subspaces (at most 3 pad ids per cell) take 32-bit offsets
    if (int64_t(Ns) * (n + 3 * int64_t(sk) * sk) >= (int64_t(1) << 32))
        return fail(TACO_ECAPACITY, "n_subspaces * (n + 3 K) must be below 2^32 (32-bit id-list offsets)");
    return TACO_OK;
}

// Copy D (host or device, [n][d]) into the padded device layout [n][d_pad].
int upload_data(taco_index* ix, const float* data, cudaStream_t st) {
    TRY(dev_alloc(&ix->d_data, size_t(ix->n) * ix->d_pad, &ix->device_bytes));
    if (ix->d_pad != ix->d)
        TACO_CUDA(cudaMemsetAsync(ix->d_data, 0, size_t(ix->n) * ix->d_pad * sizeof(float), st));
    const cudaMemcpyKind kind = is_device_pointer(data) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TACO_CUDA(cudaMemcpy2DAsync(ix->d_data, size_t(ix->d_pad) * sizeof(float), data,
                                size_t(ix->d) * sizeof(float), size_t(ix->d) * sizeof(float),
                                size_t(ix->n), kind, st));
    return TACO_OK;
}

void set_geometry(taco_index* ix, int64_t n, int d, int Ns, int s, int sk) {
    ix->n = n;
    ix->d = d;
    ix->d_pad = (d + 7) & ~7;
    ix->Ns = Ns;
    ix->s = s;
    ix->sk = sk;
    ix->K = sk * sk;
    ix->Dp = Ns * s;
    ix->h1 = s / 2;
}

// Device copy of the cell codes, for the codes fallback of flagged queries.
int enable_codes_fallback(taco_index* ix) {
    TRY(taco::ensure_device_codes(ix));
    ix->codes_fallback = true;
    return TACO_OK;
}

// FP8-e4m3 rows with one scale per block of 16 dimensions (the block's largest |coordinate|
// over all points / 448; a block is one 16-byte chunk of a row, so the select pass applies
// one scale per chunk). When N_s * s = d the rows are the transformed points B^T (o - o_bar)
// (distances are preserved, Lemma 1); otherwise the transform drops dimensions, so the rows
// are the centred points o - o_bar. Two passes over chunks of points: scales, then
// quantisation.
int build_fp8_rows(taco_index* ix, cudaStream_t st) {
    const int64_t n = ix->n;
    const bool transformed = ix->Dp == ix->d;
    const int cols = transformed ? ix->Dp : ix->d;   // FP8 coordinates per point
    ix->fp8_space = transformed ? 0 : 1;
    // row pitch: a power of two up to 64 bytes, else whole 128-byte lines, so that a row's
    // gather reads only lines of its own (the pad bytes are E4M3 zeros with scale 0)
    ix->dp8 = (cols + 15) & ~15;
    if (ix->dp8 <= 64) {
        while (ix->dp8 & (ix->dp8 - 1)) ix->dp8 += 16;
    } else {
        ix->dp8 = (ix->dp8 + 127) & ~127;
    }
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t(256) << 20) / (int64_t(cols) * 4)));
    float* tmp = nullptr;
    unsigned* maxbits = nullptr;
    TACO_CUDA(cudaMalloc(&tmp, size_t(chunk) * cols * 4));
    struct Free {
        void* a;
        void* b;
        ~Free() {
            cudaFree(a);
            cudaFree(b);
        }
    } guard{tmp, nullptr};
    TACO_CUDA(cudaMalloc(&maxbits, size_t(cols) * 4));
    guard.b = maxbits;
    TACO_CUDA(cudaMemsetAsync(maxbits, 0, size_t(cols) * 4, st));
    auto coords = [&](int64_t c0, int64_t cn) -> cudaError_t {   // the chunk's coordinates into tmp
        if (transformed)
            return launch_project(ix->d_data + c0 * ix->d_pad, cn, ix->d, ix->d_pad, ix->d_obar, ix->d_B, cols, tmp, st);
        return launch_center(ix->d_data + c0 * ix->d_pad, cn, ix->d, ix->d_pad, ix->d_obar, tmp, st);
    };
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t cn = std::min(chunk, n - c0);
        TACO_CUDA(coords(c0, cn));
        TACO_CUDA(launch_absmax_cols(tmp, cn, cols, maxbits, st));
    }
    std::vector<unsigned> mb(cols);
    TACO_CUDA(cudaMemcpyAsync(mb.data(), maxbits, size_t(cols) * 4, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    std::vector<float> sc(size_t(2) * ix->dp8, 0.f);   // [scale | 1/scale]
    const int group = 16;
    for (int g0 = 0; g0 < cols; g0 += group) {
        const int g1 = std::min(cols, g0 + group);
        float m = 0.f;
        for (int c = g0; c < g1; ++c) {
            float v;
            std::memcpy(&v, &mb[c], 4);
            m = std::max(m, v);
        }
        const float scale = m > 0.f ? m / 448.f : 1.f;
        for (int c = g0; c < g1; ++c) {
            sc[c] = scale;
            sc[ix->dp8 + c] = 1.f / scale;
        }
    }
    TRY(dev_alloc(&ix->d_fp8_scale, sc.size(), &ix->device_bytes));
    TACO_CUDA(cudaMemcpyAsync(ix->d_fp8_scale, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice, st));
    TRY(dev_alloc(&ix->d_data_fp8, size_t(n) * ix->dp8, &ix->device_bytes));
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t cn = std::min(chunk, n - c0);
        TACO_CUDA(coords(c0, cn));
        TACO_CUDA(launch_quantize_fp8(tmp, cn, cols, ix->dp8, ix->d_fp8_scale + ix->dp8,
                                      ix->d_data_fp8 + size_t(c0) * ix->dp8, st));
    }
    TACO_CUDA(cudaStreamSynchronize(st));   // sc dies on return; tmp is freed after the kernels
    return TACO_OK;
}

int finish_index(taco_index* ix, int keep_rows, cudaStream_t st, const uint16_t* dcodes = nullptr) {
    const int64_t n = ix->n;
    const int Ns = ix->Ns, K = ix->K;
    TRY(configure_search(ix));
    const int ns1 = ix->n_slabs + 1;
    // Cell lists of all subspaces in one array, built on the device (launch_build_lists):
    // subspace after subspace, cell after cell, ids ascending, each list starting on a
    // 16-byte boundary (a multiple of 4 ids) and padded to the next one with kIdPad, so the
    // counting walk reads any run of a list in aligned 4-id chunks. The slab table holds
    // absolute positions in that array.
    const uint16_t* dc = dcodes;
    uint16_t* tmp_codes = nullptr;
    uint32_t* scratch = nullptr;
    uint32_t* dstart = nullptr;
    struct Tmp {
        uint16_t** c;
        uint32_t** s;
        uint32_t** t;
        ~Tmp() {
            cudaFree(*c);
            cudaFree(*s);
            cudaFree(*t);
        }
    } tmp{&tmp_codes, &scratch, &dstart};
    for (size_t j = 0; j < ix->codes.size(); ++j)
        if (ix->codes[j] >= K)
            return fail(TACO_EINVAL, "code %d of point %lld >= K", int(ix->codes[j]), (long long)(j % size_t(n)));
    if (!dc) {
        TRY(dev_alloc(&tmp_codes, ix->codes.size(), nullptr));
        TACO_CUDA(cudaMemcpyAsync(tmp_codes, ix->codes.data(), ix->codes.size() * 2, cudaMemcpyHostToDevice, st));
        dc = tmp_codes;
    }
    const size_t m = size_t(Ns) * K;
    const size_t ids_cap = size_t(Ns) * size_t(n) + 3 * m;   // every list padded by at most 3
    TRY(dev_alloc(&scratch, size_t(lists_scratch_words(n, Ns, K)), nullptr));
    TRY(dev_alloc(&dstart, m + 1, nullptr));
    TRY(dev_alloc(&ix->d_sizes, m, &ix->device_bytes));
    TRY(dev_alloc(&ix->d_ids, ids_cap, &ix->device_bytes));
    TRY(dev_alloc(&ix->d_split, m * ns1, &ix->device_bytes));
    TACO_CUDA(cudaMemsetAsync(ix->d_ids, 0xff, ids_cap * 4, st));   // kIdPad
    TACO_CUDA(launch_build_lists(dc, n, Ns, K, scratch, ix->d_sizes, dstart, ix->d_split, ix->d_ids, st));
    uint32_t total = 0;
    TACO_CUDA(cudaMemcpyAsync(&total, dstart + m, 4, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    ix->n_ids = int64_t(total);
    // FP32 copies of o_bar, B, centroids for the query path
    std::vector<float> ob(ix->d), Bf(size_t(ix->d) * ix->Dp), cf(ix->centroids.size());
    for (int j = 0; j < ix->d; ++j) ob[j] = float(ix->o_bar[j]);
    for (size_t j = 0; j < Bf.size(); ++j) Bf[j] = float(ix->B[j]);
    for (size_t j = 0; j < cf.size(); ++j) cf[j] = float(ix->centroids[j]);
    if (!ix->d_obar) TRY(dev_alloc(&ix->d_obar, ob.size(), &ix->device_bytes));
    if (!ix->d_B) TRY(dev_alloc(&ix->d_B, Bf.size(), &ix->device_bytes));
    if (!ix->d_cent) TRY(dev_alloc(&ix->d_cent, cf.size(), &ix->device_bytes));
    TACO_CUDA(cudaMemcpyAsync(ix->d_obar, ob.data(), ob.size() * 4, cudaMemcpyHostToDevice, st));
    TACO_CUDA(cudaMemcpyAsync(ix->d_B, Bf.data(), Bf.size() * 4, cudaMemcpyHostToDevice, st));
    TACO_CUDA(cudaMemcpyAsync(ix->d_cent, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice, st));
    if (keep_rows & ~(TACO_ROWS_BF16 | TACO_ROWS_FP8)) return fail(TACO_EINVAL, "unknown keep_rows bits 0x%x", keep_rows);
    if (keep_rows & TACO_ROWS_BF16) {
        TRY(dev_alloc(&ix->d_data_bf16, size_t(n) * ix->d_pad, &ix->device_bytes));
        TACO_CUDA(launch_to_bf16(ix->d_data, ix->d_data_bf16, size_t(n) * ix->d_pad, st));
    }
    if (keep_rows & TACO_ROWS_FP8) TRY(build_fp8_rows(ix, st));
    if (!ix->d_status) {
        TRY(dev_alloc(&ix->d_status, 1, &ix->device_bytes));
        TACO_CUDA(cudaMemsetAsync(ix->d_status, 0, sizeof(int), st));
    }
    TACO_CUDA(cudaStreamSynchronize(st));
    TRY(build_centroid_tc(ix));
    if (ix->cluster == 0) TRY(enable_codes_fallback(ix));   // no cluster layout fits this n
    TACO_CUDA(cudaStreamSynchronize(st));  // host vectors above die on return
    return TACO_OK;
}

// splitmix64 (Steele, Lea, Flood: "Fast splittable pseudorandom number generators").
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// sqrt_k distinct rows by a partial Fisher-Yates shuffle (k-means initial centroids).
void pick_rows(int64_t n, int k, uint64_t seed, int64_t* out) {
    uint64_t st = seed;
    if (n <= 4 * int64_t(k) + 16) {
        std::vector<int64_t> perm(n);
        std::iota(perm.begin(), perm.end(), 0);
        for (int j = 0; j < k && j < n; ++j) {
            const int64_t r = j + int64_t(splitmix64(st) % uint64_t(n - j));
            std::swap(perm[j], perm[r]);
            out[j] = perm[j];
        }
        for (int j = int(std::min<int64_t>(k, n)); j < k; ++j) out[j] = out[j % std::max<int64_t>(n, 1)];
        return;
    }
    // sparse Fisher-Yates: swaps recorded in a small map
    std::vector<std::pair<int64_t, int64_t>> swaps;
    auto get = [&](int64_t p) {
        for (auto& s : swaps)
            if (s.first == p) return s.second;
        return p;
    };
    auto set = [&](int64_t p, int64_t v) {
        for (auto& s : swaps)
            if (s.first == p) {
                s.second = v;
                return;
            }
        swaps.push_back({p, v});
    };
    for (int j = 0; j < k; ++j) {
        const int64_t r = j + int64_t(splitmix64(st) % uint64_t(n - j));
        const int64_t vj = get(j), vr = get(r);
        set(j, vr);
        set(r, vj);
        out[j] = vr;
    }
}

int build_impl(const float* data, int64_t n, int32_t d, const taco_build_params* p, cudaStream_t st,
               taco_index** out) {
    if (!data || !p || !out) return fail(TACO_EINVAL, "null argument");
    *out = nullptr;
    if (p->reserved != 0) return fail(TACO_EINVAL, "reserved field must be 0");
    TRY(check_geometry(n, d, p->n_subspaces, p->sub_dim, p->sqrt_k));
    if (n < 2) return fail(TACO_EINVAL, "the covariance needs n >= 2");
    if (p->kmeans_iters < 0) return fail(TACO_EINVAL, "kmeans_iters < 0");
    if (n < p->sqrt_k) return fail(TACO_EINVAL, "n < sqrt_k");
    IndexPtr ix(new (std::nothrow) taco_index());
    if (!ix) return fail(TACO_ENOMEM, "host allocation failed");
    TACO_CUDA(cudaGetDevice(&ix->device));
    set_geometry(ix.get(), n, d, p->n_subspaces, p->sub_dim, p->sqrt_k);
    TRY(upload_data(ix.get(), data, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    // Alg. 1 steps 2-3: mean and covariance, FP64 accumulation on the device
    double* dsum = nullptr;
    double* dcov = nullptr;
    TRY(dev_alloc(&dsum, size_t(d), nullptr));
    std::unique_ptr<double, void (*)(double*)> g1(dsum, [](double* q) { cudaFree(q); });
    TRY(dev_alloc(&dcov, size_t(d) * d, nullptr));
    std::unique_ptr<double, void (*)(double*)> g2(dcov, [](double* q) { cudaFree(q); });
    TACO_CUDA(cudaMemsetAsync(dsum, 0, size_t(d) * 8, st));
    TACO_CUDA(cudaMemsetAsync(dcov, 0, size_t(d) * d * 8, st));
    TACO_CUDA(launch_col_mean(ix->d_data, n, d, ix->d_pad, dsum, st));
    std::vector<double> mean(d);
    TACO_CUDA(cudaMemcpyAsync(mean.data(), dsum, size_t(d) * 8, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    for (double& v : mean) v /= double(n);
    TACO_CUDA(cudaMemcpyAsync(dsum, mean.data(), size_t(d) * 8, cudaMemcpyHostToDevice, st));
    TACO_CUDA(launch_covariance(ix->d_data, n, d, ix->d_pad, dsum, dcov, st));
    std::vector<double> cov(size_t(d) * d);
    TACO_CUDA(cudaMemcpyAsync(cov.data(), dcov, cov.size() * 8, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b) {
            const double v = cov[size_t(a) * d + b] / double(n - 1);
            cov[size_t(a) * d + b] = v;
            cov[size_t(b) * d + a] = v;
        }
    // Alg. 1 step 4 and Alg. 2 (host, FP64)
    std::vector<double> vecs, vals;
    symmetric_eigen(d, cov, vecs, vals);
    std::vector<std::vector<int>> buckets;
    eigensystem_allocation(vals, p->n_subspaces, p->sub_dim, buckets);
    std::vector<int> desc(d);
    std::iota(desc.begin(), desc.end(), 0);
    std::stable_sort(desc.begin(), desc.end(), [&](int x, int y) { return vals[x] > vals[y]; });
    std::vector<int> rank_of(d);
    for (int r = 0; r < d; ++r) rank_of[desc[r]] = r;
    const int Dp = ix->Dp;
    ix->o_bar = mean;
    ix->B.assign(size_t(d) * Dp, 0.0);
    ix->alloc.assign(Dp, -1);
    int col = 0;
    for (auto& b : buckets)
        for (int e : b) {
            for (int a = 0; a < d; ++a) ix->B[size_t(a) * Dp + col] = vecs[size_t(a) * d + e];
            ix->alloc[col] = rank_of[e];
            ++col;
        }
    ix->eigvals.resize(d);
    for (int r = 0; r < d; ++r) ix->eigvals[r] = vals[desc[r]];
    // Alg. 1 steps 6-11: T = (D - o_bar) B on the device
    std::vector<float> ob(d), Bf(size_t(d) * Dp);
    for (int j = 0; j < d; ++j) ob[j] = float(mean[j]);
    for (size_t j = 0; j < Bf.size(); ++j) Bf[j] = float(ix->B[j]);
    TRY(dev_alloc(&ix->d_obar, size_t(d), &ix->device_bytes));
    TRY(dev_alloc(&ix->d_B, Bf.size(), &ix->device_bytes));
    TACO_CUDA(cudaMemcpyAsync(ix->d_obar, ob.data(), ob.size() * 4, cudaMemcpyHostToDevice, st));
    TACO_CUDA(cudaMemcpyAsync(ix->d_B, Bf.data(), Bf.size() * 4, cudaMemcpyHostToDevice, st));
    float* dT = nullptr;
    TRY(dev_alloc(&dT, size_t(n) * Dp, nullptr));
    std::unique_ptr<float, void (*)(float*)> g3(dT, [](float* q) { cudaFree(q); });
    TACO_CUDA(launch_project(ix->d_data, n, d, ix->d_pad, ix->d_obar, ix->d_B, Dp, dT, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    const auto t1 = std::chrono::steady_clock::now();
    // Alg. 3 steps 4-9: k-means on both halves of every subspace
    const int P = 2 * p->n_subspaces;
    std::vector<int64_t> init(size_t(P) * p->sqrt_k);
    for (int pr = 0; pr < P; ++pr)
        pick_rows(n, p->sqrt_k, p->seed * 0x100000001b3ull + uint64_t(pr) + 1, init.data() + size_t(pr) * p->sqrt_k);
    float* dcent = nullptr;
    uint16_t* dcodes = nullptr;
    TRY(dev_alloc(&dcent, size_t(p->n_subspaces) * p->sqrt_k * p->sub_dim, nullptr));
    std::unique_ptr<float, void (*)(float*)> g4(dcent, [](float* q) { cudaFree(q); });
    TRY(dev_alloc(&dcodes, size_t(p->n_subspaces) * n, nullptr));
    std::unique_ptr<uint16_t, void (*)(uint16_t*)> g5(dcodes, [](uint16_t* q) { cudaFree(q); });
    TACO_CUDA(launch_kmeans(dT, n, Dp, p->n_subspaces, p->sub_dim, ix->h1, p->sqrt_k, p->kmeans_iters,
                            init.data(), dcent, dcodes, st));
    std::vector<float> cent(size_t(p->n_subspaces) * p->sqrt_k * p->sub_dim);
    ix->codes.resize(size_t(p->n_subspaces) * n);
    TACO_CUDA(cudaMemcpyAsync(cent.data(), dcent, cent.size() * 4, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaMemcpyAsync(ix->codes.data(), dcodes, ix->codes.size() * 2, cudaMemcpyDeviceToHost, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    ix->centroids.assign(cent.begin(), cent.end());
    TRY(finish_index(ix.get(), p->keep_rows, st, dcodes));
    const auto t2 = std::chrono::steady_clock::now();
    ix->build_ms_transform = std::chrono::duration<double, std::milli>(t1 - t0).count();
    ix->build_ms_index = std::chrono::duration<double, std::milli>(t2 - t1).count();
    *out = ix.release();
    return TACO_OK;
}

int create_impl(const float* data, int64_t n, int32_t d, const taco_index_parts* parts, int keep_rows,
                cudaStream_t st, taco_index** out) {
    if (!data || !parts || !out || !parts->o_bar || !parts->B || !parts->centroids || !parts->codes)
        return fail(TACO_EINVAL, "null argument");
    *out = nullptr;
    if (parts->reserved != 0) return fail(TACO_EINVAL, "reserved field must be 0");
    TRY(check_geometry(n, d, parts->n_subspaces, parts->sub_dim, parts->sqrt_k));
    IndexPtr ix(new (std::nothrow) taco_index());
    if (!ix) return fail(TACO_ENOMEM, "host allocation failed");
    TACO_CUDA(cudaGetDevice(&ix->device));
    set_geometry(ix.get(), n, d, parts->n_subspaces, parts->sub_dim, parts->sqrt_k);
    ix->o_bar.assign(parts->o_bar, parts->o_bar + d);
    ix->B.assign(parts->B, parts->B + size_t(d) * ix->Dp);
    ix->centroids.assign(parts->centroids, parts->centroids + size_t(ix->Ns) * ix->sk * ix->s);
    ix->codes.assign(parts->codes, parts->codes + size_t(ix->Ns) * n);
    ix->eigvals.assign(d, 0.0);
    ix->alloc.assign(ix->Dp, -1);
    TRY(upload_data(ix.get(), data, st));
    TACO_CUDA(cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    TRY(finish_index(ix.get(), keep_rows, st));
    ix->build_ms_index = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = ix.release();
    return TACO_OK;
}

int ensure_workspace(taco_index* ix, size_t bytes, size_t host_bytes) {
    if (bytes > ix->ws.bytes) {
        cudaFree(ix->ws.base);
        ix->ws.base = nullptr;
        ix->ws.bytes = 0;
        TACO_CUDA(cudaMalloc(&ix->ws.base, bytes));
        ix->ws.bytes = bytes;
    }
    if (host_bytes > ix->ws.host_bytes) {
        if (ix->ws.host_pinned) cudaFreeHost(ix->ws.host_pinned);
        ix->ws.host_pinned = nullptr;
        ix->ws.host_bytes = 0;
        TACO_CUDA(cudaMallocHost(&ix->ws.host_pinned, host_bytes));
        ix->ws.host_bytes = host_bytes;
    }
    return TACO_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int taco::check_query_params(const taco_query_params& q, int k_stride) {
    if (q.k < 1 || q.k > k_stride) return fail(TACO_EINVAL, "k = %d must be in [1, k_stride = %d]", q.k, k_stride);
    if (q.k > TACO_MAX_K) return fail(TACO_ECAPACITY, "k = %d exceeds %d", q.k, TACO_MAX_K);
    if (q.budget < 1) return fail(TACO_EINVAL, "budget must be >= 1");
    if (q.rerank_target < 0) return fail(TACO_EINVAL, "rerank_target must be >= 0");
    if (q.select_rule != TACO_SELECT_LITERAL && q.select_rule != TACO_SELECT_PROSE)
        return fail(TACO_EINVAL, "unknown select_rule %d", q.select_rule);
    if (q.precision != TACO_PREC_FP32 && q.precision != TACO_PREC_BF16 && q.precision != TACO_PREC_FP8)
        return fail(TACO_EINVAL, "unknown precision %d", q.precision);
    if (q.precision != TACO_PREC_FP32 && q.shortlist_mult < 1)
        return fail(TACO_EINVAL, "shortlist_mult must be >= 1 for BF16 and FP8");
    if (q.probe_precision != TACO_PREC_FP32 && q.probe_precision != TACO_PREC_BF16 &&
        q.probe_precision != TACO_PREC_FP8)
        return fail(TACO_EINVAL, "probe_precision must be TACO_PREC_FP32, TACO_PREC_BF16 or TACO_PREC_FP8");
    if (q.reserved != 0) return fail(TACO_EINVAL, "reserved field must be 0");
    return TACO_OK;
}

int taco::query_list_len(const taco_query_params& q) {
    if (q.precision == TACO_PREC_BF16 || q.precision == TACO_PREC_FP8) {
        const int64_t m = int64_t(q.k) * q.shortlist_mult;
        return int(std::min<int64_t>(std::max<int64_t>(m, q.k), TACO_MAX_K));
    }
    return q.k;
}

QueryParamsDev taco::query_params_dev(const taco_query_params& q) {
    QueryParamsDev r;
    r.k = q.k;
    r.select_rule = q.select_rule;
    r.budget = q.budget;
    r.rerank_target = q.rerank_target;
    r.kk = query_list_len(q);
    r.pad = 0;
    return r;
}

SearchLayout taco::plan_search(const taco_index* ix, int64_t chunk, int kk_max, int64_t n_params,
                               bool stage_queries, bool stage_ids, bool stage_dists, int k_stride,
                               bool centroid_tc) {
    const int Ns = ix->Ns, K = ix->K;
    SearchLayout l;
    size_t off = 0;
    l.qt = off; off = align_up(off + size_t(chunk) * ix->Dp * 4);
    l.cells = off; off = align_up(off + size_t(chunk) * Ns * K * 2);
    l.nc = off; off = align_up(off + size_t(chunk) * Ns * 4);
    l.ret = off; off = align_up(off + size_t(chunk) * Ns * 8);
    const size_t lists = size_t(chunk) * ix->cluster * kListsPerCta * kk_max * 4;
    l.ld = off; off = align_up(off + lists);
    l.li = off; off = align_up(off + lists);
    // two-pass form: per-unit level counts and lists (a fixed arena slot of kArenaPerSlab
    // ids per slab of the unit's range; units that do not fit send their query to the
    // cluster kernel)
    const size_t units = size_t(chunk) * ix->tp_ranges;
    l.uge = off; off = align_up(off + units * 16 * 4);
    l.uoff = off; off = align_up(off + units * 4);
    l.ulen = off; off = align_up(off + units * 4);
    l.arena = off; off = align_up(off + units * kArenaPerSlab * ix->tp_spc * 4);
    l.qflag = off; off = align_up(off + size_t(chunk + 2) * 4);   // flags, then 2 query counters
    l.qlast = off; off = align_up(off + size_t(chunk) * 4);
    l.par = off; off = align_up(off + size_t(n_params) * sizeof(QueryParamsDev));
    l.q = off; off = align_up(off + (stage_queries ? size_t(chunk) * ix->d * 4 : 0));
    l.oi = off; off = align_up(off + (stage_ids ? size_t(chunk) * k_stride * 8 : 0));
    l.od = off; off = align_up(off + (stage_dists ? size_t(chunk) * k_stride * 4 : 0));
    l.hd = off; off = align_up(off + (centroid_tc ? size_t(chunk) * ix->Ns * 2 * ix->sk * 4 : 0));
    l.total = off;
    return l;
}

void taco::bind_workspace(SearchLaunch& L, const SearchLayout& lay, char* wb) {
    L.qt = reinterpret_cast<float*>(wb + lay.qt);
    L.cells = reinterpret_cast<uint16_t*>(wb + lay.cells);
    L.ncells = reinterpret_cast<int32_t*>(wb + lay.nc);
    L.retrieved = reinterpret_cast<int64_t*>(wb + lay.ret);
    L.lists_d = reinterpret_cast<float*>(wb + lay.ld);
    L.lists_i = reinterpret_cast<uint32_t*>(wb + lay.li);
    L.unit_ge = reinterpret_cast<uint32_t*>(wb + lay.uge);
    L.unit_off = reinterpret_cast<uint32_t*>(wb + lay.uoff);
    L.unit_len = reinterpret_cast<uint32_t*>(wb + lay.ulen);
    L.arena = reinterpret_cast<uint32_t*>(wb + lay.arena);
    L.qflag = reinterpret_cast<uint32_t*>(wb + lay.qflag);
    L.qlast = reinterpret_cast<int32_t*>(wb + lay.qlast);
    L.hd = reinterpret_cast<float*>(wb + lay.hd);
}

namespace {

int search_impl(const taco_index* cix, const float* queries, int64_t nq, const taco_query_params* per_query,
                const taco_query_params* defaults, int32_t k_stride, int64_t* out_ids, float* out_dists,
                const taco_debug_out* dbg, cudaStream_t st, const taco_params* prepared = nullptr) {
    if (!cix) return fail(TACO_EINVAL, "null index");
    taco_index* ix = const_cast<taco_index*>(cix);
    if (nq < 0) return fail(TACO_EINVAL, "nq < 0");
    if (nq == 0) return TACO_OK;
    if (!queries || !out_ids || !out_dists) return fail(TACO_EINVAL, "null queries or outputs");
    if (!per_query && !defaults && !prepared) return fail(TACO_EINVAL, "per_query and defaults are both NULL");
    if (k_stride < 1) return fail(TACO_EINVAL, "k_stride < 1");
    if (prepared) {
        if (prepared->index != cix) return fail(TACO_EINVAL, "the parameters were prepared for another index");
        if (prepared->nq != nq) return fail(TACO_EINVAL, "%lld queries for %lld prepared parameter records",
                                            (long long)nq, (long long)prepared->nq);
        if (prepared->k_max > k_stride)
            return fail(TACO_EINVAL, "a prepared query has k = %d > k_stride = %d", prepared->k_max, k_stride);
    }
    const taco_query_params& head = prepared ? prepared->head : (per_query ? per_query[0] : *defaults);
    const int precision = head.precision;
    int kk_max = 0;
    if (prepared) {
        kk_max = prepared->kk_max;
    } else if (per_query) {
        for (int64_t j = 0; j < nq; ++j) {
            TRY(check_query_params(per_query[j], k_stride));
            if (per_query[j].precision != precision || per_query[j].select_rule != head.select_rule ||
                per_query[j].probe_precision != head.probe_precision)
                return fail(TACO_EINVAL, "precision, probe_precision and select_rule must be uniform in a batch");
            kk_max = std::max(kk_max, query_list_len(per_query[j]));
        }
    } else {
        TRY(check_query_params(*defaults, k_stride));
        kk_max = query_list_len(*defaults);
    }
    if (precision == TACO_PREC_BF16 && !ix->d_data_bf16)
        return fail(TACO_EINVAL, "BF16 search needs an index with BF16 rows (TACO_ROWS_BF16)");
    if (precision == TACO_PREC_FP8 && !ix->d_data_fp8)
        return fail(TACO_EINVAL, "FP8 search needs an index with FP8 rows (TACO_ROWS_FP8)");
    const int ctc = head.probe_precision == TACO_PREC_BF16 ? 1 : (head.probe_precision == TACO_PREC_FP8 ? 2 : 0);
    if (ctc && !ix->d_cent_tc) return fail(TACO_EINVAL, "this index has no tensor-core centroid block");
    int cur_dev = 0;
    TACO_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != ix->device) return fail(TACO_EINVAL, "current device %d is not the index's device %d", cur_dev, ix->device);

    const bool q_dev = is_device_pointer(queries);
    const bool id_dev = is_device_pointer(out_ids);
    const bool dist_dev = is_device_pointer(out_dists);
    std::lock_guard<std::mutex> lock(ix->ws_mu);
    const int64_t chunk = std::min<int64_t>(nq, kQueryChunk);
    const int Ns = ix->Ns, K = ix->K;
    const SearchLayout lay = plan_search(ix, chunk, kk_max, (per_query && !prepared) ? nq : 0, !q_dev, !id_dev,
                                         !dist_dev, k_stride, ctc != 0);
    const size_t host_need = per_query ? size_t(nq) * sizeof(QueryParamsDev) : 0;
    TRY(ensure_workspace(ix, lay.total, host_need));
    char* wb = static_cast<char*>(ix->ws.base);
    const QueryParamsDev* dparams = prepared ? prepared->d_params : nullptr;
    if (per_query && !prepared) {
        QueryParamsDev* hp = static_cast<QueryParamsDev*>(ix->ws.host_pinned);
        for (int64_t j = 0; j < nq; ++j) hp[j] = query_params_dev(per_query[j]);
        QueryParamsDev* dp = reinterpret_cast<QueryParamsDev*>(wb + lay.par);
        TACO_CUDA(cudaMemcpyAsync(dp, hp, size_t(nq) * sizeof(QueryParamsDev), cudaMemcpyHostToDevice, st));
        dparams = dp;
    }
    for (int64_t c0 = 0; c0 < nq; c0 += chunk) {
        const int64_t cn = std::min(chunk, nq - c0);
        SearchLaunch L = {};
        L.ix = ix;
        L.nq = cn;
        if (q_dev) {
            L.queries = queries + c0 * ix->d;
        } else {
            float* dq = reinterpret_cast<float*>(wb + lay.q);
            TACO_CUDA(cudaMemcpyAsync(dq, queries + c0 * ix->d, size_t(cn) * ix->d * 4, cudaMemcpyHostToDevice, st));
            L.queries = dq;
        }
        L.defaults = query_params_dev(head);
        L.params = dparams ? dparams + c0 : nullptr;
        L.precision = precision;
        L.kk_max = kk_max;
        bind_workspace(L, lay, wb);
        L.centroid_tc = ctc;
        L.out_ids = id_dev ? out_ids + c0 * k_stride : reinterpret_cast<int64_t*>(wb + lay.oi);
        L.out_dists = dist_dev ? out_dists + c0 * k_stride : reinterpret_cast<float*>(wb + lay.od);
        L.k_stride = k_stride;
        if (dbg) {
            L.dbg.query_t = dbg->query_t ? dbg->query_t + c0 * ix->Dp : nullptr;
            L.dbg.probed = dbg->probed ? dbg->probed + size_t(c0) * Ns * K : nullptr;
            L.dbg.retrieved_num = dbg->retrieved_num ? dbg->retrieved_num + c0 * Ns : nullptr;
            L.dbg.sc = dbg->sc ? dbg->sc + size_t(c0) * ix->n : nullptr;
            L.dbg.collision_num = dbg->collision_num ? dbg->collision_num + c0 * (Ns + 1) : nullptr;
            L.dbg.last_collision = dbg->last_collision ? dbg->last_collision + c0 : nullptr;
            L.dbg.candidate_num = dbg->candidate_num ? dbg->candidate_num + c0 : nullptr;
        }
        TRY(run_search_chunk(L, st));
        if (!id_dev)
            TACO_CUDA(cudaMemcpyAsync(out_ids + c0 * k_stride, L.out_ids, size_t(cn) * k_stride * 8,
                                      cudaMemcpyDeviceToHost, st));
        if (!dist_dev)
            TACO_CUDA(cudaMemcpyAsync(out_dists + c0 * k_stride, L.out_dists, size_t(cn) * k_stride * 4,
                                      cudaMemcpyDeviceToHost, st));
    }
    // host outputs, or the pinned parameter staging that the next call reuses
    if (!id_dev || !dist_dev || (per_query && !prepared)) TACO_CUDA(cudaStreamSynchronize(st));
    return TACO_OK;
}

const char kMagic[8] = {'T', 'A', 'C', 'O', 'I', 'D', 'X', '1'};

}  // namespace

extern "C" {

int taco_build_index(const float* data, int64_t n, int32_t d, const taco_build_params* params, void* stream,
                     taco_index** out) {
    return build_impl(data, n, d, params, static_cast<cudaStream_t>(stream), out);
}

int taco_index_create(const float* data, int64_t n, int32_t d, const taco_index_parts* parts, int32_t keep_rows,
                      void* stream, taco_index** out) {
    return create_impl(data, n, d, parts, keep_rows, static_cast<cudaStream_t>(stream), out);
}

int taco_search_batch(const taco_index* index, const float* queries, int64_t nq, const taco_query_params* per_query,
                      const taco_query_params* defaults, int32_t k_stride, int64_t* out_ids, float* out_dists,
                      void* stream) {
    return search_impl(index, queries, nq, per_query, defaults, k_stride, out_ids, out_dists, nullptr,
                       static_cast<cudaStream_t>(stream));
}

int taco_params_create(const taco_index* index, const taco_query_params* per_query, int64_t nq, void* stream,
                       taco_params** out) {
    if (!index || !per_query || !out) return fail(TACO_EINVAL, "null index, parameters or output");
    if (nq < 1) return fail(TACO_EINVAL, "nq must be >= 1");
    *out = nullptr;
    std::unique_ptr<taco_params> p(new taco_params());
    p->index = index;
    p->nq = nq;
    p->head = per_query[0];
    std::vector<QueryParamsDev> host(static_cast<size_t>(nq));
    for (int64_t j = 0; j < nq; ++j) {
        const taco_query_params& q = per_query[j];
        TRY(check_query_params(q, TACO_MAX_K));
        if (q.precision != p->head.precision || q.select_rule != p->head.select_rule ||
            q.probe_precision != p->head.probe_precision)
            return fail(TACO_EINVAL, "precision, probe_precision and select_rule must be uniform in a batch");
        p->kk_max = std::max(p->kk_max, query_list_len(q));
        p->k_max = std::max(p->k_max, q.k);
        host[j] = query_params_dev(q);
    }
    int dev = 0;
    TACO_CUDA(cudaGetDevice(&dev));
    if (dev != index->device) return fail(TACO_EINVAL, "current device %d is not the index's device %d", dev, index->device);
    QueryParamsDev* d = nullptr;
    if (cudaMalloc(&d, host.size() * sizeof(QueryParamsDev)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TACO_ENOMEM, "cannot allocate %lld parameter records", (long long)nq);
    }
    p->d_params = d;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    TACO_CUDA(cudaMemcpyAsync(d, host.data(), host.size() * sizeof(QueryParamsDev), cudaMemcpyHostToDevice, st));
    TACO_CUDA(cudaStreamSynchronize(st));   // the host records go out of scope
    *out = p.release();
    return TACO_OK;
}

void taco_params_free(taco_params* p) {
    if (!p) return;
    cudaFree(const_cast<QueryParamsDev*>(p->d_params));
    delete p;
}

int taco_search_batch_params(const taco_index* index, const float* queries, const taco_params* params,
                             int32_t k_stride, int64_t* out_ids, float* out_dists, void* stream) {
    if (!params) return fail(TACO_EINVAL, "null parameters");
    return search_impl(index, queries, params->nq, nullptr, nullptr, k_stride, out_ids, out_dists, nullptr,
                       static_cast<cudaStream_t>(stream), params);
}

int taco_search_debug(const taco_index* index, const float* queries, int64_t nq, const taco_query_params* per_query,
                      const taco_query_params* defaults, int32_t k_stride, int64_t* out_ids, float* out_dists,
                      const taco_debug_out* debug, void* stream) {
    if (!debug) return fail(TACO_EINVAL, "null debug struct");
    return search_impl(index, queries, nq, per_query, defaults, k_stride, out_ids, out_dists, debug,
                       static_cast<cudaStream_t>(stream));
}

int taco_index_get_info(const taco_index* ix, taco_index_info* info) {
    if (!ix || !info) return fail(TACO_EINVAL, "null argument");
    info->n = ix->n;
    info->d = ix->d;
    info->n_subspaces = ix->Ns;
    info->sub_dim = ix->s;
    info->sqrt_k = ix->sk;
    info->d_pad = ix->d_pad;
    info->has_bf16 = ix->d_data_bf16 != nullptr;
    info->n_slabs = ix->n_slabs;
    info->cluster_size = ix->cluster;
    info->has_fp8 = ix->d_data_fp8 != nullptr;
    info->fp8_pitch = ix->dp8;
    info->has_centroid_tc = ix->d_cent_tc != nullptr;
    info->reserved = 0;
    info->device_bytes = ix->device_bytes;
    info->n_ids = ix->n_ids;
    info->build_ms_transform = ix->build_ms_transform;
    info->build_ms_index = ix->build_ms_index;
    return TACO_OK;
}

int taco_index_lists(const taco_index* ix, uint32_t* sizes, uint32_t* split, uint32_t* ids) {
    if (!ix) return fail(TACO_EINVAL, "null index");
    const size_t m = size_t(ix->Ns) * ix->K;
    if (sizes) TACO_CUDA(cudaMemcpy(sizes, ix->d_sizes, m * 4, cudaMemcpyDeviceToHost));
    if (split) TACO_CUDA(cudaMemcpy(split, ix->d_split, m * (ix->n_slabs + 1) * 4, cudaMemcpyDeviceToHost));
    if (ids) TACO_CUDA(cudaMemcpy(ids, ix->d_ids, size_t(ix->n_ids) * 4, cudaMemcpyDeviceToHost));
    return TACO_OK;
}

int taco_index_export(const taco_index* ix, double* o_bar, double* B, double* eigvals, int32_t* alloc,
                      double* centroids, uint16_t* codes) {
    if (!ix) return fail(TACO_EINVAL, "null index");
    if (o_bar) std::copy(ix->o_bar.begin(), ix->o_bar.end(), o_bar);
    if (B) std::copy(ix->B.begin(), ix->B.end(), B);
    if (eigvals) std::copy(ix->eigvals.begin(), ix->eigvals.end(), eigvals);
    if (alloc) std::copy(ix->alloc.begin(), ix->alloc.end(), alloc);
    if (centroids) std::copy(ix->centroids.begin(), ix->centroids.end(), centroids);
    if (codes) std::copy(ix->codes.begin(), ix->codes.end(), codes);
    return TACO_OK;
}

int taco_save_index(const taco_index* ix, const char* path) {
    if (!ix || !path) return fail(TACO_EINVAL, "null argument");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(TACO_EIO, "cannot open %s for writing", path);
    std::unique_ptr<FILE, int (*)(FILE*)> guard(f, std::fclose);
    const int64_t hdr[6] = {ix->n, ix->d, ix->Ns, ix->s, ix->sk, 0};
    std::vector<float> data(size_t(ix->n) * ix->d);
    if (cudaMemcpy2D(data.data(), size_t(ix->d) * 4, ix->d_data, size_t(ix->d_pad) * 4, size_t(ix->d) * 4,
                     size_t(ix->n), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(TACO_ECUDA, "reading the data back failed");
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 6, f) == 6 &&
              std::fwrite(ix->o_bar.data(), 8, ix->o_bar.size(), f) == ix->o_bar.size() &&
              std::fwrite(ix->B.data(), 8, ix->B.size(), f) == ix->B.size() &&
              std::fwrite(ix->eigvals.data(), 8, ix->eigvals.size(), f) == ix->eigvals.size() &&
              std::fwrite(ix->alloc.data(), 4, ix->alloc.size(), f) == ix->alloc.size() &&
              std::fwrite(ix->centroids.data(), 8, ix->centroids.size(), f) == ix->centroids.size() &&
              std::fwrite(ix->codes.data(), 2, ix->codes.size(), f) == ix->codes.size() &&
              std::fwrite(data.data(), 4, data.size(), f) == data.size();
    if (!ok) return fail(TACO_EIO, "short write to %s", path);
    return TACO_OK;
}

int taco_load_index(const char* path, int32_t keep_rows, void* stream, taco_index** out) {
    if (!path || !out) return fail(TACO_EINVAL, "null argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(TACO_EIO, "cannot open %s", path);
    std::unique_ptr<FILE, int (*)(FILE*)> guard(f, std::fclose);
    char magic[8];
    int64_t hdr[6];
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0 || std::fread(hdr, 8, 6, f) != 6)
        return fail(TACO_EIO, "%s is not a TaCo index file", path);
    const int64_t n = hdr[0];
    const int d = int(hdr[1]), Ns = int(hdr[2]), s = int(hdr[3]), sk = int(hdr[4]);
    TRY(check_geometry(n, d, Ns, s, sk));
    const size_t Dp = size_t(Ns) * s;
    std::vector<double> ob(d), B(size_t(d) * Dp), ev(d), cent(size_t(Ns) * sk * s);
    std::vector<int32_t> alloc(Dp);
    std::vector<uint16_t> codes(size_t(Ns) * n);
    std::vector<float> data(size_t(n) * d);
    bool ok = std::fread(ob.data(), 8, ob.size(), f) == ob.size() && std::fread(B.data(), 8, B.size(), f) == B.size() &&
              std::fread(ev.data(), 8, ev.size(), f) == ev.size() &&
              std::fread(alloc.data(), 4, alloc.size(), f) == alloc.size() &&
              std::fread(cent.data(), 8, cent.size(), f) == cent.size() &&
              std::fread(codes.data(), 2, codes.size(), f) == codes.size() &&
              std::fread(data.data(), 4, data.size(), f) == data.size();
    if (!ok) return fail(TACO_EIO, "%s is truncated", path);
    taco_index_parts parts = {ob.data(), B.data(), cent.data(), codes.data(), Ns, s, sk, 0};
    taco_index* ix = nullptr;
    TRY(create_impl(data.data(), n, d, &parts, keep_rows, static_cast<cudaStream_t>(stream), &ix));
    ix->eigvals = ev;
    ix->alloc = alloc;
    *out = ix;
    return TACO_OK;
}

int taco_centroid_distances(const taco_index* ix, const float* qt, int64_t nq, int32_t probe_precision, float* out,
                            void* stream) {
    if (!ix) return fail(TACO_EINVAL, "null index");
    if (nq < 0) return fail(TACO_EINVAL, "nq < 0");
    if (nq == 0) return TACO_OK;
    if (!qt || !out || !is_device_pointer(qt) || !is_device_pointer(out))
        return fail(TACO_EINVAL, "qt and out must be device pointers");
    if (probe_precision != TACO_PREC_FP32 && probe_precision != TACO_PREC_BF16 && probe_precision != TACO_PREC_FP8)
        return fail(TACO_EINVAL, "probe_precision must be TACO_PREC_FP32, TACO_PREC_BF16 or TACO_PREC_FP8");
    if (probe_precision != TACO_PREC_FP32 && !ix->d_cent_tc)
        return fail(TACO_EINVAL, "this index has no tensor-core centroid block");
    const int mode = probe_precision == TACO_PREC_BF16 ? 1 : (probe_precision == TACO_PREC_FP8 ? 2 : 0);
    TACO_CUDA(launch_centroid_dist(ix, qt, nq, mode, out, static_cast<cudaStream_t>(stream)));
    return TACO_OK;
}

int taco_index_set_option(taco_index* ix, int32_t option, int32_t value) {
    if (!ix) return fail(TACO_EINVAL, "null index");
    std::lock_guard<std::mutex> lock(ix->ws_mu);
    switch (option) {
        case TACO_OPT_CODES_FALLBACK: break;
        case TACO_OPT_SLABS_PER_RANGE:
            // 13..15 slabs take 3-bit counters: only where a count cannot exceed 7
            if (value < 1 || value > (ix->Ns <= 7 ? 15 : 12))
                return fail(TACO_EINVAL, "slabs per range %d not in 1..%d", value, ix->Ns <= 7 ? 15 : 12);
            ix->tp_spc = std::min<int>(value, ix->n_slabs);
            ix->tp_ranges = (ix->n_slabs + ix->tp_spc - 1) / ix->tp_spc;
            return TACO_OK;
        case TACO_OPT_COUNT_WARPS:
            if (value != 8 && value != 16 && value != 32) return fail(TACO_EINVAL, "count warps %d: 8, 16 or 32", value);
            ix->tp_count_warps = value;
            return TACO_OK;
        case TACO_OPT_WALK_UNROLL:
            if (value != 2 && value != 4 && value != 8) return fail(TACO_EINVAL, "walk unroll %d: 2, 4 or 8", value);
            ix->tp_walk_unroll = value;
            return TACO_OK;
        default: return fail(TACO_EINVAL, "unknown option %d", option);
    }
    if (value) return enable_codes_fallback(ix);
    if (ix->cluster == 0) return fail(TACO_ECAPACITY, "n = %lld has no cluster layout: the codes fallback stays", (long long)ix->n);
    ix->codes_fallback = false;
    return TACO_OK;
}

int taco_device_status(const taco_index* ix, int32_t* status, int32_t clear) {
    if (!ix || !status) return fail(TACO_EINVAL, "null argument");
    TACO_CUDA(cudaDeviceSynchronize());
    int v = 0;
    TACO_CUDA(cudaMemcpy(&v, ix->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear) TACO_CUDA(cudaMemset(ix->d_status, 0, sizeof(int)));
    *status = v;
    return TACO_OK;
}

int taco_profile_enable(taco_index* ix, int32_t enable) {
    if (!ix) return fail(TACO_EINVAL, "null index");
    std::lock_guard<std::mutex> lock(ix->ws_mu);
    ix->prof.enabled = enable != 0;
    return TACO_OK;
}

int taco_profile_read(taco_index* ix, taco_kernel_times* out, int32_t reset) {
    if (!ix || !out) return fail(TACO_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(ix->ws_mu);
    Profiler& pr = ix->prof;
    for (auto& p : pr.pending) {
        TACO_CUDA(cudaEventSynchronize(p.second.second));
        float ms = 0.f;
        TACO_CUDA(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
        const int slot = p.first & 0xff;            // bits 8 and up: kernels under the pair
        pr.ms[slot] += ms;
        pr.launches[slot] += std::max(1, p.first >> 8);
    }
    pr.pending.clear();
    pr.used = 0;
    for (int k = 0; k < TACO_NUM_KERNELS; ++k) {
        out->launches[k] = pr.launches[k];
        out->ms[k] = pr.ms[k];
        if (reset) {
            pr.launches[k] = 0;
            pr.ms[k] = 0.0;
        }
    }
    return TACO_OK;
}

void taco_free_index(taco_index* ix) {
    if (!ix) return;
    for (cudaEvent_t e : ix->prof.pool) cudaEventDestroy(e);
    free_device(ix);
    delete ix;
}

}  // extern "C"

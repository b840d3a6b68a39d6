// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "taco.h"

namespace taco {

// Collision counters are 4-bit nibbles, 8 per 32-bit word. Point ids are grouped into
// slabs of 2^15; one CTA of a query's cluster owns a contiguous range of slabs and keeps
// their counters in shared memory.
constexpr int kSlabLog2 = 15;
constexpr int64_t kSlabIds = int64_t(1) << kSlabLog2;
constexpr int kSlabWords = int(kSlabIds / 8);
constexpr int kSlabBytes = kSlabWords * 4;

// Queries handled per internal launch group (bounds the workspace and grid.y).
constexpr int64_t kQueryChunk = 16384;
// Top lists each CTA of a query's cluster writes (one per warp of the fused kernel).
constexpr int kListsPerCta = 16;
// List entries (ids with SC >= 2) reserved per counter slab of a (query, id range) unit.
constexpr size_t kArenaPerSlab = 512;
// Fill of the id-list padding (a cell's list is padded to a multiple of 4 ids); above every
// point id, so a range test rejects it.
constexpr uint32_t kIdPad = 0xffffffffu;

struct QueryParamsDev {
    int32_t k;
    int32_t select_rule;
    int64_t budget;
    int64_t rerank_target;
    int32_t kk;       // list length kept per warp (k, or the BF16 shortlist)
    int32_t pad;
};

// Error reporting (thread-local message).
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
// The step of a kernel-launch helper that failed (attribute, occupancy, launch), for the
// message of the caller's cuda_fail; set by the helpers before they return an error.
extern thread_local const char* g_launch_step;
#define TACO_CUDA(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::taco::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

bool is_device_pointer(const void* p);

// Device status word bits (taco_device_status): a bounded wait gave up, or (checked build) an
// index of a gather or scatter fell outside its buffer in the named pass.
constexpr int kStatusWait = 1;
constexpr int kStatusCount = 2;     // counting pass
constexpr int kStatusSelect = 4;    // select / re-rank pass and its codes fallback
constexpr int kStatusCluster = 8;   // cluster kernel and the merge of its lists

// Bounds checks of the checked build (compiled with -DTACO_CHECKED): a failed check records
// its bit in the status word and the access it guards is skipped; nothing traps. Without the
// flag every check is the constant true and compiles away.
#ifdef TACO_CHECKED
#define TACO_CHECK(status, cond, bit) ((cond) ? true : (atomicOr((status), (bit)), false))
#else
#define TACO_CHECK(status, cond, bit) true
#endif

// Raise a kernel's dynamic shared memory limit to at least `bytes` on the current device.
// The limit only ever grows, process-wide, so launches prepared by different threads (a
// server's dispatcher, callers of the batch API) never lower it under one another.
cudaError_t ensure_dynamic_smem(const void* func, size_t bytes);

// Host FP64 linear algebra (build side).
void symmetric_eigen(int d, std::vector<double>& a, std::vector<double>& vecs,
                     std::vector<double>& vals);
void eigensystem_allocation(const std::vector<double>& lam, int n_subspaces, int sub_dim,
                            std::vector<std::vector<int>>& buckets);

struct Profiler {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;                 // reusable events
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    size_t used = 0;
    int64_t launches[TACO_NUM_KERNELS] = {};
    double ms[TACO_NUM_KERNELS] = {};
};

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    void* host_pinned = nullptr;
    size_t host_bytes = 0;
};

}  // namespace taco

struct taco_index {
    int64_t n = 0;
    int d = 0, d_pad = 0, Ns = 0, s = 0, sk = 0, K = 0, Dp = 0, h1 = 0;
    int n_slabs = 0;
    int cluster = 1, slabs_per_cta = 1;   // layout of the single-pass cluster kernel
    // Tuned launch choices (taco_autotune; defaults from configure_search):
    int tp_spc = 1, tp_ranges = 1;        // slabs per id range of the two-pass counting, ranges
    int tp_spc0 = 1, tp_ranges0 = 1;      // the index's default two-pass layout (configure_search)
    int tp_lanes[3] = {0, 0, 0};          // lanes per row of the re-rank per row kind (0: auto)
    int tp_walk = -1;                     // probe by row-merge walk: -1 auto, 0 never, 1 when it fits
    int tp_count_warps = 16;              // warps per CTA of the counting pass (8, 16 or 32)
    int tp_walk_unroll = 4;               // windows of 32 four-id chunks per round of its walk (2, 4 or 8)
    // Fallback for flagged queries: the cluster kernel (all counters of a query in one
    // cluster's shared memory) or, when n is too large for that (cluster == 0) or when
    // chosen (taco_index_set_option), the codes fallback of select_rerank_kernel.
    bool codes_fallback = false;
    uint16_t* d_codes = nullptr;          // [Ns][n] cell of every point (codes fallback)
    int device = 0;
    // host copies of the parts
    std::vector<double> o_bar, B, eigvals, centroids;
    std::vector<int32_t> alloc;
    std::vector<uint16_t> codes;
    // device arrays
    float* d_data = nullptr;            // [n][d_pad]
    __nv_bfloat16* d_data_bf16 = nullptr;  // [n][d_pad] or null
    uint8_t* d_data_fp8 = nullptr;      // [n][dp8] e4m3 rows (fp8_space), or null
    float* d_fp8_scale = nullptr;       // [2][dp8]: per-dimension scale (its group's), 1/scale
    int dp8 = 0;                        // FP8 coordinates per row rounded up to 16
    int fp8_space = 0;                  // 0: B^T (o - o_bar) (N_s s = d), 1: o - o_bar
    uint8_t* d_cent_tc = nullptr;       // [2 N_s] BF16 centroid operands in the tcgen05 layout
    float* d_cent_tc_norm = nullptr;    // [2 N_s][N] squared norms of those BF16 centroids
    uint8_t* d_cent_tc8 = nullptr;      // [2 N_s] E4M3 centroid operands (c / scale of the pair)
    float* d_cent_tc8_norm = nullptr;   // [2 N_s][N] squared norms of the values they stand for
    float* d_cent_tc8_scale = nullptr;  // [2 N_s] scale of each pair (max |c| / 448)
    int* d_status = nullptr;            // device status word: 1 = a bounded device wait gave up
    float* d_obar = nullptr;            // [d]
    float* d_B = nullptr;               // [d][Dp]
    float* d_cent = nullptr;            // [Ns][sk][s]
    uint32_t* d_sizes = nullptr;        // [Ns][K]
    uint32_t* d_ids = nullptr;          // [n_ids]: cell lists, each 16-byte aligned and padded
    uint32_t* d_split = nullptr;        // [Ns][K][n_slabs + 1] absolute positions in d_ids
    int64_t n_ids = 0;                  // length of d_ids (N_s n plus the padding)
    double build_ms_transform = 0.0;    // Alg. 1 part of the build (wall time)
    double build_ms_index = 0.0;        // k-means, cell lists, row copies (wall time)
    int64_t device_bytes = 0;
    std::mutex ws_mu;
    taco::Workspace ws;
    taco::Profiler prof;
};

// Per-query parameters copied to the device once (taco_params_create).
struct taco_params {
    const taco_index* index = nullptr;
    int64_t nq = 0;
    const taco::QueryParamsDev* d_params = nullptr;   // device [nq]
    taco_query_params head{};                         // the batch-uniform fields (query 0)
    int kk_max = 0;                                   // longest list any query needs
    int k_max = 0;                                    // largest k
};

namespace taco {

// Kernel launchers (return cudaGetLastError of the launch).
cudaError_t launch_project(const float* X, int64_t rows, int d, int64_t ldx, const float* obar,
                           const float* B, int Dp, float* Y, cudaStream_t st);
cudaError_t launch_col_mean(const float* X, int64_t n, int d, int ldx, double* sums,
                            cudaStream_t st);
cudaError_t launch_covariance(const float* X, int64_t n, int d, int ldx, const double* mean,
                              double* cov, cudaStream_t st);
cudaError_t launch_kmeans(const float* T, int64_t n, int Dp, int Ns, int s, int h1, int sk,
                          int iters, const int64_t* init_rows_host, float* cent_out,
                          uint16_t* codes_out, cudaStream_t st);
cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, size_t count,
                           cudaStream_t st);
// Y[r][c] = X[r][c] - obar[c] (X row pitch ldx, Y row pitch d).
cudaError_t launch_center(const float* X, int64_t rows, int d, int64_t ldx, const float* obar, float* Y,
                          cudaStream_t st);
// Largest |Y[r][c]| of every column into maxbits[c] (float bits; atomicMax, caller zeroes).
cudaError_t launch_absmax_cols(const float* Y, int64_t rows, int Dp, unsigned* maxbits,
                               cudaStream_t st);
// out[r][c] = e4m3(Y[r][c] * inv_scale[c]) for c < Dp, 0 for Dp <= c < dp8.
cudaError_t launch_quantize_fp8(const float* Y, int64_t rows, int Dp, int dp8,
                                const float* inv_scale, uint8_t* out, cudaStream_t st);

// Cell lists of Alg. 3 on the device from the cell codes [Ns][n]: sizes [Ns * K], the padded
// list starts [Ns * K + 1] (start[Ns * K] = total ids with padding), the slab table
// [Ns * K][n_slabs + 1] and the ids (pre-filled with kIdPad by the caller). scratch holds
// lists_scratch_words(n, Ns, K) words.
int64_t lists_scratch_words(int64_t n, int Ns, int K);
cudaError_t launch_build_lists(const uint16_t* codes, int64_t n, int Ns, int K, uint32_t* scratch,
                               uint32_t* sizes, uint32_t* start, uint32_t* split, uint32_t* ids,
                               cudaStream_t st);

// Query x centroid distance block (Alg. 6 steps 4-5) as a separate kernel:
// hd[q][i][h][c] = |q'_{i,h} - C_{i,h}[c]|^2, FP32 on CUDA cores or, on tcgen05, BF16 or E4M3
// (per-pair / per-query scales) operands with FP32 accumulation.
bool centroid_tc_supported(const taco_index* ix);
int build_centroid_tc(taco_index* ix);
cudaError_t launch_centroid_dist(const taco_index* ix, const float* qt, int64_t nq, int mode,
                                 float* hd, cudaStream_t st);

struct SearchLaunch {
    const taco_index* ix;
    const float* queries;      // device [nq][d]
    int64_t nq;
    QueryParamsDev defaults;
    const QueryParamsDev* params;  // device [nq] or null
    int precision;
    int kk_max;
    float* qt;                 // device [nq][Dp]
    uint16_t* cells;           // device [nq][Ns][K]
    int32_t* ncells;           // device [nq][Ns]
    int64_t* retrieved;        // device [nq][Ns]
    float* lists_d;            // device [nq][cluster][kListsPerCta][kk_max]
    uint32_t* lists_i;         // device [nq][cluster][kListsPerCta][kk_max]
    // two-pass form (null unit_ge: cluster kernel for every query)
    uint32_t* unit_ge;         // device [nq][tp_ranges][16]
    uint32_t* unit_off;        // device [nq][tp_ranges]
    uint32_t* unit_len;        // device [nq][tp_ranges]
    uint32_t* arena;           // device [nq][tp_ranges][kArenaPerSlab * tp_spc]
    uint32_t* qflag;           // device [nq + 2]: flags, then the passes' query counters
    int32_t* qlast;            // device [nq] Alg. 5 threshold of flagged queries
    int64_t* out_ids;
    float* out_dists;
    int k_stride;
    taco_debug_out dbg;        // device pointers, already offset to this chunk
    bool skip_profile;         // record no profiling events (launches that may be captured)
    int centroid_tc;           // centroid distances from a tcgen05 block into hd: 0 none,
                               // 1 BF16 operands, 2 E4M3 operands
    float* hd;                 // device [nq][Ns][2][sk] (centroid_tc != 0)
    // id-range shards (taco_shard_*): phase 0 runs the whole search; phase 1 the transform,
    // probe and counting of the ranges [shard_r0, shard_r1) and their level counts into
    // shard_hist [nq][Ns + 1]; phase 2 Alg. 5 on the all-shard counts ghist [nq][Ns + 1], the
    // select / re-rank of the shard's ranges and the codes fallback over the shard's ids
    int phase;
    int shard_r0, shard_r1;    // shard_r1 <= 0: all ranges
    int64_t* shard_hist;
    const int64_t* ghist;
};
int run_search_chunk(const SearchLaunch& L, cudaStream_t st);
cudaError_t launch_shard_hist(const uint32_t* unit_ge, int64_t nq, int nr, int r0, int r1, int Ns, int64_t points,
                              int64_t* hist, cudaStream_t st);

// Byte offsets of one launch group's device workspace (each 256-byte aligned).
struct SearchLayout {
    size_t qt, cells, nc, ret, ld, li, uge, uoff, ulen, arena, qflag, qlast, par, q, oi, od, hd;
    size_t total;
};
// Workspace of `chunk` queries with lists of kk_max entries; `n_params` per-query parameter
// records, and staging for queries / ids / distances when the caller's are not on the device.
SearchLayout plan_search(const taco_index* ix, int64_t chunk, int kk_max, int64_t n_params,
                         bool stage_queries, bool stage_ids, bool stage_dists, int k_stride,
                         bool centroid_tc = false);
// The workspace pointers of a SearchLaunch over `wb` laid out by `lay` (two-pass form).
void bind_workspace(SearchLaunch& L, const SearchLayout& lay, char* wb);
// Device form of the query parameters and the list length they need.
int check_query_params(const taco_query_params& q, int k_stride);
int query_list_len(const taco_query_params& q);
QueryParamsDev query_params_dev(const taco_query_params& q);
// Event pair around one kernel launch when profiling is enabled (no-op otherwise).
int prof_begin(taco_index* ix, int slot, cudaStream_t st, cudaEvent_t* b, cudaEvent_t* e);
int prof_end(taco_index* ix, int slot, cudaStream_t st, cudaEvent_t b, cudaEvent_t e);
int configure_search(taco_index* ix);
// Device copy of the cell codes (the codes fallback), made once.
int ensure_device_codes(taco_index* ix);

}  // namespace taco

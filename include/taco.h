/*
 * taco.h -- C ABI of the GB300 (sm_103a) TaCo query path.
 *
 * TaCo (arXiv 2603.24919) answers k-approximate-nearest-neighbour queries (Def. 3) over a
 * dataset D of n points in R^d. The index (Alg. 3) holds an entropy-balanced orthonormal
 * transform B (Alg. 1, Alg. 2), and for each of N_s subspaces of s transformed
 * dimensions an inverted multi-index: two sets of sqrt(K) half-subspace centroids and the
 * list of point ids in each of the K = sqrt(K)^2 cells. A query (Alg. 6) is transformed,
 * probes each subspace's cells nearest-first until a collision budget is met (Alg. 4),
 * counts per point the subspaces it collided in (SC-score, Def. 6), keeps the points of
 * the highest SC levels (Alg. 5) and returns the k nearest of them by exact distance.
 *
 * Conventions shared by every entry point:
 *   - Return value: TACO_OK (0) or a negative TACO_E* code; taco_last_error() then holds a
 *     message for the calling thread. No entry point aborts the process.
 *   - Pointers are host or device pointers as each argument states. "host or device"
 *     arguments are classified with cudaPointerGetAttributes.
 *   - Work is ordered on the caller's CUDA stream (`stream`, a cudaStream_t; NULL = the
 *     legacy default stream). Calls return once the work is enqueued, except where an
 *     argument is a host output, in which case the call synchronises the stream first.
 *   - Matrices are row-major, float32 unless stated. Point ids are 0-based row numbers.
 *   - One search at a time per index: searches on one index share its workspace and are
 *     serialised on the host; two streams searching one index concurrently would race on
 *     the device.
 */
#ifndef TACO_H_
#define TACO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------- */
#define TACO_OK 0
#define TACO_EINVAL (-1)    /* bad argument: null pointer, size or parameter out of range */
#define TACO_ENOMEM (-2)    /* device or host allocation failed */
#define TACO_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define TACO_ETIMEOUT (-4)  /* reserved: a bounded device wait gave up */
#define TACO_ECAPACITY (-5) /* the request exceeds a compiled capacity (n, k, sqrt_k) */
#define TACO_EIO (-6)       /* file could not be read or written, or has a bad format */
#define TACO_EAGAIN (-7)    /* a server's request queue is full: collect results, then retry */

/* ---- enums ------------------------------------------------------------------------- */
#define TACO_PREC_FP32 0    /* re-rank candidates with FP32 distances */
#define TACO_PREC_BF16 1    /* re-rank with a BF16 copy of D, then exact FP32 on a shortlist */
#define TACO_PREC_FP8 2     /* re-rank with an FP8-e4m3 copy of the points, then exact FP32 on a
                               shortlist: of the transformed points B^T (o - o_bar) when
                               N_s*s = d (distances preserved, Lemma 1), else of the centred
                               points o - o_bar; one scale per block of 16 dimensions. The
                               candidate distances form each block's differences and squares in
                               half precision (query coordinates clamped to 4x the block's
                               largest point coordinate) and sum the blocks in FP32 */

/* Row copies an index keeps besides the FP32 rows (bit mask, the keep_rows arguments). */
#define TACO_ROWS_BF16 1    /* BF16 copy of D, [n][d_pad] */
#define TACO_ROWS_FP8 2     /* FP8-e4m3 copy, [n][fp8_pitch] (see TACO_PREC_FP8) */

#define TACO_SELECT_LITERAL 0 /* Alg. 5 as printed: stop at j when h[j] > R - sum_{j'>=j} h */
#define TACO_SELECT_PROSE 1   /* Alg. 5 as described: stop when sum_{j'>=j} h[j'] > R */

/* Compiled capacities. */
#define TACO_MAX_SUBSPACES 15  /* SC-scores are held in 4-bit counters */
#define TACO_MAX_SQRT_K 128
#define TACO_MAX_K 512         /* k, and the BF16 shortlist, per query */

typedef struct taco_index taco_index; /* opaque; owns all device memory of one index */

/* Build parameters (Alg. 3 inputs; Table 1 notation). */
typedef struct {
    int32_t n_subspaces;   /* N_s, 1..TACO_MAX_SUBSPACES */
    int32_t sub_dim;       /* s; N_s * s <= d. Half 1 = first floor(s/2) dims, half 2 = rest */
    int32_t sqrt_k;        /* sqrt(K): centroids per half-subspace, 1..TACO_MAX_SQRT_K */
    int32_t kmeans_iters;  /* t: Lloyd iterations of each half-subspace k-means */
    uint64_t seed;         /* seeds the k-means initial centroids */
    int32_t keep_rows;     /* TACO_ROWS_* mask: row copies for TACO_PREC_BF16 / TACO_PREC_FP8 */
    int32_t reserved;      /* must be 0 */
} taco_build_params;

/* Query parameters (Alg. 6 inputs). One struct per query, or one for the whole batch. */
typedef struct {
    int32_t k;             /* results wanted, 1..TACO_MAX_K and <= k_stride */
    int32_t precision;     /* TACO_PREC_*; must be the same for every query of a batch */
    int64_t budget;        /* collision budget per subspace: B = ceil(alpha * n) >= 1 (Alg. 4) */
    int64_t rerank_target; /* R = floor(beta * n) >= 0 (Alg. 5) */
    int32_t select_rule;   /* TACO_SELECT_*; must be the same for every query of a batch */
    int32_t shortlist_mult;/* TACO_PREC_BF16 / _FP8: exact FP32 re-rank of min(mult*k, TACO_MAX_K) */
    int32_t probe_precision;/* query x centroid distances (Alg. 6 steps 4-5): TACO_PREC_FP32 on CUDA
                               cores; TACO_PREC_BF16: BF16 operands on the tcgen05 tensor cores
                               with FP32 accumulation; TACO_PREC_FP8: E4M3 operands (kind::f8f6f4),
                               each centroid half scaled by its (subspace, half)'s max |c| / 448
                               and each half-query by its own max |q| / 448, FP32 accumulation
                               (both need taco_index_info.has_centroid_tc). Must be the same for
                               every query of a batch */
    int32_t reserved;      /* must be 0 */
} taco_query_params;

/* An index given by its parts (e.g. built elsewhere); all pointers are host pointers. */
typedef struct {
    const double* o_bar;       /* [d]      data mean (Alg. 1) */
    const double* B;           /* [d][N_s*s] transform; column c of subspace i is B[:, i*s + c] */
    const double* centroids;   /* [N_s][sqrt_k][s]: row r holds half-1 centroid r in dims
                                  [0, floor(s/2)) and half-2 centroid r in [floor(s/2), s) */
    const uint16_t* codes;     /* [N_s][n] cell of each point: r * sqrt_k + c */
    int32_t n_subspaces, sub_dim, sqrt_k;
    int32_t reserved;          /* must be 0 */
} taco_index_parts;

typedef struct {
    int64_t n;
    int32_t d, n_subspaces, sub_dim, sqrt_k;
    int32_t d_pad;             /* row pitch of the device copy of D, in elements */
    int32_t has_bf16;
    int32_t n_slabs;           /* id slabs of 32768 points (collision-counter granularity) */
    int32_t cluster_size;      /* CTAs that share one query's counters in the cluster kernel;
                                  0 when n is too large for a cluster (codes fallback) */
    int32_t has_fp8;           /* FP8 rows kept (TACO_ROWS_FP8) */
    int32_t fp8_pitch;         /* row pitch of the FP8 rows in bytes (N_s*s, or d when N_s*s < d,
                                  rounded up to a power of two up to 64, else to whole
                                  128-byte lines) */
    int32_t has_centroid_tc;   /* the tcgen05 centroid blocks (BF16 and E4M3) are available
                                  (sqrt_k <= 128 and the operands of 128 queries fit shared memory) */
    int32_t reserved;
    int64_t device_bytes;      /* device memory owned by the index, workspace excluded */
    int64_t n_ids;             /* length of the cell-list array (taco_index_lists) */
    double build_ms_transform; /* wall time of Alg. 1 (mean, covariance, eigensystem, Alg. 2,
                                  projection of D); 0 for an index made from its parts */
    double build_ms_index;     /* wall time of the rest of the build: k-means of Alg. 3, the
                                  cell lists and slab table, the reduced-precision row copies */
} taco_index_info;

/* Optional device outputs of taco_search_debug (any may be NULL). */
typedef struct {
    float* query_t;            /* [nq][N_s*s] transformed queries B^T (q - o_bar) */
    uint8_t* probed;           /* [nq][N_s][K] 1 where Alg. 4 retrieved the cell */
    int64_t* retrieved_num;    /* [nq][N_s] sum of retrieved cell sizes (Alg. 4) */
    uint8_t* sc;               /* [nq][n] SC-score of every point (Def. 6) */
    int64_t* collision_num;    /* [nq][N_s+1] collision_num of Alg. 5 */
    int32_t* last_collision;   /* [nq] last_collision of Alg. 5 (-1 .. N_s) */
    int64_t* candidate_num;    /* [nq] candidate_num = |C| of Alg. 5 */
} taco_debug_out;

/*
 * taco_build_index -- build the index of Alg. 3 (with Alg. 1 and Alg. 2) from D.
 *   data    host or device, [n][d] float32 (finite values). Copied; the caller keeps it.
 *   n >= 2, 1 <= d; params as documented above.
 * Mean and covariance are accumulated in FP64 on the device, the eigendecomposition and the
 * allocation of Alg. 2 run in FP64 on the host, k-means runs on the device. Synchronises
 * `stream`. On success *out owns the index (free with taco_free_index).
 */
int taco_build_index(const float* data, int64_t n, int32_t d, const taco_build_params* params,
                     void* stream, taco_index** out);

/*
 * taco_index_create -- make an index from given parts (Alg. 3 output) and the data D.
 *   data host or device [n][d] float32; parts host pointers as in taco_index_parts.
 *   keep_rows TACO_ROWS_* mask of the reduced-precision row copies to build.
 * Cell lists are rebuilt from codes with ids ascending in every cell. Synchronises `stream`.
 * FP8 rows: every point is transformed (Alg. 1) or centred (see TACO_PREC_FP8), each block
 * of 16 dimensions' scale is its largest |coordinate| / 448 (the e4m3 maximum), and
 * coordinates are rounded to nearest e4m3.
 */
int taco_index_create(const float* data, int64_t n, int32_t d, const taco_index_parts* parts,
                      int32_t keep_rows, void* stream, taco_index** out);

/*
 * taco_search_batch -- Alg. 6 for nq queries.
 *   queries    host or device, [nq][d] float32.
 *   per_query  host pointer to nq structs, or NULL to use *defaults for every query.
 *   defaults   host pointer; required when per_query is NULL.
 *   k_stride   row length of the outputs (>= every query's k).
 *   out_ids    host or device, [nq][k_stride] int64: ids ascending by (distance, id);
 *              entries past min(k, |C|) are -1.
 *   out_dists  host or device, [nq][k_stride] float32: Euclidean (not squared) distances;
 *              +inf where out_ids is -1.
 * Errors: TACO_EINVAL for bad arguments; TACO_ECAPACITY for k > TACO_MAX_K.
 */
int taco_search_batch(const taco_index* index, const float* queries, int64_t nq,
                      const taco_query_params* per_query, const taco_query_params* defaults,
                      int32_t k_stride, int64_t* out_ids, float* out_dists, void* stream);

/*
 * Per-query parameters resident on the device, for batches searched again and again (a
 * benchmark loop, a fixed request mix, a captured CUDA graph). taco_search_batch with a
 * per_query array converts and copies the nq records on every call and synchronises the
 * stream afterwards (its pinned staging is reused); a taco_params batch does that once.
 * The paper has no counterpart: this only moves Alg. 6's per-query inputs (k, B, R of Alg. 4
 * and Alg. 5) to the device ahead of time.
 */
typedef struct taco_params taco_params;

/*
 * taco_params_create -- check the nq host records per_query (as taco_search_batch does, with
 * k <= TACO_MAX_K; precision, select_rule and probe_precision uniform), copy them to device
 * memory allocated here, and return the handle in *out. Synchronises `stream`. The handle is
 * tied to `index` and to nq. Errors: TACO_EINVAL, TACO_ECAPACITY (k > TACO_MAX_K), TACO_ENOMEM.
 */
int taco_params_create(const taco_index* index, const taco_query_params* per_query, int64_t nq,
                       void* stream, taco_params** out);

/* taco_params_free -- release a parameter batch (NULL is a no-op). No search using it may be
 * running or queued. */
void taco_params_free(taco_params* params);

/*
 * taco_search_batch_params -- taco_search_batch for the params->nq queries with the prepared
 * per-query parameters (query j uses record j). Arguments and results as taco_search_batch;
 * k_stride must be >= every prepared k. Nothing is copied from the host and the call does not
 * synchronise the stream unless an output is a host pointer. With device queries and outputs
 * and a workspace already large enough (an earlier call of the same shape), the call only
 * enqueues kernels, so it can be captured in a CUDA graph.
 */
int taco_search_batch_params(const taco_index* index, const float* queries, const taco_params* params,
                             int32_t k_stride, int64_t* out_ids, float* out_dists, void* stream);

/*
 * taco_search_batch_noalloc -- taco_search_batch for callers that may not allocate device
 * memory (a process whose device memory is owned by its own pool or framework, or a
 * request path where a cudaMalloc, which can synchronise the device, is not allowed).
 * The paper has no counterpart: this is a deployment variant of the same Alg. 6 kernels.
 *   queries    device, [nq][d] float32.     out_ids / out_dists  device, [nq][k_stride].
 *   params     host pointer, one struct for the whole batch (no per-query parameters).
 * Scratch lives in a fixed 64 MiB array in device memory that every GPU which loads the
 * library holds until the process exits; the call itself calls no allocating routine.
 * Every scratch byte read by a call is written earlier in the same call, so nothing needs
 * clearing between calls. Limits: nq <= 16384 and the batch's scratch must fit the array,
 * else TACO_ECAPACITY. The scratch is six regions, each rounded up to 256 bytes, of
 * nq*4*Dp, nq*2*N_s*K, nq*4*N_s, nq*8*N_s and twice nq*64*C*kk bytes, where Dp is N_s*s,
 * C the index's cluster_size and kk the k of the query or its BF16 shortlist
 * min(shortlist_mult*k, TACO_MAX_K). FP8 rows (TACO_PREC_FP8) and the tensor-core centroid
 * block (probe_precision TACO_PREC_BF16) are refused with TACO_EINVAL.
 * TACO_ECAPACITY also for an index whose cluster_size is 0 (n above 16 x 11 x 2^15 points for d up to 1,300).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. All calls share the array, so calls
 * that overlap on the GPU (other streams, other threads) race: serialise them.
 * Returns TACO_EINVAL while profiling (taco_profile_enable) is on for the index.
 */
int taco_search_batch_noalloc(const taco_index* index, const float* queries, int64_t nq,
                              const taco_query_params* params, int32_t k_stride,
                              int64_t* out_ids, float* out_dists, void* stream);

/*
 * Id-range shards (Alg. 6 split over the points; Def. 6 and Alg. 5 need one exchange).
 * Shard s of S holds id ranges [s R / S, (s + 1) R / S) of the index's R two-pass ranges
 * (taco_index_info's layout; 1 <= S <= R). Every shard probes the same cells (the global cell
 * sizes), counts the collisions of its own ids, and reports its level counts; Alg. 5 then
 * runs on the counts summed over all shards, so every shard takes the candidates the
 * one-index search would take among its ids, and the k nearest of the shards' results by
 * (distance, id) are the one-index result (FP32 rows exactly; BF16 / FP8 rows re-rank each
 * shard's own shortlist, so the merged shortlist holds S times the candidates). Queries the
 * threshold takes below level 2, or whose entries overflow a shard's arena slot, are answered
 * by the codes fallback over the shard's ids. In this library the shards run in one process
 * on the index's device; the caller sums the counts and merges the results (on a multi-GPU
 * node: an all-reduce of [nq][N_s + 1] int64 and an all-gather of [nq][k] results).
 *
 * taco_shard_count -- the transform, probe and counting of `shard` for a batch (queries
 *   [nq][d] host or device, 1 <= nq <= 16384; per_query or defaults as in taco_search_batch;
 *   k_stride: the row length of the results the select will write). Writes the shard's level
 *   counts hist [nq][N_s + 1] int64 (host or device): hist[q][0] = the shard's points,
 *   hist[q][j] = its ids with SC >= j. Returns a handle that owns the batch's device state
 *   (queries, probed cells, counts, entries) until taco_shard_free. Synchronises `stream`
 *   when hist or per_query is on the host. TACO_EINVAL on bad arguments (shard, n_shards,
 *   nq, parameters), TACO_ENOMEM / CUDA errors on allocation. The index's layout must not
 *   change (taco_autotune, taco_index_set_option) between the count and the select.
 * taco_shard_select -- Alg. 5 on global_hist [nq][N_s + 1] int64 (host or device: the sum of
 *   every shard's hist), then the shard's candidates, re-rank and k nearest: out_ids [nq]
 *   [k_stride] int64 and out_dists float (host or device; -1 / +inf past the shard's
 *   candidates). Synchronises `stream`.
 * taco_shard_free -- releases a handle (NULL is a no-op). A handle refers to its index: free
 *   every handle of an index before taco_index_free.
 */
typedef struct taco_shard_search taco_shard_search;
int taco_shard_count(const taco_index* index, int32_t shard, int32_t n_shards, const float* queries, int64_t nq,
                     const taco_query_params* per_query, const taco_query_params* defaults, int32_t k_stride,
                     int64_t* hist, void* stream, taco_shard_search** out);
int taco_shard_select(taco_shard_search* shard, const int64_t* global_hist, int64_t* out_ids, float* out_dists,
                      void* stream);
int taco_shard_free(taco_shard_search* shard);

/*
 * taco_centroid_distances -- the query x centroid distance block of Alg. 6 steps 4-5 alone:
 *   qt     device, [nq][N_s*s] float32 transformed queries B^T (q - o_bar).
 *   out    device, [nq][N_s][2][sqrt_k] float32: out[q][i][h][c] = |q'_{i,h} - C_{i,h}[c]|^2,
 *          half h = 0 the first floor(s/2) dimensions of subspace i, h = 1 the rest.
 *   probe_precision  TACO_PREC_FP32 (CUDA cores, sum of squared differences), TACO_PREC_BF16
 *          (tcgen05 tensor cores: BF16 operands, FP32 accumulation of |q|^2 + |c|^2 - 2 q.c,
 *          clamped at 0) or TACO_PREC_FP8 (tcgen05: E4M3 of c / s_c and q / s_q with s_c = max |c|
 *          / 448 over the (subspace, half)'s centroids and s_q = max |q| / 448 over the half-query,
 *          each value rounded to nearest even; |q|^2, |c|^2 and q.c of the rounded values times
 *          the scales, FP32 accumulation). TACO_EINVAL unless has_centroid_tc.
 * Asynchronous on `stream`. A bounded device wait that gives up sets the status word read by
 * taco_device_status.
 */
int taco_centroid_distances(const taco_index* index, const float* qt, int64_t nq,
                            int32_t probe_precision, float* out, void* stream);

/*
 * taco_index_set_option -- set a launch option of the index.
 *   TACO_OPT_CODES_FALLBACK: value != 0 answers the queries the two-pass search cannot finish
 *   (Alg. 5 threshold below 2, or a level list past its slot) by the codes fallback: SC-scores
 *   recomputed from the cell codes of every probed point and bitmaps of the probed cells
 *   (keeps a device copy of the codes, 2 bytes per point and subspace); value 0 uses the
 *   cluster kernel (all of a query's counters in one thread-block cluster's shared memory).
 *   An index whose n is too large for any cluster (more than 16 x 11 slabs of 2^15 points)
 *   always uses the codes fallback (TACO_ECAPACITY for value 0).
 *   TACO_OPT_SLABS_PER_RANGE: counter slabs per id range of the two-pass counting, 1 .. 12
 *   with 4-bit counters, and 13 .. 15 with 3-bit counters for an index of N_s <= 7 (a value
 *   above the index's n_slabs acts as n_slabs; n_ranges follows; TACO_ECAPACITY at search
 *   time if the counters do not fit an SM; TACO_EINVAL outside the range).
 *   TACO_OPT_COUNT_WARPS: warps per counting CTA, 8, 16 or 32.
 *   TACO_OPT_WALK_UNROLL: loads of four ids in flight per lane in the counting walk, 2, 4 or 8
 *   (8 takes effect with 16 warps only; an unbuilt pair runs 16 warps x 4).
 *   The last three are the choices taco_autotune makes; they change no result beyond the FP32
 *   summation order of a distance. Other values: TACO_EINVAL.
 * Must not run while searches or a server use the index.
 */
#define TACO_OPT_CODES_FALLBACK 1
#define TACO_OPT_SLABS_PER_RANGE 2
#define TACO_OPT_COUNT_WARPS 3
#define TACO_OPT_WALK_UNROLL 4
int taco_index_set_option(taco_index* index, int32_t option, int32_t value);

/* taco_device_status -- synchronise the device and read (clear != 0: then reset) the index's
 * device status word: 0 = no device-side wait ever gave up, 1 = one did (its results are not
 * valid). Kernels never trap; they record the failure here and return. */
int taco_device_status(const taco_index* index, int32_t* status, int32_t clear);

/* Launch layout chosen by taco_autotune. */
typedef struct {
    int32_t slabs_per_range;   /* counter slabs (2^15 ids, 16 KB of 4-bit counters each) per id
                                  range of the two-pass collision counting */
    int32_t n_ranges;          /* id ranges per query */
    int32_t lanes_per_row;     /* lanes gathering one candidate row in the re-rank (0 = auto) */
    int32_t probe_walk;        /* -1: row-merge walk for small budgets (auto), 0: histogram only */
    int32_t count_warps;       /* warps per CTA of the counting pass (8, 16 or 32) */
    int32_t walk_unroll;       /* loads of four ids in flight per lane in its walk (2 or 4, or 8
                                  with 16 warps) */
    double ms_before;          /* mean ms of one search of the sample before tuning */
    double ms_after;           /* with the chosen layout */
    int32_t trials;            /* searches timed */
    int32_t reserved;
} taco_tune_result;

/*
 * taco_autotune -- time searches of a sample batch (queries: device [nq][d]; params: one
 * struct for the batch) on `stream` over the launch layouts above (coordinate descent: counter
 * layout, counting CTA size and walk depth, lanes per row for the params' row kind, probe
 * strategy; each candidate: one untimed and `reps` timed searches) and keep the fastest for
 * this index's later searches. The layout changes no result beyond the FP32 summation order
 * of a candidate's distance. reps <= 0 restores the default layout. Synchronises `stream`; must not run while
 * other searches or a server use the index. Profiling must be off (TACO_EINVAL).
 */
int taco_autotune(taco_index* index, const float* queries, int64_t nq, const taco_query_params* params,
                  int32_t reps, void* stream, taco_tune_result* out);

/* taco_search_debug -- taco_search_batch that also writes the intermediate results
 * selected in *debug (device pointers). Test aid; same errors as taco_search_batch. */
int taco_search_debug(const taco_index* index, const float* queries, int64_t nq,
                      const taco_query_params* per_query, const taco_query_params* defaults,
                      int32_t k_stride, int64_t* out_ids, float* out_dists,
                      const taco_debug_out* debug, void* stream);

/* taco_index_get_info -- sizes and layout of an index (host output). */
int taco_index_get_info(const taco_index* index, taco_index_info* info);

/*
 * taco_index_export -- copy the index parts to host buffers (any may be NULL):
 *   o_bar [d] f64, B [d][N_s*s] f64, eigvals [d] f64 (covariance eigenvalues, descending;
 *   zeros for an index made by taco_index_create), alloc [N_s*s] i32 (rank, in descending
 *   eigenvalue order, of the eigenvector in each column of B; -1 when unknown),
 *   centroids [N_s][sqrt_k][s] f64, codes [N_s][n] u16.
 */
int taco_index_export(const taco_index* index, double* o_bar, double* B, double* eigvals,
                      int32_t* alloc, double* centroids, uint16_t* codes);

/*
 * taco_index_lists -- copy the index's cell lists (Alg. 3's IMI) to host buffers (any may be
 * NULL; inspection and test aid):
 *   sizes [N_s][K] u32       |IMI_i[cell]|
 *   split [N_s][K][n_slabs + 1] u32: position in ids of the first id >= t * 2^15 of the cell's
 *                            list (t = n_slabs: the end of the list)
 *   ids   [info.n_ids] u32   the lists, subspace after subspace and cell after cell, ids
 *                            ascending; each list starts at a multiple of 4 and is padded to the
 *                            next one with 0xffffffff.
 * The lists are built on the device (a stable counting sort of the ids by cell code, one slab
 * of 2^15 ids at a time). Synchronises the device.
 */
int taco_index_lists(const taco_index* index, uint32_t* sizes, uint32_t* split, uint32_t* ids);

/* taco_save_index / taco_load_index -- binary file with the parts and D (little endian).
 * Loading rebuilds the device index; taco_load_index synchronises `stream`. */
int taco_save_index(const taco_index* index, const char* path);
int taco_load_index(const char* path, int32_t keep_rows, void* stream, taco_index** out);

/* Per-kernel device time of the search path, accumulated while profiling is enabled.
 * launches[] counts kernel launches (slot 1 counts both probe kernels when the row-merge walk
 * runs before the histogram kernel; one event pair times them together).
 * Kernel slots: 0 transform (Alg. 6 step 1), 1 cell probe (Alg. 4), 2 collision counting
 * into per-range level lists (Def. 6), 3 selection and re-rank (Alg. 5, Alg. 6 step 9),
 * 4 fallback for the queries the two-pass form cannot finish (threshold below 2, or a level
 * list past its slot): the cluster kernel, or the codes fallback (TACO_OPT_CODES_FALLBACK);
 * the cluster kernel answers every query in taco_search_batch_noalloc; 5 merge of the
 * cluster kernel's lists,
 * 6 query x centroid block on the tensor cores (probe_precision TACO_PREC_BF16). */
#define TACO_NUM_KERNELS 7
typedef struct {
    int64_t launches[TACO_NUM_KERNELS];
    double ms[TACO_NUM_KERNELS];
} taco_kernel_times;

/* taco_profile_enable -- start (enable != 0) or stop recording a CUDA event pair on the
 * search stream around every kernel launch of this index. Recording adds no
 * synchronisation; events are read by taco_profile_read. */
int taco_profile_enable(taco_index* index, int32_t enable);

/* taco_profile_read -- wait for the recorded events, add their elapsed times to *out
 * (host struct, overwritten) and, if reset != 0, clear the accumulated totals. */
int taco_profile_read(taco_index* index, taco_kernel_times* out, int32_t reset);

/* ---- serving loop ---------------------------------------------------------------------
 * A server keeps an index resident and answers single-query requests (Alg. 6 per query)
 * with continuous batching: a dispatcher thread packs the requests waiting in its queue
 * into device batches and launches each on one of `slots` CUDA streams, each stream with
 * its own device workspace and pinned staging, so batches that are admitted while others
 * run overlap on the device; a completion thread hands results back as batches finish.
 * A request's result depends on that request alone (its query and parameters), never on
 * the batch it rode in. The paper has no serving loop; this is the deployment form of the
 * same search kernels.
 *
 * Admission: a request enters the queue only if fewer than queue_capacity requests are
 * held (else TACO_EAGAIN). A batch takes queued requests in arrival order while its
 * device workspace (per-query probed-cell lists, collision-count level lists, top lists
 * sized by the largest list length in the batch) fits the slot's slot_bytes and it has
 * fewer than max_batch queries. A batch is dispatched when a slot is free and either no
 * batch is running, the batch is full, or its oldest request has waited max_wait_us.
 * With use_graphs, each slot replays a CUDA graph captured per (batch-size bucket, list
 * bucket); batches are padded to the bucket with copies of their first request, whose
 * results are dropped. The index must outlive the server, must not be freed, profiled or
 * autotuned while the server runs, and may still be searched directly (taco_search_batch)
 * meanwhile.
 */
typedef struct taco_server taco_server;

typedef struct {
    int32_t max_batch;       /* queries per device batch, 1..16384 */
    int32_t slots;           /* device batches in flight at once, 1..8 */
    int32_t queue_capacity;  /* requests held at once (queued, running, or done but not yet
                                collected by taco_server_wait), >= max_batch */
    int32_t max_list;        /* largest list length a request may need: k, or for BF16
                                min(shortlist_mult * k, TACO_MAX_K); 1..TACO_MAX_K */
    int32_t precision;       /* TACO_PREC_* of every request */
    int32_t select_rule;     /* TACO_SELECT_* of every request */
    int64_t max_wait_us;     /* longest a queued request waits for its batch to fill, >= 0 */
    int64_t slot_bytes;      /* device workspace per slot; 0 = enough for max_batch queries
                                at max_list. Smaller values admit fewer queries per batch */
    int32_t use_graphs;      /* nonzero: replay captured CUDA graphs (see above) */
    int32_t probe_precision; /* taco_query_params.probe_precision of every request */
} taco_server_params;

/* Timing of one request, steady clock in nanoseconds. */
typedef struct {
    int64_t submit_ns;       /* taco_server_submit accepted it */
    int64_t dispatch_ns;     /* its batch was launched */
    int64_t done_ns;         /* its batch's results reached host memory */
    int32_t batch_size;      /* real queries in that batch */
    int32_t slot;            /* the slot (stream) that ran it */
} taco_request_info;

typedef struct {
    int64_t submitted, completed, rejected;   /* requests accepted / answered / EAGAIN */
    int64_t batches, graph_launches, graph_captures;
    int64_t max_batch_seen;                   /* largest batch launched */
    int64_t max_in_flight;                    /* most batches running at once */
    int64_t slot_bytes;                       /* device workspace per slot */
} taco_server_stats;

/*
 * taco_server_create -- start a server on `index` (the current device must be the index's).
 * Allocates every slot's stream, device workspace and pinned staging, and starts the
 * dispatcher and completion threads. Errors: TACO_EINVAL (bad parameters), TACO_ENOMEM,
 * TACO_ECUDA, TACO_ECAPACITY (slot_bytes too small for one query at max_list).
 */
int taco_server_create(const taco_index* index, const taco_server_params* params,
                       taco_server** out);

/*
 * taco_server_submit -- queue one request. query: host pointer, [d] float32 (copied before
 * return). params: host pointer; its precision and select_rule must match the server's and
 * its list length must not exceed max_list. On success *ticket names the request.
 * Returns TACO_EAGAIN when queue_capacity requests are held.
 */
int taco_server_submit(taco_server* server, const float* query, const taco_query_params* params,
                       uint64_t* ticket);

/*
 * taco_server_submit_many -- queue m requests in one call (queries: host [m][d], params: host
 * [m]; tickets: host [m] out). Takes requests in order while the queue has places, sets
 * *accepted to how many, and returns TACO_EAGAIN if that is fewer than m (the rest were not
 * queued). One lock acquisition and one wake-up for the whole burst.
 */
int taco_server_submit_many(taco_server* server, const float* queries, int64_t m,
                            const taco_query_params* params, uint64_t* tickets, int64_t* accepted);

/*
 * taco_server_wait -- wait up to timeout_us (< 0: no limit) for request `ticket`, then copy
 * its result to host buffers ids [k_stride] int64 and dists [k_stride] float32 (ascending
 * by (distance, id); -1 / +inf past min(k, |C|)) and, if info is not NULL, its timing.
 * Collecting frees the request's place in the queue; each ticket is collected once.
 * Returns TACO_ETIMEOUT if the request is not done in time (it stays queued), TACO_EINVAL
 * for an unknown or already collected ticket or k_stride < k, or the error of its batch.
 */
int taco_server_wait(taco_server* server, uint64_t ticket, int64_t timeout_us, int32_t k_stride,
                     int64_t* ids, float* dists, taco_request_info* info);

/* taco_server_get_stats -- counters since creation (host output). */
int taco_server_get_stats(taco_server* server, taco_server_stats* stats);

/*
 * taco_server_replay -- open-loop load driver over a server: submits query j (row j of the
 * host array queries [nq][d], parameters params[j]) at arrival_ns[j] nanoseconds after the
 * call starts (arrival_ns ascending; all requests already due go in one
 * taco_server_submit_many burst), retrying what the queue refuses, while the calling thread
 * collects the results in order into ids / dists [nq][k_stride] and latency_ns[nq] =
 * completion time - arrival time (queueing included). Returns after every request is
 * answered, with the first error met, if any. No other thread may collect (taco_server_wait)
 * this call's tickets.
 */
int taco_server_replay(taco_server* server, const float* queries, int64_t nq,
                       const taco_query_params* params, const int64_t* arrival_ns,
                       int32_t k_stride, int64_t* ids, float* dists, int64_t* latency_ns);

/* taco_server_destroy -- stop accepting requests, finish the batches in flight, join the
 * threads and free every slot (NULL is a no-op). Requests still queued and uncollected
 * results are dropped. No other call on the server may be running or follow. */
void taco_server_destroy(taco_server* server);

/* taco_free_index -- release an index and all its device memory (NULL is a no-op). */
void taco_free_index(taco_index* index);

/* taco_last_error -- message of the last failed call on this thread ("" if none). */
const char* taco_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TACO_H_ */

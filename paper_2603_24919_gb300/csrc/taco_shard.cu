// Id-range shards of one index. A search split over S shards, each holding a contiguous run of
// the index's id ranges (on a multi-GPU node: the id-range slice of every cell list and the
// rows of its ids, the centroids and the global cell sizes replicated), gives exactly the
// one-index result with one exchange of Alg. 5's level counts and one of the results:
//   - transform, centroid distances and probe (Alg. 6 steps 1-6) use the global cell sizes,
//     so every shard probes the same cells;
//   - each shard counts collisions in its own ranges (Def. 6; an id's SC needs only the
//     cells that hold it, and all of them list it in the id's own range);
//   - Alg. 5 runs on the level counts summed over the shards (the all-reduce of
//     [N_s + 1] counts per query), so every shard finds the same threshold;
//   - each shard re-ranks its candidates and returns its k nearest; the k nearest of the
//     shards' lists by (distance, id) are the search's (the all-gather and merge).
// Here the shards are run in one process on one device (the reduce and the merge are the
// caller's, on the host); each shard's handle owns its workspace from the count to the
// select, so the shards of a batch can be counted before any is selected.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "taco_internal.h"

using namespace taco;

struct taco_shard_search {
    taco_index* ix = nullptr;
    int shard_r0 = 0, shard_r1 = 0;
    int64_t nq = 0;
    int32_t k_stride = 0;
    taco_query_params head{};
    int kk_max = 0;
    bool per_query = false;
    int ctc = 0;
    SearchLayout lay{};
    char* ws = nullptr;          // device workspace of the batch (owned)
    int64_t* d_hist = nullptr;   // device [nq][N_s + 1]: the shard's counts, then the global ones
    bool counted = false;
    ~taco_shard_search() { cudaFree(ws); }
};

namespace {

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

SearchLaunch make_launch(const taco_shard_search* h, int phase, cudaStream_t) {
    taco_index* ix = h->ix;
    SearchLaunch L = {};
    L.ix = ix;
    L.nq = h->nq;
    L.queries = reinterpret_cast<const float*>(h->ws + h->lay.q);
    L.defaults = query_params_dev(h->head);
    L.params = h->per_query ? reinterpret_cast<const QueryParamsDev*>(h->ws + h->lay.par) : nullptr;
    L.precision = h->head.precision;
    L.kk_max = h->kk_max;
    bind_workspace(L, h->lay, h->ws);
    L.centroid_tc = h->ctc;
    L.out_ids = reinterpret_cast<int64_t*>(h->ws + h->lay.oi);
    L.out_dists = reinterpret_cast<float*>(h->ws + h->lay.od);
    L.k_stride = h->k_stride;
    L.skip_profile = true;
    L.phase = phase;
    L.shard_r0 = h->shard_r0;
    L.shard_r1 = h->shard_r1;
    L.shard_hist = h->d_hist;
    L.ghist = h->d_hist;
    return L;
}

}  // namespace

extern "C" {

int taco_shard_count(const taco_index* index, int32_t shard, int32_t n_shards, const float* queries, int64_t nq,
                     const taco_query_params* per_query, const taco_query_params* defaults, int32_t k_stride,
                     int64_t* hist, void* stream, taco_shard_search** out) {
    if (!index || !queries || !hist || !out) return fail(TACO_EINVAL, "null argument");
    *out = nullptr;
    taco_index* ix = const_cast<taco_index*>(index);
    if (nq < 1 || nq > kQueryChunk) return fail(TACO_EINVAL, "nq must be in [1, %lld]", (long long)kQueryChunk);
    if (n_shards < 1 || n_shards > ix->tp_ranges)
        return fail(TACO_EINVAL, "n_shards must be in [1, %d] (the index's id ranges)", ix->tp_ranges);
    if (shard < 0 || shard >= n_shards) return fail(TACO_EINVAL, "shard %d not in [0, %d)", shard, n_shards);
    if (!per_query && !defaults) return fail(TACO_EINVAL, "per_query and defaults are both NULL");
    if (k_stride < 1) return fail(TACO_EINVAL, "k_stride < 1");
    const taco_query_params& head = per_query ? per_query[0] : *defaults;
    int kk_max = 0;
    if (per_query) {
        for (int64_t j = 0; j < nq; ++j) {
            if (int rc = check_query_params(per_query[j], k_stride)) return rc;
            if (per_query[j].precision != head.precision || per_query[j].select_rule != head.select_rule ||
                per_query[j].probe_precision != head.probe_precision)
                return fail(TACO_EINVAL, "precision, probe_precision and select_rule must be uniform in a batch");
            kk_max = std::max(kk_max, query_list_len(per_query[j]));
        }
    } else {
        if (int rc = check_query_params(head, k_stride)) return rc;
        kk_max = query_list_len(head);
    }
    if (head.precision == TACO_PREC_BF16 && !ix->d_data_bf16)
        return fail(TACO_EINVAL, "BF16 search needs an index with BF16 rows (TACO_ROWS_BF16)");
    if (head.precision == TACO_PREC_FP8 && !ix->d_data_fp8)
        return fail(TACO_EINVAL, "FP8 search needs an index with FP8 rows (TACO_ROWS_FP8)");
    const int ctc = head.probe_precision == TACO_PREC_BF16 ? 1 : (head.probe_precision == TACO_PREC_FP8 ? 2 : 0);
    if (ctc && !ix->d_cent_tc) return fail(TACO_EINVAL, "this index has no tensor-core centroid block");
    int cur_dev = 0;
    TACO_CUDA(cudaGetDevice(&cur_dev));
    if (cur_dev != ix->device) return fail(TACO_EINVAL, "current device %d is not the index's device %d", cur_dev, ix->device);
    if (int rc = ensure_device_codes(ix)) return rc;   // flagged queries take the codes fallback
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    taco_shard_search* h = new (std::nothrow) taco_shard_search();
    if (!h) return fail(TACO_ENOMEM, "host allocation failed");
    h->ix = ix;
    // shard s holds ranges [s R / S, (s + 1) R / S) of the index's R id ranges
    h->shard_r0 = int(int64_t(shard) * ix->tp_ranges / n_shards);
    h->shard_r1 = int(int64_t(shard + 1) * ix->tp_ranges / n_shards);
    h->nq = nq;
    h->k_stride = k_stride;
    h->head = head;
    h->kk_max = kk_max;
    h->per_query = per_query != nullptr;
    h->ctc = ctc;
    // queries, parameters and results always staged in the handle's workspace
    h->lay = plan_search(ix, nq, kk_max, per_query ? nq : 0, true, true, true, k_stride, ctc != 0);
    const size_t hist_off = round256(h->lay.total);
    const size_t hist_bytes = size_t(nq) * (ix->Ns + 1) * sizeof(int64_t);
    const cudaError_t ea = cudaMalloc(&h->ws, hist_off + hist_bytes);
    if (ea != cudaSuccess) {
        delete h;
        return cuda_fail(ea, "shard workspace", __FILE__, __LINE__);
    }
    h->d_hist = reinterpret_cast<int64_t*>(h->ws + hist_off);
    auto bail = [&](int rc) {
        delete h;
        return rc;
    };
    const cudaMemcpyKind qk = is_device_pointer(queries) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(h->ws + h->lay.q, queries, size_t(nq) * ix->d * sizeof(float), qk, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "shard queries", __FILE__, __LINE__));
    if (per_query) {
        QueryParamsDev* hp = new (std::nothrow) QueryParamsDev[size_t(nq)];
        if (!hp) return bail(fail(TACO_ENOMEM, "host allocation failed"));
        for (int64_t j = 0; j < nq; ++j) hp[j] = query_params_dev(per_query[j]);
        e = cudaMemcpyAsync(h->ws + h->lay.par, hp, size_t(nq) * sizeof(QueryParamsDev), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // hp dies here
        delete[] hp;
        if (e != cudaSuccess) return bail(cuda_fail(e, "shard parameters", __FILE__, __LINE__));
    }
    {
        std::lock_guard<std::mutex> lock(ix->ws_mu);   // the layout (tuned) must not change meanwhile
        if (int rc = run_search_chunk(make_launch(h, 1, st), st)) return bail(rc);
    }
    const cudaMemcpyKind hk = is_device_pointer(hist) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    e = cudaMemcpyAsync(hist, h->d_hist, hist_bytes, hk, st);
    if (e == cudaSuccess && hk == cudaMemcpyDeviceToHost) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "shard counts", __FILE__, __LINE__));
    h->counted = true;
    *out = h;
    return TACO_OK;
}

int taco_shard_select(taco_shard_search* h, const int64_t* global_hist, int64_t* out_ids, float* out_dists,
                      void* stream) {
    if (!h || !global_hist || !out_ids || !out_dists) return fail(TACO_EINVAL, "null argument");
    if (!h->counted) return fail(TACO_EINVAL, "the shard has not been counted");
    taco_index* ix = h->ix;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t hist_bytes = size_t(h->nq) * (ix->Ns + 1) * sizeof(int64_t);
    const cudaMemcpyKind gk = is_device_pointer(global_hist) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TACO_CUDA(cudaMemcpyAsync(h->d_hist, global_hist, hist_bytes, gk, st));
    {
        std::lock_guard<std::mutex> lock(ix->ws_mu);
        if (int rc = run_search_chunk(make_launch(h, 2, st), st)) return rc;
    }
    const size_t n_out = size_t(h->nq) * h->k_stride;
    const cudaMemcpyKind ik = is_device_pointer(out_ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind dk = is_device_pointer(out_dists) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TACO_CUDA(cudaMemcpyAsync(out_ids, h->ws + h->lay.oi, n_out * sizeof(int64_t), ik, st));
    TACO_CUDA(cudaMemcpyAsync(out_dists, h->ws + h->lay.od, n_out * sizeof(float), dk, st));
    // the global counts arrive before the select reads them; host copies are complete on return
    TACO_CUDA(cudaStreamSynchronize(st));
    return TACO_OK;
}

int taco_shard_free(taco_shard_search* h) {
    delete h;   // cudaFree of the workspace waits for work still using it
    return TACO_OK;
}

}  // extern "C"

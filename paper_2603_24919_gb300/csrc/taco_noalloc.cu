// Search entry point for callers that must not allocate device memory.
//
// taco_search_batch keeps its per-call scratch (transformed queries, probed-cell lists)
// in a workspace that it grows with cudaMalloc. Some callers cannot allow that: a process
// whose device memory is carved up in advance by its own pool or by a framework that owns
// every allocation, or a latency-bound serving loop where a cudaMalloc (which may
// synchronise the device and stall other streams) is not acceptable on the request path.
// taco_search_batch_noalloc runs the same kernels with their scratch in the fixed array
// below instead, and calls no allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "taco_internal.h"

namespace taco {
namespace {

// The scratch of this entry point. Every GPU that loads the library holds it until the
// process exits. All calls share it.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TACO_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        TACO_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TACO_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace taco

using namespace taco;

extern "C" int taco_search_batch_noalloc(const taco_index* index, const float* queries, int64_t nq,
                                         const taco_query_params* params, int32_t k_stride,
                                         int64_t* out_ids, float* out_dists, void* stream) {
    if (!index || !params) return fail(TACO_EINVAL, "null index or params");
    if (nq < 0) return fail(TACO_EINVAL, "nq < 0");
    if (nq == 0) return TACO_OK;
    if (!queries || !out_ids || !out_dists) return fail(TACO_EINVAL, "null queries or outputs");
    if (!is_device_pointer(queries) || !is_device_pointer(out_ids) || !is_device_pointer(out_dists))
        return fail(TACO_EINVAL, "taco_search_batch_noalloc takes device pointers only");
    const taco_query_params& q = *params;
    // the checks of taco_search_batch, then what this entry point does not support
    if (int rc = check_query_params(q, k_stride)) return rc;
    if (q.precision == TACO_PREC_FP8)
        return fail(TACO_EINVAL, "taco_search_batch_noalloc re-ranks with FP32 or BF16 rows only");
    if (q.probe_precision != TACO_PREC_FP32)
        return fail(TACO_EINVAL, "taco_search_batch_noalloc computes centroid distances in FP32 only");
    if (q.precision == TACO_PREC_BF16 && !index->d_data_bf16)
        return fail(TACO_EINVAL, "BF16 needs an index with BF16 rows");
    if (nq > kQueryChunk)
        return fail(TACO_ECAPACITY, "nq = %lld exceeds %lld queries per call", (long long)nq,
                    (long long)kQueryChunk);
    taco_index* ix = const_cast<taco_index*>(index);
    if (ix->cluster == 0)
        return fail(TACO_ECAPACITY, "n = %lld is too large for the single-pass kernel of this entry point",
                    (long long)ix->n);
    int dev = 0;
    TACO_CUDA(cudaGetDevice(&dev));
    if (dev != ix->device) return fail(TACO_EINVAL, "current device %d is not the index's device %d", dev, ix->device);
    // scratch layout per query, as in the allocating entry point
    const size_t per_qt = up256(size_t(nq) * ix->Dp * 4);
    const size_t per_cells = up256(size_t(nq) * ix->Ns * ix->K * 2);
    const size_t per_nc = up256(size_t(nq) * ix->Ns * 4);
    const size_t per_ret = up256(size_t(nq) * ix->Ns * 8);
    const int kk = query_list_len(q);
    const size_t per_list = up256(size_t(nq) * ix->cluster * kListsPerCta * kk * 4);
    const size_t need = per_qt + per_cells + per_nc + per_ret + 2 * per_list;
    if (need > kNoAllocScratchBytes) {
        const size_t one = size_t(ix->Dp) * 4 + size_t(ix->Ns) * ix->K * 2 + size_t(ix->Ns) * 12 +
                           size_t(ix->cluster) * kListsPerCta * kk * 8;   // per query, unrounded
        return fail(TACO_ECAPACITY,
                    "nq = %lld needs %zu bytes of scratch; the fixed scratch holds %zu bytes "
                    "(about %zu queries of this index per call)",
                    (long long)nq, need, kNoAllocScratchBytes, kNoAllocScratchBytes / one);
    }
    void* base = nullptr;
    if (int rc = scratch_address(dev, &base)) return rc;
    if (ix->prof.enabled) return fail(TACO_EINVAL, "disable profiling before taco_search_batch_noalloc");
    char* b = static_cast<char*>(base);
    SearchLaunch L = {};
    L.ix = ix;
    L.queries = queries;
    L.nq = nq;
    const QueryParamsDev d = query_params_dev(q);
    L.defaults = d;
    L.params = nullptr;
    L.precision = q.precision;
    L.kk_max = d.kk;
    L.qt = reinterpret_cast<float*>(b);
    L.cells = reinterpret_cast<uint16_t*>(b + per_qt);
    L.ncells = reinterpret_cast<int32_t*>(b + per_qt + per_cells);
    L.retrieved = reinterpret_cast<int64_t*>(b + per_qt + per_cells + per_nc);
    L.lists_d = reinterpret_cast<float*>(b + per_qt + per_cells + per_nc + per_ret);
    L.lists_i = reinterpret_cast<uint32_t*>(b + per_qt + per_cells + per_nc + per_ret + per_list);
    L.out_ids = out_ids;
    L.out_dists = out_dists;
    L.k_stride = k_stride;
    return run_search_chunk(L, static_cast<cudaStream_t>(stream));
}

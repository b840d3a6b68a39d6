// Autotuner of the search's launch layout: times real searches of a sample batch on the
// caller's stream and keeps the fastest choice of
//   - the counter layout of the two-pass collision counting: slabs of 2^15 ids per id range
//     (16 KB of 4-bit counters per slab in shared memory; fewer slabs per range = more,
//     smaller units per query and more resident CTAs; more = fewer units, longer walks),
//   - the lanes that gather one candidate row in the select / re-rank pass (4 .. 32),
//   - the threads of a counting CTA (256, 512 or 1024) and the depth of its walk (2, 4 or 8
//     loads of four ids in flight per lane),
//   - whether small budgets are probed by the row-merge walk or always by the histogram
//     kernel.
// The choices change no result beyond the summation order of a candidate's FP32 distance
// (the lanes split a row differently): the counting and selection are exact integer work.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "taco_internal.h"

using namespace taco;

namespace {

struct Choice {
    int spc, ranges, lanes, walk, warps, unroll;
};

void apply(taco_index* ix, const Choice& c, int rk) {
    ix->tp_spc = c.spc;
    ix->tp_ranges = c.ranges;
    ix->tp_lanes[rk] = c.lanes;
    ix->tp_walk = c.walk;
    ix->tp_count_warps = c.warps;
    ix->tp_walk_unroll = c.unroll;
}

// Mean ms of one search of the sample after one untimed search; <0 on failure.
int time_search(const taco_index* ix, const float* q, int64_t nq, const taco_query_params& p, int64_t* ids,
                float* dists, int reps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
    if (int rc = taco_search_batch(ix, q, nq, nullptr, &p, p.k, ids, dists, st)) return rc;
    TACO_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r)
        if (int rc = taco_search_batch(ix, q, nq, nullptr, &p, p.k, ids, dists, st)) return rc;
    TACO_CUDA(cudaEventRecord(e1, st));
    TACO_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    TACO_CUDA(cudaEventElapsedTime(&t, e0, e1));
    *ms = double(t) / reps;
    return TACO_OK;
}

}  // namespace

extern "C" int taco_autotune(taco_index* ix, const float* queries, int64_t nq, const taco_query_params* params,
                             int32_t reps, void* stream, taco_tune_result* out) {
    if (!ix || !params || !out) return fail(TACO_EINVAL, "null argument");
    const int rk = params->precision == TACO_PREC_FP8 ? 2 : (params->precision == TACO_PREC_BF16 ? 1 : 0);
    const Choice defaults{ix->tp_spc0, ix->tp_ranges0, 0, -1, 16, 4};
    if (reps <= 0) {   // back to the defaults
        apply(ix, defaults, rk);
        for (int& l : ix->tp_lanes) l = 0;
        *out = taco_tune_result{defaults.spc, defaults.ranges, 0, -1, 16, 4, 0.0, 0.0, 0, 0};
        return TACO_OK;
    }
    if (!queries || nq < 1 || !is_device_pointer(queries)) return fail(TACO_EINVAL, "need device queries, nq >= 1");
    if (int rc = check_query_params(*params, params->k)) return rc;
    if (ix->prof.enabled) return fail(TACO_EINVAL, "disable profiling before taco_autotune");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t* ids = nullptr;
    float* dists = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct Guard {
        int64_t** i;
        float** d;
        cudaEvent_t* a;
        cudaEvent_t* b;
        ~Guard() {
            cudaFree(*i);
            cudaFree(*d);
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
        }
    } guard{&ids, &dists, &e0, &e1};
    TACO_CUDA(cudaMalloc(&ids, size_t(nq) * params->k * 8));
    TACO_CUDA(cudaMalloc(&dists, size_t(nq) * params->k * 4));
    TACO_CUDA(cudaEventCreate(&e0));
    TACO_CUDA(cudaEventCreate(&e1));

    Choice cur{ix->tp_spc, ix->tp_ranges, ix->tp_lanes[rk], ix->tp_walk, ix->tp_count_warps, ix->tp_walk_unroll};
    double ms_before = 0.0;
    if (int rc = time_search(ix, queries, nq, *params, ids, dists, reps, st, e0, e1, &ms_before)) return rc;
    double best = ms_before;
    int trials = 1;
    auto trial = [&](const Choice& c) -> int {
        apply(ix, c, rk);
        double ms = 0.0;
        int rc = time_search(ix, queries, nq, *params, ids, dists, reps, st, e0, e1, &ms);
        ++trials;
        if (rc == TACO_ECAPACITY) return TACO_OK;   // this layout does not fit: skip it
        if (rc) return rc;
        if (ms < best) {
            best = ms;
            cur = c;
        }
        return TACO_OK;
    };
    // 1. counter layout: slabs per range (16 KB each at 4 bits) up to what a CTA's shared
    //    memory holds (up to 5 slabs, two 512-thread counting CTAs share an SM); 15 slabs at
    //    3 bits where N_s <= 7
    for (int spc : {1, 2, 4, 5, 8, 12, 15}) {
        if (spc > ix->n_slabs || spc == cur.spc || (spc > 12 && ix->Ns > 7)) continue;
        Choice c = cur;
        c.spc = spc;
        c.ranges = (ix->n_slabs + spc - 1) / spc;
        if (int rc = trial(c)) {
            apply(ix, cur, rk);
            return rc;
        }
    }
    // 1b. threads of the counting CTA (256 or 512: two CTAs per SM where the counters fit;
    //     1024: one) and the depth of its walk (2, 4 or 8 chunk loads in flight per lane; 8
    //     only with 512 threads)
    for (const int2 v : {make_int2(16, 4), make_int2(16, 2), make_int2(8, 2), make_int2(8, 4),
                         make_int2(32, 2), make_int2(32, 4), make_int2(16, 8)}) {
        if (v.x == cur.warps && v.y == cur.unroll) continue;
        Choice c = cur;
        c.warps = v.x;
        c.unroll = v.y;
        if (int rc = trial(c)) {
            apply(ix, cur, rk);
            return rc;
        }
    }
    // 2. lanes per candidate row of the re-rank
    for (int lanes : {4, 8, 16, 32}) {
        if (lanes == cur.lanes) continue;
        Choice c = cur;
        c.lanes = lanes;
        if (int rc = trial(c)) {
            apply(ix, cur, rk);
            return rc;
        }
    }
    // 3. probe strategy
    for (int walk : {-1, 0}) {
        if (walk == cur.walk) continue;
        Choice c = cur;
        c.walk = walk;
        if (int rc = trial(c)) {
            apply(ix, cur, rk);
            return rc;
        }
    }
    apply(ix, cur, rk);
    *out = taco_tune_result{cur.spc, cur.ranges, cur.lanes, cur.walk, cur.warps, cur.unroll, ms_before, best, trials, 0};
    return TACO_OK;
}

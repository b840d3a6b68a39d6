// Serving loop over a resident index: continuous batching of single-query requests.
//
// Requests enter a bounded queue (taco_server_submit). A dispatcher thread packs queued
// requests, oldest first, into a device batch for a free slot (a CUDA stream with its own
// device workspace and pinned staging), within the slot's workspace bytes, and launches
// the search kernels on that stream: host->device copy of the queries and per-query
// parameters, the whole Alg. 6 pipeline (run_search_chunk), device->host copy of the top
// lists, and an event. While a batch runs, new requests keep queueing and the next batch is
// launched on another slot as soon as one is free, so batches overlap on the device. A
// completion thread waits for the slots' events in launch order and hands each request its
// rows. Each query's answer depends on that query and its parameters alone.
//
// With CUDA graphs on, a batch is padded to a size bucket (powers of two up to 64, then
// multiples of 64) and its list length to the bucket of the kernel's register lists
// (32 / 128 / 512); the first batch of a (size, list) bucket on a slot runs directly (it
// also sets the kernels' launch attributes on the dispatcher thread), the second captures
// the same launch sequence into a graph, and later ones replay it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <utility>
#include <vector>

#include "taco_internal.h"

using namespace taco;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr int kMaxSlots = 8;
constexpr int kTicketShift = 24;   // ticket = sequence << 24 | queue position
constexpr int kMaxQueue = 1 << kTicketShift;

enum RequestState : int { kFree = 0, kQueued, kRunning, kDone };

struct Request {
    uint64_t ticket = 0;
    int state = kFree;
    taco_query_params p = {};
    int kk = 0;        // list length the request needs
    int rc = TACO_OK;
    taco_request_info info = {};
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    char* ws = nullptr;                // device workspace
    float* h_q = nullptr;              // pinned [max_batch][d]
    QueryParamsDev* h_p = nullptr;     // pinned [max_batch]
    int64_t* h_ids = nullptr;          // pinned [max_batch][max_list]
    float* h_d = nullptr;              // pinned [max_batch][max_list]
    bool busy = false;
    int rc = TACO_OK;
    int64_t dispatch_ns = 0;
    std::vector<int> reqs;             // queue positions of the batch's real requests
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    std::set<std::pair<int, int>> seen;
};

int size_bucket(int n, int max_batch) {
    int b = 1;
    if (n <= 64) {
        while (b < n) b <<= 1;
    } else {
        b = (n + 63) / 64 * 64;
    }
    return std::min(b, max_batch);
}

int list_bucket(int kk) { return kk <= 32 ? 32 : (kk <= 128 ? 128 : TACO_MAX_K); }

}  // namespace

struct taco_server {
    const taco_index* ix = nullptr;
    taco_server_params p = {};
    int d = 0;
    int k_out = 0;                     // row length of the staged results (= max_list)
    size_t ws_bytes = 0;               // device workspace allocated per slot
    std::mutex mu;
    std::condition_variable cv_dispatch;   // queue or slots changed
    std::condition_variable cv_complete;   // a batch was launched
    std::condition_variable cv_done;       // a request finished
    std::vector<Request> reqs;
    std::vector<float> q_store;        // [queue_capacity][d]
    std::vector<int64_t> id_store;     // [queue_capacity][max_list]
    std::vector<float> d_store;        // [queue_capacity][max_list]
    std::vector<int> free_pos;
    std::deque<int> pending;
    std::deque<int> inflight;          // slot ids in launch order
    Slot slots[kMaxSlots];
    uint64_t seq = 0;
    bool stop = false;
    bool dispatch_exited = false;
    int fatal = TACO_OK;
    taco_server_stats st = {};
    std::thread dispatcher, completer;
};

namespace {

size_t batch_bytes(const taco_server* S, int n, int kk) {
    const int nl = S->p.use_graphs ? size_bucket(n, S->p.max_batch) : n;
    const int kl = S->p.use_graphs ? list_bucket(kk) : kk;
    return plan_search(S->ix, nl, kl, nl, true, true, true, S->k_out, S->p.probe_precision != TACO_PREC_FP32).total;
}

// Enqueue one batch of nl staged queries on the slot's stream (also used under capture).
int enqueue_batch(taco_server* S, Slot& sl, const SearchLayout& lay, int nl, int kl) {
    const taco_index* ix = S->ix;
    char* wb = sl.ws;
    TACO_CUDA(cudaMemcpyAsync(wb + lay.q, sl.h_q, size_t(nl) * S->d * 4, cudaMemcpyHostToDevice, sl.stream));
    TACO_CUDA(cudaMemcpyAsync(wb + lay.par, sl.h_p, size_t(nl) * sizeof(QueryParamsDev), cudaMemcpyHostToDevice,
                              sl.stream));
    SearchLaunch L = {};
    L.ix = ix;
    L.queries = reinterpret_cast<const float*>(wb + lay.q);
    L.nq = nl;
    L.defaults = sl.h_p[0];
    L.params = reinterpret_cast<const QueryParamsDev*>(wb + lay.par);
    L.precision = S->p.precision;
    L.kk_max = kl;
    bind_workspace(L, lay, wb);
    L.centroid_tc = S->p.probe_precision == TACO_PREC_BF16 ? 1 : (S->p.probe_precision == TACO_PREC_FP8 ? 2 : 0);
    L.out_ids = reinterpret_cast<int64_t*>(wb + lay.oi);
    L.out_dists = reinterpret_cast<float*>(wb + lay.od);
    L.k_stride = S->k_out;
    L.skip_profile = true;
    if (int rc = run_search_chunk(L, sl.stream)) return rc;
    TACO_CUDA(cudaMemcpyAsync(sl.h_ids, wb + lay.oi, size_t(nl) * S->k_out * 8, cudaMemcpyDeviceToHost, sl.stream));
    TACO_CUDA(cudaMemcpyAsync(sl.h_d, wb + lay.od, size_t(nl) * S->k_out * 4, cudaMemcpyDeviceToHost, sl.stream));
    return TACO_OK;
}

// Stage the batch's queries and parameters and launch it (directly or as a graph).
int launch_batch(taco_server* S, Slot& sl, int kk_max, int64_t* n_launch, int64_t* n_capture) {
    const int n = int(sl.reqs.size());
    const bool graphs = S->p.use_graphs != 0;
    const int nl = graphs ? size_bucket(n, S->p.max_batch) : n;
    const int kl = graphs ? list_bucket(kk_max) : kk_max;
    for (int j = 0; j < nl; ++j) {
        const int src = sl.reqs[j < n ? j : 0];   // padding repeats the first request
        std::memcpy(sl.h_q + size_t(j) * S->d, S->q_store.data() + size_t(src) * S->d, size_t(S->d) * 4);
        sl.h_p[j] = query_params_dev(S->reqs[src].p);
    }
    const SearchLayout lay = plan_search(S->ix, nl, kl, nl, true, true, true, S->k_out,
                                         S->p.probe_precision != TACO_PREC_FP32);
    const std::pair<int, int> key(nl, kl);
    auto it = sl.graphs.find(key);
    if (it != sl.graphs.end()) {
        TACO_CUDA(cudaGraphLaunch(it->second, sl.stream));
        ++*n_launch;
    } else if (graphs && sl.seen.count(key)) {
        TACO_CUDA(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_batch(S, sl, lay, nl, kl);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(sl.stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture", __FILE__, __LINE__);
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        sl.graphs[key] = ge;
        ++*n_capture;
        TACO_CUDA(cudaGraphLaunch(ge, sl.stream));
        ++*n_launch;
    } else {
        if (int rc = enqueue_batch(S, sl, lay, nl, kl)) return rc;
        if (graphs) sl.seen.insert(key);
    }
    TACO_CUDA(cudaEventRecord(sl.done, sl.stream));
    return TACO_OK;
}

int free_slot(const taco_server* S) {
    for (int i = 0; i < S->p.slots; ++i)
        if (!S->slots[i].busy) return i;
    return -1;
}

void finish_requests(taco_server* S, Slot& sl, int rc, int64_t done_ns, bool copy) {
    const int n = int(sl.reqs.size());
    for (int j = 0; j < n; ++j) {
        const int r = sl.reqs[j];
        Request& R = S->reqs[r];
        if (copy) {
            std::memcpy(S->id_store.data() + size_t(r) * S->k_out, sl.h_ids + size_t(j) * S->k_out,
                        size_t(S->k_out) * 8);
            std::memcpy(S->d_store.data() + size_t(r) * S->k_out, sl.h_d + size_t(j) * S->k_out,
                        size_t(S->k_out) * 4);
        }
        R.rc = rc;
        R.info.dispatch_ns = sl.dispatch_ns;
        R.info.done_ns = done_ns;
        R.info.batch_size = n;
        R.info.slot = int(&sl - S->slots);
        R.state = kDone;
    }
    S->st.completed += n;
    sl.reqs.clear();
    sl.busy = false;
}

void dispatch_loop(taco_server* S) {
    cudaSetDevice(S->ix->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_dispatch.wait(lk, [&] { return S->stop || (!S->pending.empty() && free_slot(S) >= 0); });
        if (S->pending.empty() || free_slot(S) < 0) {
            if (S->stop) break;
            continue;
        }
        // batching window: while another batch runs, wait for the batch to fill or its
        // oldest request to reach max_wait_us
        if (!S->inflight.empty() && int(S->pending.size()) < S->p.max_batch && !S->stop) {
            const int64_t deadline = S->reqs[S->pending.front()].info.submit_ns + S->p.max_wait_us * 1000;
            const int64_t now = now_ns();
            if (now < deadline) {
                S->cv_dispatch.wait_for(lk, std::chrono::nanoseconds(deadline - now));
                continue;
            }
        }
        const int si = free_slot(S);
        Slot& sl = S->slots[si];
        int kk_max = 0;
        sl.reqs.clear();
        while (!S->pending.empty() && int(sl.reqs.size()) < S->p.max_batch) {
            const int r = S->pending.front();
            const int kk2 = std::max(kk_max, S->reqs[r].kk);
            if (batch_bytes(S, int(sl.reqs.size()) + 1, kk2) > S->ws_bytes) {
                if (!sl.reqs.empty()) break;
                // not even alone (the index's layout grew since the server started)
                S->pending.pop_front();
                Request& R = S->reqs[r];
                R.rc = fail(TACO_ECAPACITY, "a request no longer fits the slot workspace");
                R.info.dispatch_ns = R.info.done_ns = now_ns();
                R.state = kDone;
                S->st.completed++;
                S->cv_done.notify_all();
                continue;
            }
            sl.reqs.push_back(r);
            kk_max = kk2;
            S->pending.pop_front();
            S->reqs[r].state = kRunning;
        }
        if (sl.reqs.empty()) continue;   // every request taken was refused
        sl.busy = true;
        sl.dispatch_ns = now_ns();
        const int nb = int(sl.reqs.size());
        const int fatal = S->fatal;
        lk.unlock();
        int64_t n_launch = 0, n_capture = 0;
        const int rc = fatal ? fatal : launch_batch(S, sl, kk_max, &n_launch, &n_capture);
        lk.lock();
        S->st.graph_launches += n_launch;
        S->st.graph_captures += n_capture;
        if (rc != TACO_OK) {
            if (!S->fatal) S->fatal = rc;
            finish_requests(S, sl, rc, now_ns(), false);
            S->cv_done.notify_all();
            continue;
        }
        S->st.batches++;
        S->st.max_batch_seen = std::max<int64_t>(S->st.max_batch_seen, nb);
        S->inflight.push_back(si);
        S->st.max_in_flight = std::max<int64_t>(S->st.max_in_flight, int64_t(S->inflight.size()));
        S->cv_complete.notify_one();
    }
    S->dispatch_exited = true;
    S->cv_complete.notify_all();
}

void complete_loop(taco_server* S) {
    cudaSetDevice(S->ix->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_complete.wait(lk, [&] { return !S->inflight.empty() || S->dispatch_exited; });
        if (S->inflight.empty()) break;
        const int si = S->inflight.front();
        Slot& sl = S->slots[si];
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(sl.done);
        const int64_t t = now_ns();
        lk.lock();
        S->inflight.pop_front();
        const int rc = e == cudaSuccess ? TACO_OK : cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
        if (rc && !S->fatal) S->fatal = rc;
        finish_requests(S, sl, rc, t, rc == TACO_OK);
        S->cv_done.notify_all();
        S->cv_dispatch.notify_one();
    }
}

void release_slots(taco_server* S) {
    for (Slot& sl : S->slots) {
        for (auto& g : sl.graphs) cudaGraphExecDestroy(g.second);
        sl.graphs.clear();
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFree(sl.ws);
        cudaFreeHost(sl.h_q);
        cudaFreeHost(sl.h_p);
        cudaFreeHost(sl.h_ids);
        cudaFreeHost(sl.h_d);
        sl = Slot();
    }
}

int check_request(const taco_server* S, const taco_query_params& q) {
    if (int rc = check_query_params(q, TACO_MAX_K)) return rc;
    if (q.precision != S->p.precision || q.select_rule != S->p.select_rule ||
        q.probe_precision != S->p.probe_precision)
        return fail(TACO_EINVAL, "precision, probe_precision and select_rule must match the server's");
    if (query_list_len(q) > S->p.max_list)
        return fail(TACO_EINVAL, "list length %d exceeds the server's max_list %d", query_list_len(q), S->p.max_list);
    return TACO_OK;
}

}  // namespace

extern "C" {

int taco_server_create(const taco_index* index, const taco_server_params* params, taco_server** out) {
    if (!index || !params || !out) return fail(TACO_EINVAL, "null argument");
    *out = nullptr;
    const taco_server_params& p = *params;
    if (p.max_batch < 1 || p.max_batch > kQueryChunk) return fail(TACO_EINVAL, "max_batch must be in [1, %lld]", (long long)kQueryChunk);
    if (p.slots < 1 || p.slots > kMaxSlots) return fail(TACO_EINVAL, "slots must be in [1, %d]", kMaxSlots);
    if (p.queue_capacity < p.max_batch || p.queue_capacity >= kMaxQueue)
        return fail(TACO_EINVAL, "queue_capacity must be in [max_batch, %d)", kMaxQueue);
    if (p.max_list < 1 || p.max_list > TACO_MAX_K) return fail(TACO_EINVAL, "max_list must be in [1, %d]", TACO_MAX_K);
    if (p.precision != TACO_PREC_FP32 && p.precision != TACO_PREC_BF16 && p.precision != TACO_PREC_FP8)
        return fail(TACO_EINVAL, "unknown precision");
    if ((p.precision == TACO_PREC_BF16 && !index->d_data_bf16) || (p.precision == TACO_PREC_FP8 && !index->d_data_fp8))
        return fail(TACO_EINVAL, "the index has no row copy for the server's precision");
    if (p.select_rule != TACO_SELECT_LITERAL && p.select_rule != TACO_SELECT_PROSE)
        return fail(TACO_EINVAL, "unknown select_rule");
    if (p.max_wait_us < 0 || p.slot_bytes < 0) return fail(TACO_EINVAL, "bad max_wait_us or slot_bytes");
    if (p.probe_precision != TACO_PREC_FP32 && p.probe_precision != TACO_PREC_BF16 &&
        p.probe_precision != TACO_PREC_FP8)
        return fail(TACO_EINVAL, "probe_precision must be TACO_PREC_FP32, TACO_PREC_BF16 or TACO_PREC_FP8");
    if (p.probe_precision != TACO_PREC_FP32 && !index->d_cent_tc)
        return fail(TACO_EINVAL, "this index has no tensor-core centroid block");
    int dev = 0;
    TACO_CUDA(cudaGetDevice(&dev));
    if (dev != index->device) return fail(TACO_EINVAL, "current device %d is not the index's device %d", dev, index->device);
    taco_server* S = new (std::nothrow) taco_server();
    if (!S) return fail(TACO_ENOMEM, "host allocation failed");
    S->ix = index;
    S->p = p;
    S->d = index->d;
    S->k_out = p.max_list;
    const size_t worst = batch_bytes(S, p.max_batch, p.max_list);
    if (S->p.slot_bytes == 0) S->p.slot_bytes = int64_t(worst);
    if (size_t(S->p.slot_bytes) < batch_bytes(S, 1, p.max_list)) {
        delete S;
        return fail(TACO_ECAPACITY, "slot_bytes %lld cannot hold one query at max_list %d",
                    (long long)p.slot_bytes, p.max_list);
    }
    const size_t ws_bytes = std::min(size_t(S->p.slot_bytes), worst);
    S->ws_bytes = ws_bytes;
    S->st.slot_bytes = int64_t(ws_bytes);
    try {
        S->reqs.resize(size_t(p.queue_capacity));
        S->q_store.resize(size_t(p.queue_capacity) * S->d);
        S->id_store.resize(size_t(p.queue_capacity) * S->k_out);
        S->d_store.resize(size_t(p.queue_capacity) * S->k_out);
        S->free_pos.reserve(size_t(p.queue_capacity));
    } catch (...) {
        delete S;
        return fail(TACO_ENOMEM, "host allocation of the request queue failed");
    }
    for (int i = p.queue_capacity - 1; i >= 0; --i) S->free_pos.push_back(i);
    for (int i = 0; i < p.slots; ++i) {
        Slot& sl = S->slots[i];
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.ws, ws_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_q, size_t(p.max_batch) * S->d * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_p, size_t(p.max_batch) * sizeof(QueryParamsDev));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_ids, size_t(p.max_batch) * S->k_out * 8);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_d, size_t(p.max_batch) * S->k_out * 4);
        if (e != cudaSuccess) {
            release_slots(S);
            delete S;
            return cuda_fail(e, "server slot allocation", __FILE__, __LINE__);
        }
    }
    try {
        S->dispatcher = std::thread(dispatch_loop, S);
        S->completer = std::thread(complete_loop, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            if (!S->dispatcher.joinable()) S->dispatch_exited = true;
        }
        S->cv_dispatch.notify_all();
        S->cv_complete.notify_all();
        if (S->dispatcher.joinable()) S->dispatcher.join();
        if (S->completer.joinable()) S->completer.join();
        release_slots(S);
        delete S;
        return fail(TACO_ENOMEM, "could not start the server threads");
    }
    *out = S;
    return TACO_OK;
}

namespace {

// Queue requests [0, m) under the lock while places are free; returns how many.
int64_t enqueue_locked(taco_server* S, const float* queries, int64_t m, const taco_query_params* params,
                       uint64_t* tickets) {
    const int64_t t = now_ns();
    int64_t j = 0;
    for (; j < m && !S->free_pos.empty(); ++j) {
        const int r = S->free_pos.back();
        S->free_pos.pop_back();
        Request& R = S->reqs[r];
        R.ticket = (++S->seq << kTicketShift) | uint64_t(r);
        R.state = kQueued;
        R.p = params[j];
        R.kk = query_list_len(params[j]);
        R.rc = TACO_OK;
        R.info = taco_request_info{};
        R.info.submit_ns = t;
        std::memcpy(S->q_store.data() + size_t(r) * S->d, queries + size_t(j) * S->d, size_t(S->d) * 4);
        S->pending.push_back(r);
        tickets[j] = R.ticket;
    }
    S->st.submitted += j;
    return j;
}

}  // namespace

int taco_server_submit(taco_server* S, const float* query, const taco_query_params* params, uint64_t* ticket) {
    if (!S || !query || !params || !ticket) return fail(TACO_EINVAL, "null argument");
    if (int rc = check_request(S, *params)) return rc;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop) return fail(TACO_EINVAL, "the server is stopping");
    if (S->fatal) return fail(S->fatal, "the server stopped after a device error");
    if (enqueue_locked(S, query, 1, params, ticket) == 0) {
        S->st.rejected++;
        return fail(TACO_EAGAIN, "the request queue is full (%d requests held)", S->p.queue_capacity);
    }
    lk.unlock();
    S->cv_dispatch.notify_one();
    return TACO_OK;
}

int taco_server_submit_many(taco_server* S, const float* queries, int64_t m, const taco_query_params* params,
                            uint64_t* tickets, int64_t* accepted) {
    if (!S || !queries || !params || !tickets || !accepted || m < 0) return fail(TACO_EINVAL, "null argument or m < 0");
    *accepted = 0;
    for (int64_t j = 0; j < m; ++j)
        if (int rc = check_request(S, params[j])) return rc;
    if (m == 0) return TACO_OK;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop) return fail(TACO_EINVAL, "the server is stopping");
    if (S->fatal) return fail(S->fatal, "the server stopped after a device error");
    *accepted = enqueue_locked(S, queries, m, params, tickets);
    if (*accepted < m) S->st.rejected += m - *accepted;
    lk.unlock();
    if (*accepted) S->cv_dispatch.notify_one();
    return *accepted == m ? TACO_OK
                          : fail(TACO_EAGAIN, "the request queue took %lld of %lld requests", (long long)*accepted,
                                 (long long)m);
}

int taco_server_wait(taco_server* S, uint64_t ticket, int64_t timeout_us, int32_t k_stride, int64_t* ids,
                     float* dists, taco_request_info* info) {
    if (!S || !ids || !dists) return fail(TACO_EINVAL, "null argument");
    const uint64_t r = ticket & ((uint64_t(1) << kTicketShift) - 1u);
    std::unique_lock<std::mutex> lk(S->mu);
    if (r >= S->reqs.size() || S->reqs[r].ticket != ticket || S->reqs[r].state == kFree)
        return fail(TACO_EINVAL, "unknown or already collected ticket");
    Request& R = S->reqs[r];
    if (k_stride < R.p.k) return fail(TACO_EINVAL, "k_stride %d < k %d", k_stride, R.p.k);
    auto ready = [&] { return R.state == kDone; };
    if (timeout_us < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return fail(TACO_ETIMEOUT, "request not answered within %lld us", (long long)timeout_us);
    }
    const int rc = R.rc;
    if (rc == TACO_OK) {
        const int64_t* src_i = S->id_store.data() + r * S->k_out;
        const float* src_d = S->d_store.data() + r * S->k_out;
        for (int t = 0; t < k_stride; ++t) {
            const bool in = t < R.p.k;
            ids[t] = in ? src_i[t] : -1;
            dists[t] = in ? src_d[t] : __builtin_huge_valf();
        }
    }
    if (info) *info = R.info;
    R.state = kFree;
    R.ticket = 0;
    S->free_pos.push_back(int(r));
    return rc == TACO_OK ? TACO_OK : fail(rc, "the request's batch failed");
}

int taco_server_get_stats(taco_server* S, taco_server_stats* stats) {
    if (!S || !stats) return fail(TACO_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *stats = S->st;
    return TACO_OK;
}

int taco_server_replay(taco_server* S, const float* queries, int64_t nq, const taco_query_params* params,
                       const int64_t* arrival_ns, int32_t k_stride, int64_t* ids, float* dists,
                       int64_t* latency_ns) {
    if (!S || !queries || !params || !arrival_ns || !ids || !dists || !latency_ns)
        return fail(TACO_EINVAL, "null argument");
    if (nq < 0 || k_stride < 1) return fail(TACO_EINVAL, "nq < 0 or k_stride < 1");
    for (int64_t j = 0; j < nq; ++j) {
        if (j && arrival_ns[j] < arrival_ns[j - 1]) return fail(TACO_EINVAL, "arrival_ns must ascend");
        if (params[j].k > k_stride) return fail(TACO_EINVAL, "k of request %lld exceeds k_stride", (long long)j);
        if (int rc = check_request(S, params[j])) return rc;
    }
    std::vector<uint64_t> tickets(size_t(nq), 0);
    std::atomic<int64_t> submitted(0);
    std::atomic<int> first_rc(TACO_OK);
    const int64_t t0 = now_ns();
    // producer: every request due by now goes in one call (a burst), the rest waits
    std::thread producer([&] {
        int64_t j = 0;
        while (j < nq) {
            const int64_t due = t0 + arrival_ns[j];
            int64_t now = now_ns();
            if (now < due) {
                if (due - now > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(due - now - 100000));
                continue;
            }
            int64_t e = j + 1;
            while (e < nq && t0 + arrival_ns[e] <= now) ++e;
            int64_t got = 0;
            const int rc = taco_server_submit_many(S, queries + size_t(j) * S->d, e - j, params + j,
                                                   tickets.data() + j, &got);
            j += got;
            submitted.store(j, std::memory_order_release);
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->cv_done.notify_all();   // the collector waits for submissions on this condition
            }
            if (rc == TACO_EAGAIN) {
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            } else if (rc != TACO_OK) {
                int z = TACO_OK;
                first_rc.compare_exchange_strong(z, rc);
                break;
            }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->cv_done.notify_all();
    });
    // collector: takes every finished request in order under one lock acquisition
    int64_t j = 0;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        while (j < nq) {
            const int64_t sub = submitted.load(std::memory_order_acquire);
            if (j >= sub) {
                if (first_rc.load() != TACO_OK) break;
                S->cv_done.wait_for(lk, std::chrono::microseconds(200));
                continue;
            }
            const uint64_t tk = tickets[size_t(j)];
            const uint64_t r = tk & ((uint64_t(1) << kTicketShift) - 1u);
            Request& R = S->reqs[r];
            if (R.state != kDone) {
                S->cv_done.wait_for(lk, std::chrono::microseconds(200));
                continue;
            }
            int64_t* oi = ids + size_t(j) * k_stride;
            float* od = dists + size_t(j) * k_stride;
            const int64_t* src_i = S->id_store.data() + r * S->k_out;
            const float* src_d = S->d_store.data() + r * S->k_out;
            for (int t = 0; t < k_stride; ++t) {
                const bool in = R.rc == TACO_OK && t < R.p.k;
                oi[t] = in ? src_i[t] : -1;
                od[t] = in ? src_d[t] : __builtin_huge_valf();
            }
            latency_ns[j] = R.info.done_ns - (t0 + arrival_ns[j]);
            if (R.rc != TACO_OK) {
                int z = TACO_OK;
                first_rc.compare_exchange_strong(z, R.rc);
            }
            R.state = kFree;
            R.ticket = 0;
            S->free_pos.push_back(int(r));
            ++j;
        }
    }
    producer.join();
    const int rc = first_rc.load();
    return rc == TACO_OK ? TACO_OK : fail(rc, "a replayed request failed");
}

void taco_server_destroy(taco_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued requests are dropped (answered with an error); running batches finish
        for (int r : S->pending) {
            S->reqs[r].rc = TACO_EINVAL;
            S->reqs[r].state = kDone;
        }
        S->pending.clear();
    }
    S->cv_done.notify_all();
    S->cv_dispatch.notify_all();
    if (S->dispatcher.joinable()) S->dispatcher.join();
    if (S->completer.joinable()) S->completer.join();
    release_slots(S);
    delete S;
}

}  // extern "C"

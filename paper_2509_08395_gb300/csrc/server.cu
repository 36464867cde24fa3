// Continuous-batching server (sindi_server_*): a native request loop around
// the search. One worker thread per server forms micro-batches from the
// submission queue and runs each on a free device slot; completions are
// detected with CUDA events and handed back through tickets.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "nvtx.cuh"

namespace sindi {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<int32_t> idx;
    std::vector<float> val;
    Clock::time_point t_submit, t_done;
    std::vector<uint32_t> ids;
    std::vector<float> scores;
    int state = 0;  // 0 queued, 1 on the device, 2 finished
    sindi_status status = SINDI_OK;
    std::string error;  // why it failed (the worker's own last-error string is not the poller's)
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t* h_indptr = nullptr;
    int32_t* h_idx = nullptr;
    float* h_val = nullptr;
    uint32_t* h_ids = nullptr;
    float* h_sc = nullptr;
    int64_t* d_indptr = nullptr;
    int32_t* d_idx = nullptr;
    float* d_val = nullptr;
    uint32_t* d_ids = nullptr;
    float* d_sc = nullptr;
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<std::shared_ptr<Request>> batch;
    bool busy = false;
};

struct Server {
    const IndexImpl* ix = nullptr;
    sindi_server_params prm{};
    size_t slot_bytes = 0;
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv_work;   // worker: new requests or shutdown
    std::condition_variable cv_done;   // pollers: a request finished
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread worker;

    // counters (under mu)
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_queries = 0;
    uint32_t in_flight = 0, peak_in_flight = 0;
    std::vector<double> latencies_ms;

    void run();
    bool launch(Slot& s, std::vector<std::shared_ptr<Request>>&& batch);
    void finish(Slot& s);
};

static void free_slot(Slot& s) {
    if (s.stream) (void)cudaStreamSynchronize(s.stream);
    void* dev[] = {s.d_indptr, s.d_idx, s.d_val, s.d_ids, s.d_sc, s.d_ws};
    for (void* p : dev)
        if (p) (void)cudaFree(p);
    void* host[] = {s.h_indptr, s.h_idx, s.h_val, s.h_ids, s.h_sc};
    for (void* p : host)
        if (p) (void)cudaFreeHost(p);
    if (s.done) (void)cudaEventDestroy(s.done);
    if (s.stream) (void)cudaStreamDestroy(s.stream);
    s = Slot();
}

// Copies a batch into the slot's pinned buffers and queues copy-in, search,
// copy-out and the completion event on the slot's stream.
bool Server::launch(Slot& s, std::vector<std::shared_ptr<Request>>&& batch) {
    const int64_t nb = (int64_t)batch.size();
    const uint32_t k = prm.search.k;
    int64_t nnz = 0;
    s.h_indptr[0] = 0;
    for (int64_t i = 0; i < nb; i++) {
        const Request& r = *batch[i];
        std::copy(r.idx.begin(), r.idx.end(), s.h_idx + nnz);
        std::copy(r.val.begin(), r.val.end(), s.h_val + nnz);
        nnz += (int64_t)r.idx.size();
        s.h_indptr[i + 1] = nnz;
    }
    sindi_search_params sp = prm.search;
    sp.mode = SINDI_MODE_BATCHED;
    sindi_status st = SINDI_OK;
    try {
        SINDI_CUDA(cudaMemcpyAsync(s.d_indptr, s.h_indptr, 8 * (nb + 1), cudaMemcpyHostToDevice, s.stream));
        if (nnz > 0) {
            SINDI_CUDA(cudaMemcpyAsync(s.d_idx, s.h_idx, 4 * nnz, cudaMemcpyHostToDevice, s.stream));
            SINDI_CUDA(cudaMemcpyAsync(s.d_val, s.h_val, 4 * nnz, cudaMemcpyHostToDevice, s.stream));
        }
        st = search_in_workspace(*ix, s.d_indptr, s.d_idx, s.d_val, nb, sp, s.d_ids, s.d_sc, s.stream, s.d_ws,
                                 s.ws_bytes);
        if (st == SINDI_OK) {
            SINDI_CUDA(cudaMemcpyAsync(s.h_ids, s.d_ids, 4 * (size_t)nb * k, cudaMemcpyDeviceToHost, s.stream));
            SINDI_CUDA(cudaMemcpyAsync(s.h_sc, s.d_sc, 4 * (size_t)nb * k, cudaMemcpyDeviceToHost, s.stream));
        }
        SINDI_CUDA(cudaEventRecord(s.done, s.stream));
    } catch (const CudaError& e) {
        set_last_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");
        st = SINDI_ERR_CUDA;
    }
    s.batch = std::move(batch);
    s.busy = true;
    if (st != SINDI_OK) {
        const std::string why = "batch of " + std::to_string(nb) + " failed: " + sindi_last_error();
        for (auto& r : s.batch) {
            r->status = st;
            r->error = why;
        }
    }
    return st == SINDI_OK;
}

// Results of a finished slot back into its requests.
void Server::finish(Slot& s) {
    const uint32_t k = prm.search.k;
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < s.batch.size(); i++) {
        Request& r = *s.batch[i];
        if (r.status == SINDI_OK) {
            r.ids.assign(s.h_ids + i * k, s.h_ids + (i + 1) * k);
            r.scores.assign(s.h_sc + i * k, s.h_sc + (i + 1) * k);
            completed++;
        } else {
            failed++;
        }
        r.t_done = now;
        r.state = 2;
        latencies_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    }
    s.batch.clear();
    s.busy = false;
    in_flight--;
    cv_done.notify_all();
}

void Server::run() {
    (void)cudaSetDevice(ix->device);
    const auto max_wait = std::chrono::microseconds(prm.max_wait_us);
    for (;;) {
        // completions
        bool any_busy = false;
        for (auto& s : slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaSuccess) {
                finish(s);
            } else if (q != cudaErrorNotReady) {
                for (auto& r : s.batch) {
                    r->status = SINDI_ERR_CUDA;
                    r->error = std::string("batch failed on the device: ") + cudaGetErrorString(q);
                }
                finish(s);
            } else {
                any_busy = true;
            }
        }
        // admissions: every free slot takes up to max_batch queued requests
        std::vector<std::pair<Slot*, std::vector<std::shared_ptr<Request>>>> starts;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stopping && queue.empty() && !any_busy) break;
            for (auto& s : slots) {
                if (s.busy || queue.empty()) continue;
                // a partial batch may wait for company while other slots are busy
                if (!stopping && queue.size() < prm.max_batch && any_busy && prm.max_wait_us > 0 &&
                    Clock::now() - queue.front()->t_submit < max_wait)
                    break;
                std::vector<std::shared_ptr<Request>> b;
                while (!queue.empty() && b.size() < prm.max_batch) {
                    b.push_back(queue.front());
                    queue.pop_front();
                    b.back()->state = 1;
                }
                s.busy = true;  // reserved; launched below without the lock
                in_flight++;
                peak_in_flight = std::max(peak_in_flight, in_flight);
                batches++;
                batched_queries += b.size();
                starts.emplace_back(&s, std::move(b));
            }
            if (starts.empty()) {
                if (any_busy || !queue.empty())
                    cv_work.wait_for(lk, std::chrono::microseconds(20));
                else
                    cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
        for (auto& st : starts) {
            NvtxRange range("sindi_server batch of %lld (slot %lld)", (long long)st.second.size(),
                            (long long)(st.first - slots.data()));
            if (!launch(*st.first, std::move(st.second))) finish(*st.first);
        }
    }
}

}  // namespace sindi

using namespace sindi;

struct sindi_server {
    Server impl;
};

extern "C" {

sindi_status sindi_server_create(const sindi_index* index, const sindi_server_params* params, sindi_server** out) {
    set_last_error("");
    if (!index || !params || !out) {
        set_last_error("index / params / out is NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    sindi_server_params p = *params;
    if (p.max_batch == 0) p.max_batch = 256;
    if (p.max_slots == 0) p.max_slots = 4;
    if (p.max_query_nnz == 0) p.max_query_nnz = 512;
    const sindi_search_params& sp = p.search;
    if (p.max_batch > 4096 || p.max_slots > 64 || p.max_query_nnz > 2048 || sp.k < 1 || sp.k > kMaxK ||
        (sp.gamma != 0 && (sp.gamma < sp.k || sp.gamma > kMaxGamma)) || !(sp.beta > 0.0 && sp.beta <= 1.0) ||
        !valid_block_threads(sp.block_threads) || sp.group > kMaxQueryGroup ||
        sp.accumulator > SINDI_ACCUM_FIXED32) {
        set_last_error("max_batch <= 4096, max_slots <= 64, max_query_nnz <= 2048; k in [1, 1024]; gamma 0 or in "
                       "[k, 8192]; beta in (0, 1]; block_threads 0, 1, 256, 512 or 1024; group 0..8; accumulator 0..2");
        return SINDI_ERR_INVALID_ARG;
    }
    if (sp.beta < 1.0) {
        set_last_error("query pruning (beta < 1) allocates its pruned queries: use sindi_search");
        return SINDI_ERR_UNSUPPORTED;
    }
    const IndexImpl& ix = index->impl;
    int prev = -1;
    (void)cudaGetDevice(&prev);
    (void)cudaSetDevice(ix.device);
    auto* h = new (std::nothrow) sindi_server;
    if (!h) return SINDI_ERR_OOM;
    Server& S = h->impl;
    S.ix = &ix;
    S.prm = p;
    sindi_search_params bsp = sp;
    bsp.mode = SINDI_MODE_BATCHED;
    const size_t ws = search_workspace_bytes(ix, bsp, p.max_batch);
    const size_t nnz_cap = (size_t)p.max_batch * p.max_query_nnz;
    S.slot_bytes = ws + 8 * (p.max_batch + 1) + 8 * nnz_cap + 8 * (size_t)p.max_batch * sp.k;
    uint32_t n_slots = p.max_slots;
    if (p.memory_budget > 0) n_slots = (uint32_t)std::min<uint64_t>(n_slots, p.memory_budget / S.slot_bytes);
    if (n_slots == 0) {
        delete h;
        set_last_error("memory_budget admits no slot: one slot needs " + std::to_string(S.slot_bytes) + " bytes");
        if (prev >= 0) (void)cudaSetDevice(prev);
        return SINDI_ERR_OOM;
    }
    sindi_status st = SINDI_OK;
    try {
        S.slots.resize(n_slots);
        for (auto& s : S.slots) {
            SINDI_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
            SINDI_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
            SINDI_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s.h_indptr), 8 * (p.max_batch + 1)));
            SINDI_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s.h_idx), 4 * nnz_cap));
            SINDI_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s.h_val), 4 * nnz_cap));
            SINDI_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s.h_ids), 4 * (size_t)p.max_batch * sp.k));
            SINDI_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s.h_sc), 4 * (size_t)p.max_batch * sp.k));
            SINDI_CUDA(cudaMalloc(reinterpret_cast<void**>(&s.d_indptr), 8 * (p.max_batch + 1)));
            SINDI_CUDA(cudaMalloc(reinterpret_cast<void**>(&s.d_idx), 4 * nnz_cap));
            SINDI_CUDA(cudaMalloc(reinterpret_cast<void**>(&s.d_val), 4 * nnz_cap));
            SINDI_CUDA(cudaMalloc(reinterpret_cast<void**>(&s.d_ids), 4 * (size_t)p.max_batch * sp.k));
            SINDI_CUDA(cudaMalloc(reinterpret_cast<void**>(&s.d_sc), 4 * (size_t)p.max_batch * sp.k));
            SINDI_CUDA(cudaMalloc(&s.d_ws, ws));
            s.ws_bytes = ws;
        }
    } catch (const CudaError& e) {
        set_last_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");
        st = e.code == cudaErrorMemoryAllocation ? SINDI_ERR_OOM : SINDI_ERR_CUDA;
    }
    if (st != SINDI_OK) {
        for (auto& s : S.slots) free_slot(s);
        delete h;
        if (prev >= 0) (void)cudaSetDevice(prev);
        return st;
    }
    S.worker = std::thread([&S] { S.run(); });
    if (prev >= 0) (void)cudaSetDevice(prev);
    *out = h;
    return SINDI_OK;
}

sindi_status sindi_server_submit(sindi_server* server, const int32_t* q_indices, const float* q_values, int32_t nnz,
                                 uint64_t* ticket) {
    if (!server || !ticket || nnz < 0 || (nnz > 0 && (!q_indices || !q_values))) return SINDI_ERR_INVALID_ARG;
    Server& S = server->impl;
    if ((uint32_t)nnz > S.prm.max_query_nnz) {
        set_last_error("query longer than max_query_nnz");
        return SINDI_ERR_INVALID_ARG;
    }
    auto r = std::make_shared<Request>();
    r->idx.assign(q_indices, q_indices + nnz);
    r->val.assign(q_values, q_values + nnz);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.stopping) {
            set_last_error("server is shutting down");
            return SINDI_ERR_INVALID_ARG;
        }
        r->ticket = S.next_ticket++;
        S.live[r->ticket] = r;
        S.queue.push_back(r);
        S.submitted++;
        *ticket = r->ticket;
    }
    S.cv_work.notify_one();
    return SINDI_OK;
}

sindi_status sindi_server_poll(sindi_server* server, uint64_t ticket, int32_t wait_ms, uint32_t* ids, float* scores,
                               double* latency_ms) {
    if (!server) return SINDI_ERR_INVALID_ARG;
    Server& S = server->impl;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.live.find(ticket);
    if (it == S.live.end()) {
        set_last_error("unknown ticket");
        return SINDI_ERR_INVALID_ARG;
    }
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->state == 2; };
    if (!ready()) {
        if (wait_ms < 0) S.cv_done.wait(lk, ready);
        else if (wait_ms > 0) S.cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    }
    if (!ready()) return SINDI_ERR_TIMEOUT;
    S.live.erase(it);
    lk.unlock();
    if (r->status != SINDI_OK) {
        set_last_error(r->error);
        return r->status;
    }
    if (ids) std::copy(r->ids.begin(), r->ids.end(), ids);
    if (scores) std::copy(r->scores.begin(), r->scores.end(), scores);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return SINDI_OK;
}

sindi_status sindi_server_stats(sindi_server* server, sindi_server_stats_t* out, int reset) {
    if (!server || !out) return SINDI_ERR_INVALID_ARG;
    Server& S = server->impl;
    std::lock_guard<std::mutex> lk(S.mu);
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->failed = S.failed;
    out->batches = S.batches;
    out->n_slots = (uint32_t)S.slots.size();
    out->peak_in_flight = S.peak_in_flight;
    out->slot_bytes = S.slot_bytes;
    out->mean_batch = S.batches ? (double)S.batched_queries / (double)S.batches : 0.0;
    std::vector<double> v = S.latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * (double)v.size()) - 1);
        return v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.empty() ? 0.0 : v.back();
    if (reset) {
        S.latencies_ms.clear();
        S.submitted = S.completed = S.failed = S.batches = S.batched_queries = 0;
        S.peak_in_flight = S.in_flight;
    }
    return SINDI_OK;
}

void sindi_server_destroy(sindi_server* server) {
    if (!server) return;
    Server& S = server->impl;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stopping = true;
    }
    S.cv_work.notify_all();
    if (S.worker.joinable()) S.worker.join();
    int prev = -1;
    (void)cudaGetDevice(&prev);
    (void)cudaSetDevice(S.ix->device);
    for (auto& s : S.slots) free_slot(s);
    if (prev >= 0) (void)cudaSetDevice(prev);
    delete server;
}

}  // extern "C"

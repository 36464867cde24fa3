// The C ABI (include/sindi.h): argument checks, host/device staging, memory
// pool, error reporting. The computation lives in build.cu and search.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "common.cuh"
#include "index.cuh"
#include "nvtx.cuh"
#include "primitives.cuh"

namespace sindi {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

bool trace_on() {
    static const bool on = [] {
        const char* e = std::getenv("SINDI_TRACE");
        return e && e[0] && e[0] != '0';
    }();
    return on;
}

// One pool per device, owned by the library, that keeps freed blocks for
// reuse (release threshold = unlimited); big temporaries of a build are
// returned with an explicit trim.
cudaMemPool_t library_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool;
    SINDI_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = ~0ull;
    SINDI_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    pools[device] = pool;
    return pool;
}

enum class Where { Host, Device, Invalid };

static Where where_is(const void* p) {
    if (!p) return Where::Invalid;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return Where::Host;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? Where::Device : Where::Host;
}

static sindi_status from_cuda(const CudaError& e) {
    set_last_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");
    if (e.code == cudaErrorMemoryAllocation) return SINDI_ERR_OOM;
    return SINDI_ERR_CUDA;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) (void)cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) (void)cudaSetDevice(prev);
    }
};

static void free_index_memory(IndexImpl& ix, cudaStream_t s) {
    void* ptrs[] = {ix.indptr, ix.indices, ix.values, ix.seg, ix.pid, ix.pval, ix.scale, ix.vmax, ix.kept, ix.err};
    for (void* p : ptrs)
        if (p) (void)cudaFreeAsync(p, s);
    (void)cudaStreamSynchronize(s);
    ix.indptr = nullptr;
    ix.indices = nullptr;
    ix.values = nullptr;
    ix.seg = nullptr;
    ix.pid = nullptr;
    ix.pval = nullptr;
    ix.scale = nullptr;
    ix.vmax = nullptr;
    ix.kept = nullptr;
    ix.err = nullptr;
    {
        std::lock_guard<std::mutex> lk(ix.lane_mu);
        for (cudaStream_t l : ix.lanes) (void)cudaStreamDestroy(l);
        ix.lanes.clear();
    }
    std::lock_guard<std::mutex> lk(ix.graph_mu);
    if (ix.graph_exec) (void)cudaGraphExecDestroy(ix.graph_exec);
    if (ix.graph_ws) (void)cudaFree(ix.graph_ws);
    if (ix.graph_done) (void)cudaEventDestroy(ix.graph_done);
    ix.graph_exec = nullptr;
    ix.graph_ws = nullptr;
    ix.graph_done = nullptr;
}

static std::string query_error_text(uint32_t e) {
    std::string m;
    if (e & kErrQueryDim) m += "a query dim outside [0, dim); ";
    if (e & kErrQueryValue) m += "a non-finite query value; ";
    if (e & kErrQueryDup) m += "a dim repeated within a query; ";
    if (e & kErrQueryTooLong) m += "a query with more than 2048 entries; ";
    if (e & kErrCandOverflow) m += "candidate buffer overflow; ";
    if (e & kErrBounds) m += "an offset or id out of bounds (checked build; the access was skipped); ";
    if (e & kErrTimeout) m += "a bounded device wait gave up; ";
    return m;
}

static sindi_status status_of_error_word(uint32_t e) {
    if (e == 0) return SINDI_OK;
    set_last_error("device error word: " + query_error_text(e));
    if (e & kErrTimeout) return SINDI_ERR_TIMEOUT;
    return SINDI_ERR_INVALID_DATA;
}

// ---------------------------------------------------------------------------
// Index files (sindi_index_save / sindi_index_load): a fixed header, then the
// device arrays in order, host byte order. Arrays move through one pinned
// staging buffer in pieces, so an index larger than host memory still fits.
// ---------------------------------------------------------------------------

constexpr char kFileMagic[8] = {'S', 'I', 'N', 'D', 'I', 'G', 'B', '3'};
constexpr uint32_t kFileVersion = 1;
constexpr size_t kStageBytes = (size_t)64 << 20;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n_docs;
    int32_t dim;
    uint32_t lambda;
    uint32_t sigma;
    int32_t dtype;
    double alpha;
    int32_t prune;
    uint32_t prune_n;
    int64_t doc_nnz;
    int64_t postings;
};

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

struct Pinned {
    void* p = nullptr;
    ~Pinned() {
        if (p) (void)cudaFreeHost(p);
    }
};

// Device -> file, through the staging buffer.
static bool write_device(FILE* f, const void* dev, size_t bytes, void* stage) {
    const unsigned char* d = static_cast<const unsigned char*>(dev);
    for (size_t off = 0; off < bytes; off += kStageBytes) {
        const size_t n = bytes - off < kStageBytes ? bytes - off : kStageBytes;
        SINDI_CUDA(cudaMemcpy(stage, d + off, n, cudaMemcpyDeviceToHost));
        if (std::fwrite(stage, 1, n, f) != n) return false;
    }
    return true;
}

// File -> device, through the staging buffer; `check` sees every piece on the
// host first (element-aligned pieces) and may reject it.
template <typename T, typename Check>
static bool read_device(FILE* f, T* dev, size_t count, void* stage, const Check& check, cudaStream_t s) {
    const size_t per = kStageBytes / sizeof(T);
    for (size_t off = 0; off < count; off += per) {
        const size_t n = count - off < per ? count - off : per;
        if (std::fread(stage, sizeof(T), n, f) != n) return false;
        if (!check(static_cast<const T*>(stage), off, n)) return false;
        SINDI_CUDA(cudaMemcpyAsync(dev + off, stage, n * sizeof(T), cudaMemcpyHostToDevice, s));
        SINDI_CUDA(cudaStreamSynchronize(s));
    }
    return true;
}


}  // namespace sindi

using namespace sindi;

// Replays of the recorded plain graph share its workspace: a plain call on
// another stream must not start before the previous replay has ended. A
// stream being captured never replays the graph and may not wait on an
// event recorded outside its capture.
static void after_last_graph_replay(const IndexImpl& ix, const sindi_search_params& prm, cudaStream_t s) {
    if (prm.mode != SINDI_MODE_PLAIN || prm.beta < 1.0) return;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    SINDI_CUDA(cudaStreamIsCapturing(s, &cst));
    if (cst != cudaStreamCaptureStatusNone) return;
    cudaEvent_t last = nullptr;
    {
        std::lock_guard<std::mutex> lk(ix.graph_mu);
        last = ix.graph_exec ? ix.graph_done : nullptr;
    }
    if (last) SINDI_CUDA(cudaStreamWaitEvent(s, last, 0));
}

extern "C" {

const char* sindi_last_error(void) { return g_last_error.c_str(); }

const char* sindi_version(void) { return "sindi-gb300 0.1 (sm_103a)"; }

sindi_status sindi_build(const int64_t* indptr, const int32_t* indices, const float* values, int64_t n_docs,
                         int32_t dim, const sindi_build_params* params, void* stream, sindi_index** out) {
    NvtxRange range("sindi_build n_docs=%lld dim=%lld", (long long)n_docs, (long long)dim);
    SINDI_TRACE_MSG("sindi_build: enter n_docs=%lld dim=%d", (long long)n_docs, (int)dim);
    set_last_error("");
    if (!out) {
        set_last_error("out is NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    sindi_build_params prm = params ? *params : sindi_build_params{0, SINDI_F32, 1.0, SINDI_PRUNE_MASS, 0};
    if (n_docs < 0 || n_docs >= (int64_t)0xFFFFFFFFLL || dim <= 0 || !indptr) {
        set_last_error("n_docs must be in [0, 2^32 - 1), dim > 0, indptr not NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    if (!(prm.alpha > 0.0 && prm.alpha <= 1.0) || prm.window > kMaxWindow || prm.value_dtype < SINDI_F32 ||
        prm.value_dtype > SINDI_F8E4M3) {
        set_last_error("alpha must be in (0, 1], window in [0, 32768], value_dtype a sindi_dtype");
        return SINDI_ERR_INVALID_ARG;
    }
    if (prm.prune < SINDI_PRUNE_MASS || prm.prune > SINDI_PRUNE_MASS_LIST ||
        (prm.prune != SINDI_PRUNE_MASS && prm.prune_n == 0)) {
        set_last_error("prune must be a sindi_prune; prune_n >= 1 for VECTOR_NUMBER, LIST and MASS_LIST");
        return SINDI_ERR_INVALID_ARG;
    }
    if ((uint64_t)dim * (uint64_t)std::max<int64_t>(1, (n_docs + std::max<uint32_t>(prm.window, 1) - 1) /
                                                          std::max<uint32_t>(prm.window, 1)) >= (1ull << 34)) {
        set_last_error("dim * n_windows too large for the offset table");
        return SINDI_ERR_UNSUPPORTED;
    }
    const Where w_ptr = where_is(indptr);
    SINDI_TRACE_MSG("sindi_build: indptr is %s", w_ptr == Where::Device ? "device" : "host");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_last_error("no CUDA device");
        return SINDI_ERR_CUDA;
    }
    sindi_index* h = new (std::nothrow) sindi_index;
    if (!h) return SINDI_ERR_OOM;
    IndexImpl& ix = h->impl;
    try {
        ix.device = dev;
        SINDI_TRACE_MSG("sindi_build: device %d, creating pool", dev);
        ix.pool = library_pool(dev);
        SINDI_TRACE_MSG("sindi_build: pool ready");
        ix.n_docs = n_docs;
        ix.dim = dim;
        ix.lambda = prm.window ? prm.window : kDefaultWindow;
        ix.sigma = (uint32_t)((n_docs + ix.lambda - 1) / ix.lambda);
        ix.dtype = prm.value_dtype;
        ix.prune = prm.prune;
        ix.prune_n = prm.prune == SINDI_PRUNE_MASS ? 0u : prm.prune_n;
        // alpha applies to the mass-ratio methods only
        ix.alpha = (prm.prune == SINDI_PRUNE_MASS || prm.prune == SINDI_PRUNE_MASS_LIST) ? prm.alpha : 1.0;
        Pool P{ix.pool, s};
        ix.err = P.alloc<uint32_t>(1);
        SINDI_CUDA(cudaMemsetAsync(ix.err, 0, 4, s));
        ix.indptr = P.alloc<int64_t>(n_docs + 1);
        SINDI_CUDA(cudaMemcpyAsync(ix.indptr, indptr, sizeof(int64_t) * (n_docs + 1),
                                   w_ptr == Where::Device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        // indptr validity first: the number of entries comes from it
        SINDI_TRACE_MSG("sindi_build: indptr copied; validating");
        launch_validate_indptr(ix.indptr, n_docs, ix.err, s);
        uint32_t e = 0;
        int64_t nnz = 0;
        SINDI_CUDA(cudaMemcpyAsync(&e, ix.err, 4, cudaMemcpyDeviceToHost, s));
        SINDI_CUDA(cudaMemcpyAsync(&nnz, ix.indptr + n_docs, 8, cudaMemcpyDeviceToHost, s));
        SINDI_CUDA(cudaStreamSynchronize(s));
        if (e != 0 || nnz < 0) {
            free_index_memory(ix, s);
            delete h;
            set_last_error("malformed documents: indptr[0] != 0 or decreasing");
            return SINDI_ERR_INVALID_DATA;
        }
        if (nnz > 0 && (!indices || !values)) {
            free_index_memory(ix, s);
            delete h;
            set_last_error("indices / values are NULL");
            return SINDI_ERR_INVALID_ARG;
        }
        SINDI_TRACE_MSG("sindi_build: indptr ok, nnz=%lld", (long long)nnz);
        ix.doc_nnz = nnz;
        ix.indices = P.alloc<int32_t>(nnz);
        ix.values = P.alloc<float>(nnz);
        if (nnz > 0) {
            const bool dsrc = where_is(indices) == Where::Device;
            SINDI_CUDA(cudaMemcpyAsync(ix.indices, indices, sizeof(int32_t) * nnz,
                                       dsrc ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
            SINDI_CUDA(cudaMemcpyAsync(ix.values, values, sizeof(float) * nnz,
                                       where_is(values) == Where::Device ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyHostToDevice,
                                       s));
        }
        SINDI_TRACE_MSG("sindi_build: documents on device; building lists");
        sindi_status st = build_lists(ix, s);
        SINDI_TRACE_MSG("sindi_build: lists done, status %d", (int)st);
        SINDI_CUDA(cudaStreamSynchronize(s));
        SINDI_CUDA(cudaMemPoolTrimTo(ix.pool, 0));
        if (st != SINDI_OK) {
            free_index_memory(ix, s);
            delete h;
            return st;
        }
    } catch (const CudaError& e) {
        SINDI_TRACE_MSG("sindi_build: CUDA error %s at %s", cudaGetErrorString(e.code), e.where.c_str());
        sindi_status st = from_cuda(e);
        free_index_memory(ix, s);
        delete h;
        return st;
    } catch (const std::bad_alloc&) {
        free_index_memory(ix, s);
        delete h;
        set_last_error("host out of memory");
        return SINDI_ERR_OOM;
    }
    *out = h;
    return SINDI_OK;
}

sindi_status sindi_search(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                          const float* q_values, int64_t n_queries, const sindi_search_params* params,
                          uint32_t* out_ids, float* out_scores, void* stream) {
    NvtxRange range("sindi_search n_queries=%lld mode=%lld", (long long)n_queries,
                    params ? (long long)params->mode : -1LL);
    set_last_error("");
    if (!index || !params) {
        set_last_error("index / params is NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    const sindi_search_params prm = *params;
    if (prm.k < 1 || prm.k > kMaxK || (prm.gamma != 0 && (prm.gamma < prm.k || prm.gamma > kMaxGamma)) ||
        !(prm.beta > 0.0 && prm.beta <= 1.0) || prm.mode > SINDI_MODE_BATCHED ||
        !valid_block_threads(prm.block_threads) || prm.group > kMaxQueryGroup ||
        prm.accumulator > SINDI_ACCUM_FIXED32) {
        set_last_error("k in [1, 1024]; gamma 0 or in [k, 8192]; beta in (0, 1]; mode 0/1; block_threads 0, 1 (pipelined), 256, 512 or 1024; group 0..8; accumulator 0..2");
        return SINDI_ERR_INVALID_ARG;
    }

    if (n_queries < 0 || n_queries > (int64_t)1 << 31) {
        set_last_error("n_queries out of range");
        return SINDI_ERR_INVALID_ARG;
    }
    if (n_queries == 0) return SINDI_OK;
    if (!q_indptr || !out_ids || !out_scores) {
        set_last_error("NULL query or output pointer");
        return SINDI_ERR_INVALID_ARG;
    }
    const IndexImpl& ix = index->impl;
    DeviceGuard dg(ix.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool in_dev = where_is(q_indptr) == Where::Device;
    const bool out_dev = where_is(out_ids) == Where::Device;
    if (in_dev && out_dev) {
        if (!q_indices || !q_values) {
            set_last_error("NULL query arrays");
            return SINDI_ERR_INVALID_ARG;
        }
        try {
            after_last_graph_replay(ix, prm, s);
            return search_impl(ix, q_indptr, q_indices, q_values, n_queries, prm, out_ids, out_scores, s);
        } catch (const CudaError& e) {
            return from_cuda(e);
        }
    }
    // staged path: copy host inputs in, run, copy results out, synchronise
    Pool P{ix.pool, s};
    int64_t* d_ip = nullptr;
    int32_t* d_ix = nullptr;
    float* d_v = nullptr;
    uint32_t* d_ids = nullptr;
    float* d_sc = nullptr;
    sindi_status st = SINDI_OK;
    try {
        const int64_t* ip = q_indptr;
        const int32_t* qi = q_indices;
        const float* qv = q_values;
        if (!in_dev) {
            const int64_t nnz = q_indptr[n_queries];
            if (q_indptr[0] != 0 || nnz < 0 || (nnz > 0 && (!q_indices || !q_values))) {
                set_last_error("malformed query indptr");
                return SINDI_ERR_INVALID_ARG;
            }
            for (int64_t r = 0; r < n_queries; r++)
                if (q_indptr[r + 1] < q_indptr[r]) {
                    set_last_error("query indptr decreases");
                    return SINDI_ERR_INVALID_ARG;
                }
            d_ip = P.alloc<int64_t>(n_queries + 1);
            d_ix = P.alloc<int32_t>(nnz);
            d_v = P.alloc<float>(nnz);
            SINDI_CUDA(cudaMemcpyAsync(d_ip, q_indptr, 8 * (n_queries + 1), cudaMemcpyHostToDevice, s));
            if (nnz > 0) {
                SINDI_CUDA(cudaMemcpyAsync(d_ix, q_indices, 4 * nnz, cudaMemcpyHostToDevice, s));
                SINDI_CUDA(cudaMemcpyAsync(d_v, q_values, 4 * nnz, cudaMemcpyHostToDevice, s));
            }
            ip = d_ip;
            qi = d_ix;
            qv = d_v;
        }
        uint32_t* oi = out_ids;
        float* os = out_scores;
        const size_t nout = (size_t)n_queries * prm.k;
        if (!out_dev) {
            d_ids = P.alloc<uint32_t>(nout);
            d_sc = P.alloc<float>(nout);
            oi = d_ids;
            os = d_sc;
        }
        after_last_graph_replay(ix, prm, s);
        st = search_impl(ix, ip, qi, qv, n_queries, prm, oi, os, s);
        if (st == SINDI_OK && !out_dev) {
            SINDI_CUDA(cudaMemcpyAsync(out_ids, d_ids, 4 * nout, cudaMemcpyDeviceToHost, s));
            SINDI_CUDA(cudaMemcpyAsync(out_scores, d_sc, 4 * nout, cudaMemcpyDeviceToHost, s));
        }
        P.free(d_ip);
        P.free(d_ix);
        P.free(d_v);
        P.free(d_ids);
        P.free(d_sc);
        SINDI_CUDA(cudaStreamSynchronize(s));
        if (st == SINDI_OK) {
            uint32_t e = 0;
            SINDI_CUDA(cudaMemcpy(&e, ix.err, 4, cudaMemcpyDeviceToHost));
            if (e) {
                SINDI_CUDA(cudaMemset(ix.err, 0, 4));
                st = status_of_error_word(e);
            }
        }
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
    return st;
}

sindi_status sindi_merge_topk(const uint32_t* ids, const float* scores, int32_t n_shards, int64_t n_queries,
                              uint32_t k_in, const int64_t* id_offset, uint32_t k, uint32_t* out_ids,
                              float* out_scores, void* stream) {
    NvtxRange range("sindi_merge_topk n_shards=%lld n_queries=%lld", (long long)n_shards, (long long)n_queries);
    set_last_error("");
    if (n_shards < 1 || (uint32_t)n_shards > kMaxShards || k_in < 1 || k < 1 || k > kMaxK ||
        (uint64_t)n_shards * k_in > kMaxShardEntries || n_queries < 0 || n_queries > 0x7FFFFFFFLL || !id_offset) {
        set_last_error("1 <= n_shards <= 64, k_in >= 1, n_shards * k_in <= 8192, 1 <= k <= 1024, "
                       "0 <= n_queries < 2^31, id_offset not NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    if (n_queries == 0) return SINDI_OK;
    if (!ids || !scores || !out_ids || !out_scores || where_is(ids) != Where::Device ||
        where_is(scores) != Where::Device || where_is(out_ids) != Where::Device ||
        where_is(out_scores) != Where::Device) {
        set_last_error("ids, scores and both outputs must be device memory");
        return SINDI_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_shards; s++) {
        if (id_offset[s] < 0 || id_offset[s] >= 0xFFFFFFFFLL) {
            set_last_error("id_offset out of range: 0 <= id_offset < 0xFFFFFFFF");
            return SINDI_ERR_INVALID_ARG;
        }
    }
    try {
        merge_shards(ids, scores, (uint32_t)n_shards, n_queries, k_in, id_offset, k, out_ids, out_scores,
                     static_cast<cudaStream_t>(stream));
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
    return SINDI_OK;
}

sindi_status sindi_search_noalloc(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                                  const float* q_values, int64_t n_queries, const sindi_search_params* params,
                                  uint32_t* out_ids, float* out_scores, void* stream) {
    NvtxRange range("sindi_search_noalloc n_queries=%lld mode=%lld", (long long)n_queries,
                    params ? (long long)params->mode : -1LL);
    set_last_error("");
    if (!index || !params) {
        set_last_error("index / params is NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    const sindi_search_params prm = *params;
    if (prm.k < 1 || prm.k > kMaxK || (prm.gamma != 0 && (prm.gamma < prm.k || prm.gamma > kMaxGamma)) ||
        !(prm.beta > 0.0 && prm.beta <= 1.0) || prm.mode > SINDI_MODE_BATCHED ||
        !valid_block_threads(prm.block_threads) || prm.group > kMaxQueryGroup ||
        prm.accumulator > SINDI_ACCUM_FIXED32) {
        set_last_error("k in [1, 1024]; gamma 0 or in [k, 8192]; beta in (0, 1]; mode 0/1; block_threads 0, 1 (pipelined), 256, 512 or 1024; group 0..8; accumulator 0..2");
        return SINDI_ERR_INVALID_ARG;
    }
    if (prm.beta < 1.0) {
        set_last_error("query pruning (beta < 1) allocates its pruned queries: use sindi_search");
        return SINDI_ERR_UNSUPPORTED;
    }
    if (n_queries < 0 || n_queries > (int64_t)1 << 31) {
        set_last_error("n_queries out of range");
        return SINDI_ERR_INVALID_ARG;
    }
    if (n_queries == 0) return SINDI_OK;
    if (!q_indptr || !q_indices || !q_values || !out_ids || !out_scores) {
        set_last_error("NULL query or output pointer");
        return SINDI_ERR_INVALID_ARG;
    }
    const IndexImpl& ix = index->impl;
    DeviceGuard dg(ix.device);
    if (where_is(q_indptr) != Where::Device || where_is(q_indices) != Where::Device ||
        where_is(q_values) != Where::Device || where_is(out_ids) != Where::Device ||
        where_is(out_scores) != Where::Device) {
        set_last_error("sindi_search_noalloc takes device buffers only (staging host buffers would allocate)");
        return SINDI_ERR_INVALID_ARG;
    }
    try {
        return search_noalloc_impl(ix, q_indptr, q_indices, q_values, n_queries, prm, out_ids, out_scores,
                                   static_cast<cudaStream_t>(stream));
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
}

sindi_status sindi_check(const sindi_index* index, void* stream) {
    set_last_error("");
    if (!index) return SINDI_ERR_INVALID_ARG;
    const IndexImpl& ix = index->impl;
    DeviceGuard dg(ix.device);
    try {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        SINDI_CUDA(cudaStreamSynchronize(s));
        uint32_t e = 0;
        SINDI_CUDA(cudaMemcpy(&e, ix.err, 4, cudaMemcpyDeviceToHost));
        if (e) SINDI_CUDA(cudaMemset(ix.err, 0, 4));
        return status_of_error_word(e);
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
}

sindi_status sindi_index_info(const sindi_index* index, sindi_index_info_t* out) {
    if (!index || !out) return SINDI_ERR_INVALID_ARG;
    const IndexImpl& ix = index->impl;
    out->n_docs = ix.n_docs;
    out->dim = ix.dim;
    out->value_dtype = ix.dtype;
    out->window = ix.lambda;
    out->n_windows = ix.sigma;
    out->postings = ix.postings;
    out->doc_nnz = ix.doc_nnz;
    out->index_bytes = (int64_t)(((int64_t)ix.dim * ix.sigma + 1) * 4 + ix.postings * (2 + (int64_t)ix.value_bytes()) +
                                 (int64_t)ix.dim * 4);
    out->doc_bytes = (ix.n_docs + 1) * 8 + ix.doc_nnz * 8;
    out->alpha = ix.alpha;
    out->prune = ix.prune;
    out->prune_n = ix.prune_n;
    return SINDI_OK;
}

sindi_status sindi_index_export(const sindi_index* index, uint32_t* seg, uint16_t* ids, void* vals, float* scale,
                                uint32_t* kept) {
    set_last_error("");
    if (!index) return SINDI_ERR_INVALID_ARG;
    const IndexImpl& ix = index->impl;
    DeviceGuard dg(ix.device);
    try {
        if (seg) SINDI_CUDA(cudaMemcpy(seg, ix.seg, 4 * ((size_t)ix.dim * ix.sigma + 1), cudaMemcpyDeviceToHost));
        if (ids && ix.postings) SINDI_CUDA(cudaMemcpy(ids, ix.pid, 2 * (size_t)ix.postings, cudaMemcpyDeviceToHost));
        if (vals && ix.postings)
            SINDI_CUDA(cudaMemcpy(vals, ix.pval, ix.value_bytes() * (size_t)ix.postings, cudaMemcpyDeviceToHost));
        if (scale) SINDI_CUDA(cudaMemcpy(scale, ix.scale, 4 * (size_t)ix.dim, cudaMemcpyDeviceToHost));
        if (kept && ix.n_docs) SINDI_CUDA(cudaMemcpy(kept, ix.kept, 4 * (size_t)ix.n_docs, cudaMemcpyDeviceToHost));
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
    return SINDI_OK;
}


sindi_status sindi_index_save(const sindi_index* index, const char* path) {
    NvtxRange range("sindi_index_save");
    set_last_error("");
    if (!index || !path) {
        set_last_error("index and path must not be NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    const IndexImpl& ix = index->impl;
    DeviceGuard dg(ix.device);
    File file;
    file.f = std::fopen(path, "wb");
    if (!file.f) {
        set_last_error(std::string("cannot open ") + path + " for writing");
        return SINDI_ERR_INVALID_ARG;
    }
    FileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kFileMagic, 8);
    h.version = kFileVersion;
    h.header_bytes = (uint32_t)sizeof(FileHeader);
    h.n_docs = ix.n_docs;
    h.dim = ix.dim;
    h.lambda = ix.lambda;
    h.sigma = ix.sigma;
    h.dtype = ix.dtype;
    h.alpha = ix.alpha;
    h.prune = ix.prune;
    h.prune_n = ix.prune_n;
    h.doc_nnz = ix.doc_nnz;
    h.postings = ix.postings;
    try {
        Pinned stage;
        SINDI_CUDA(cudaMallocHost(&stage.p, kStageBytes));
        SINDI_CUDA(cudaDeviceSynchronize());  // the index is complete before it is read
        bool ok = std::fwrite(&h, sizeof(h), 1, file.f) == 1;
        const size_t S = (size_t)ix.dim * ix.sigma + 1, P = (size_t)ix.postings;
        ok = ok && write_device(file.f, ix.seg, 4 * S, stage.p);
        ok = ok && write_device(file.f, ix.pid, 2 * P, stage.p);
        ok = ok && write_device(file.f, ix.pval, ix.value_bytes() * P, stage.p);
        ok = ok && write_device(file.f, ix.scale, 4 * (size_t)ix.dim, stage.p);
        ok = ok && write_device(file.f, ix.kept, 4 * (size_t)ix.n_docs, stage.p);
        ok = ok && write_device(file.f, ix.indptr, 8 * ((size_t)ix.n_docs + 1), stage.p);
        ok = ok && write_device(file.f, ix.indices, 4 * (size_t)ix.doc_nnz, stage.p);
        ok = ok && write_device(file.f, ix.values, 4 * (size_t)ix.doc_nnz, stage.p);
        if (!ok || std::fflush(file.f) != 0) {
            set_last_error(std::string("write to ") + path + " failed");
            return SINDI_ERR_INVALID_ARG;
        }
    } catch (const CudaError& e) {
        return from_cuda(e);
    }
    return SINDI_OK;
}

sindi_status sindi_index_load(const char* path, void* stream, sindi_index** out) {
    NvtxRange range("sindi_index_load");
    set_last_error("");
    if (!path || !out) {
        set_last_error("path and out must not be NULL");
        return SINDI_ERR_INVALID_ARG;
    }
    File file;
    file.f = std::fopen(path, "rb");
    if (!file.f) {
        set_last_error(std::string("cannot open ") + path);
        return SINDI_ERR_INVALID_ARG;
    }
    FileHeader h;
    if (std::fread(&h, sizeof(h), 1, file.f) != 1 || std::memcmp(h.magic, kFileMagic, 8) != 0 ||
        h.version != kFileVersion || h.header_bytes != sizeof(FileHeader)) {
        set_last_error(std::string(path) + " is not an index file of this version");
        return SINDI_ERR_INVALID_DATA;
    }
    const uint64_t lam = h.lambda ? h.lambda : 1;
    if (h.n_docs < 0 || h.n_docs >= (int64_t)0xFFFFFFFFLL || h.dim <= 0 || h.lambda == 0 ||
        h.lambda > (uint32_t)kMaxWindow || (uint64_t)h.sigma != ((uint64_t)h.n_docs + lam - 1) / lam ||
        h.dtype < SINDI_F32 || h.dtype > SINDI_F8E4M3 || h.prune < SINDI_PRUNE_MASS ||
        h.prune > SINDI_PRUNE_MASS_LIST || h.doc_nnz < 0 || h.postings < 0 || h.postings > h.doc_nnz || h.postings > kMaxPostings ||
        !(h.alpha > 0.0 && h.alpha <= 1.0) || (uint64_t)h.dim * h.sigma >= (1ull << 34)) {
        set_last_error(std::string(path) + ": inconsistent header");
        return SINDI_ERR_INVALID_DATA;
    }
    const size_t vbytes = h.dtype == SINDI_F32 ? 4 : (h.dtype == SINDI_F16 ? 2 : 1);
    const size_t S = (size_t)h.dim * h.sigma + 1, P = (size_t)h.postings;
    const size_t want = sizeof(h) + 4 * S + (2 + vbytes) * P + 4 * (size_t)h.dim + 4 * (size_t)h.n_docs +
                        8 * ((size_t)h.n_docs + 1) + 8 * (size_t)h.doc_nnz;
    if (std::fseek(file.f, 0, SEEK_END) != 0 || (size_t)std::ftell(file.f) != want ||
        std::fseek(file.f, (long)sizeof(h), SEEK_SET) != 0) {
        set_last_error(std::string(path) + ": file size does not match its header");
        return SINDI_ERR_INVALID_DATA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_last_error("no CUDA device");
        return SINDI_ERR_CUDA;
    }
    sindi_index* hnd = new (std::nothrow) sindi_index;
    if (!hnd) return SINDI_ERR_OOM;
    IndexImpl& ix = hnd->impl;
    try {
        ix.device = dev;
        ix.pool = library_pool(dev);
        ix.n_docs = h.n_docs;
        ix.dim = h.dim;
        ix.lambda = h.lambda;
        ix.sigma = h.sigma;
        ix.dtype = h.dtype;
        ix.alpha = h.alpha;
        ix.prune = h.prune;
        ix.prune_n = h.prune_n;
        ix.doc_nnz = h.doc_nnz;
        ix.postings = h.postings;
        Pool Pl{ix.pool, s};
        ix.err = Pl.alloc<uint32_t>(1);
        SINDI_CUDA(cudaMemsetAsync(ix.err, 0, 4, s));
        const size_t Pp = (P + 7) & ~(size_t)7;  // the scan reads aligned groups of 8
        ix.seg = Pl.alloc<uint32_t>(S);
        ix.pid = Pl.alloc<uint16_t>(Pp);
        ix.pval = Pl.alloc<uint8_t>(Pp * vbytes);
        ix.scale = Pl.alloc<float>(h.dim);
        ix.kept = Pl.alloc<uint32_t>(h.n_docs > 0 ? h.n_docs : 1);
        ix.indptr = Pl.alloc<int64_t>(h.n_docs + 1);
        ix.indices = Pl.alloc<int32_t>(h.doc_nnz > 0 ? h.doc_nnz : 1);
        ix.values = Pl.alloc<float>(h.doc_nnz > 0 ? h.doc_nnz : 1);
        if (Pp > P) {
            SINDI_CUDA(cudaMemsetAsync(ix.pid + P, 0, 2 * (Pp - P), s));
            SINDI_CUDA(cudaMemsetAsync(static_cast<uint8_t*>(ix.pval) + P * vbytes, 0, (Pp - P) * vbytes, s));
        }
        Pinned stage;
        SINDI_CUDA(cudaMallocHost(&stage.p, kStageBytes));
        // every offset the kernels follow is checked on the host on its way in
        uint32_t seg_prev = 0;
        int64_t ip_prev = 0;
        const uint32_t lambda = h.lambda;
        const int32_t dim = h.dim;
        auto any = [](const void*, size_t, size_t) { return true; };
        bool ok = read_device(file.f, ix.seg, S, stage.p, [&](const uint32_t* v, size_t off, size_t n) {
            for (size_t t = 0; t < n; t++) {
                if ((off + t == 0 && v[t] != 0) || v[t] < seg_prev) return false;
                seg_prev = v[t];
            }
            return off + n < S || (uint64_t)seg_prev == (uint64_t)P;
        }, s);
        ok = ok && read_device(file.f, ix.pid, P, stage.p, [&](const uint16_t* v, size_t, size_t n) {
            for (size_t t = 0; t < n; t++)
                if (v[t] >= lambda) return false;
            return true;
        }, s);
        ok = ok && read_device(file.f, static_cast<uint8_t*>(ix.pval), P * vbytes, stage.p,
                               [&](const uint8_t* v, size_t o, size_t n) { return any(v, o, n); }, s);
        ok = ok && read_device(file.f, ix.scale, (size_t)h.dim, stage.p,
                               [&](const float* v, size_t o, size_t n) { return any(v, o, n); }, s);
        ok = ok && read_device(file.f, ix.kept, (size_t)h.n_docs, stage.p,
                               [&](const uint32_t* v, size_t o, size_t n) { return any(v, o, n); }, s);
        ok = ok && read_device(file.f, ix.indptr, (size_t)h.n_docs + 1, stage.p,
                               [&](const int64_t* v, size_t off, size_t n) {
            for (size_t t = 0; t < n; t++) {
                if ((off + t == 0 && v[t] != 0) || v[t] < ip_prev) return false;
                ip_prev = v[t];
            }
            return off + n < (size_t)h.n_docs + 1 || ip_prev == h.doc_nnz;
        }, s);
        ok = ok && read_device(file.f, ix.indices, (size_t)h.doc_nnz, stage.p, [&](const int32_t* v, size_t, size_t n) {
            for (size_t t = 0; t < n; t++)
                if (v[t] < 0 || v[t] >= dim) return false;
            return true;
        }, s);
        ok = ok && read_device(file.f, ix.values, (size_t)h.doc_nnz, stage.p,
                               [&](const float* v, size_t o, size_t n) { return any(v, o, n); }, s);
        if (!ok) {
            free_index_memory(ix, s);
            delete hnd;
            set_last_error(std::string(path) + ": truncated, or an offset or id out of range");
            return SINDI_ERR_INVALID_DATA;
        }
        SINDI_CUDA(cudaStreamSynchronize(s));
        list_value_bounds(ix, s);
        ix.nonneg = postings_nonnegative(ix, s);
    } catch (const CudaError& e) {
        sindi_status st = from_cuda(e);
        free_index_memory(ix, s);
        delete hnd;
        return st;
    }
    *out = hnd;
    return SINDI_OK;
}

sindi_status sindi_set_timing(const sindi_index* index, int enable) {
    if (!index) return SINDI_ERR_INVALID_ARG;
    index->impl.timing.store(enable ? 1 : 0);
    return SINDI_OK;
}

sindi_status sindi_get_stats(const sindi_index* index, sindi_stats_t* out) {
    if (!index || !out) return SINDI_ERR_INVALID_ARG;
    const IndexImpl& ix = index->impl;
    out->launches = ix.launches.load();
    out->scan_launches = ix.scan_launches.load();
    out->queries = ix.queries.load();
    out->scan_timed = ix.scan_timed.load();
    std::lock_guard<std::mutex> lk(ix.tmu);
    out->scan_ms = ix.scan_ms;
    return SINDI_OK;
}

sindi_status sindi_reset_stats(const sindi_index* index) {
    if (!index) return SINDI_ERR_INVALID_ARG;
    const IndexImpl& ix = index->impl;
    ix.launches = 0;
    ix.scan_launches = 0;
    ix.queries = 0;
    ix.scan_timed = 0;
    std::lock_guard<std::mutex> lk(ix.tmu);
    ix.scan_ms = 0.0;
    return SINDI_OK;
}

void sindi_index_free(sindi_index* index) {
    if (!index) return;
    {
        DeviceGuard dg(index->impl.device);
        (void)cudaDeviceSynchronize();
        free_index_memory(index->impl, nullptr);
    }
    delete index;
}

}  // extern "C"

// Graph-captured searches (sindi_plan_*): the batched schedule of a fixed
// query batch recorded once as a CUDA graph, then replayed with one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>

#include "common.cuh"
#include "index.cuh"
#include "nvtx.cuh"

namespace sindi {

constexpr size_t kPlanWorkspaceBudget = (size_t)4 << 30;  // device bytes of a plan's working memory

struct Plan {
    const IndexImpl* ix = nullptr;
    int64_t n_queries = 0;
    uint64_t kernels = 0;      // kernel nodes of the graph (launches per replay)
    uint64_t scans = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void free_plan(Plan& p) {
    if (p.exec) (void)cudaGraphExecDestroy(p.exec);
    if (p.graph) (void)cudaGraphDestroy(p.graph);
    if (p.capture_stream) (void)cudaStreamDestroy(p.capture_stream);
    if (p.ws) (void)cudaFree(p.ws);
    p = Plan();
}

}  // namespace sindi

using namespace sindi;

struct sindi_plan {
    Plan impl;
};

extern "C" {

sindi_status sindi_plan_create(const sindi_index* index, const int64_t* q_indptr, const int32_t* q_indices,
                               const float* q_values, int64_t n_queries, const sindi_search_params* params,
                               uint32_t* out_ids, float* out_scores, sindi_plan** out) {
    NvtxRange range("sindi_plan_create n_queries=%lld k=%lld", (long long)n_queries,
                    params ? (long long)params->k : -1LL);
    set_last_error("");
    if (!index || !params || !out || !q_indptr || !q_indices || !q_values || !out_ids || !out_scores ||
        n_queries <= 0 || n_queries > 65535) {
        set_last_error("index, params, query and output buffers must be given; 1 <= n_queries <= 65535");
        return SINDI_ERR_INVALID_ARG;
    }
    sindi_search_params prm = *params;
    if (prm.k < 1 || prm.k > kMaxK || (prm.gamma != 0 && (prm.gamma < prm.k || prm.gamma > kMaxGamma)) ||
        !(prm.beta > 0.0 && prm.beta <= 1.0) ||
        !valid_block_threads(prm.block_threads) || prm.group > kMaxQueryGroup ||
        prm.accumulator > SINDI_ACCUM_FIXED32) {
        set_last_error("k in [1, 1024]; gamma 0 or in [k, 8192]; beta in (0, 1]; block_threads 0, 1 (pipelined), 256, 512 or 1024; group 0..8; accumulator 0..2");
        return SINDI_ERR_INVALID_ARG;
    }
    if (prm.beta < 1.0) {
        set_last_error("query pruning (beta < 1) allocates its pruned queries: use sindi_search");
        return SINDI_ERR_UNSUPPORTED;
    }
    prm.mode = SINDI_MODE_BATCHED;
    const IndexImpl& ix = index->impl;
    int prev = -1;
    (void)cudaGetDevice(&prev);
    (void)cudaSetDevice(ix.device);
    auto* h = new (std::nothrow) sindi_plan;
    if (!h) return SINDI_ERR_OOM;
    Plan& P = h->impl;
    P.ix = &ix;
    P.n_queries = n_queries;
    sindi_status st = SINDI_OK;
    try {
        configure_search_kernels(ix.device);
        const uint64_t launches0 = ix.launches.load(), scans0 = ix.scan_launches.load();
        // the whole batch in one launch group when its working memory fits the budget; otherwise the
        // graph holds several launch groups that reuse one workspace (still one graph launch per run)
        const size_t one = search_workspace_bytes(ix, prm, 1);
        P.ws_bytes = std::min(search_workspace_bytes(ix, prm, n_queries), std::max(one, kPlanWorkspaceBudget));
        SINDI_CUDA(cudaMalloc(&P.ws, P.ws_bytes));
        SINDI_CUDA(cudaStreamCreateWithFlags(&P.capture_stream, cudaStreamNonBlocking));
        SINDI_CUDA(cudaStreamBeginCapture(P.capture_stream, cudaStreamCaptureModeThreadLocal));
        st = search_in_workspace(ix, q_indptr, q_indices, q_values, n_queries, prm, out_ids, out_scores,
                                 P.capture_stream, P.ws, P.ws_bytes);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(P.capture_stream, &g);
        P.graph = g;
        if (st == SINDI_OK) {
            SINDI_CUDA(ce);
            SINDI_CUDA(cudaGraphInstantiate(&P.exec, P.graph, 0));
        }
        // capture counted the launches once; each replay counts them again
        P.kernels = ix.launches.load() - launches0;
        P.scans = ix.scan_launches.load() - scans0;
        ix.launches -= P.kernels;
        ix.scan_launches -= P.scans;
    } catch (const CudaError& e) {
        set_last_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");
        st = e.code == cudaErrorMemoryAllocation ? SINDI_ERR_OOM : SINDI_ERR_CUDA;
    }
    if (prev >= 0) (void)cudaSetDevice(prev);
    if (st != SINDI_OK) {
        free_plan(P);
        delete h;
        return st;
    }
    *out = h;
    return SINDI_OK;
}

sindi_status sindi_plan_launch(sindi_plan* plan, void* stream) {
    NvtxRange range("sindi_plan_launch");
    if (!plan || !plan->impl.exec) return SINDI_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(plan->impl.exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
        return SINDI_ERR_CUDA;
    }
    plan->impl.ix->queries += (uint64_t)plan->impl.n_queries;
    plan->impl.ix->launches += plan->impl.kernels;
    plan->impl.ix->scan_launches += plan->impl.scans;
    return SINDI_OK;
}

void sindi_plan_free(sindi_plan* plan) {
    if (!plan) return;
    int prev = -1;
    (void)cudaGetDevice(&prev);
    (void)cudaSetDevice(plan->impl.ix->device);
    (void)cudaDeviceSynchronize();
    free_plan(plan->impl);
    if (prev >= 0) (void)cudaSetDevice(prev);
    delete plan;
}

}  // extern "C"

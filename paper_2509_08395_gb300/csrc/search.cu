// Search on the device: Algorithm 4 per query, with Algorithm 2 as its coarse
// stage.
//
//   scan_window  (one block per (query, window)): the query's postings in the
//       window, I_{j,w} for every term j, are scatter-added into an FP32 score
//       array A[lambda] in shared memory (Alg. 2, the product + accumulation
//       loops); then the window's best g (score, id) pairs are selected by a
//       radix select over A (the heap update of Alg. 2) and appended to the
//       query's candidate list. A per-query bound (the best threshold any
//       finished window has published) drops candidates that cannot reach
//       the global top g.
//   merge        (one block per query): the global top g of all windows
//       (the heap H of Alg. 2 across windows). With gamma = 0 these are the
//       sorted results; otherwise they are the gamma reorder candidates.
//   rerank       (several blocks per query): delta(x_i, q) from the unpruned
//       document and the unpruned query (Alg. 4, the reorder loop); the last
//       block of a query selects and sorts the top k.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "primitives.cuh"

namespace sindi {

constexpr int kScanThreads = 512;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kTermChunk = kScanThreads;   // query terms staged per pass (one per thread)
constexpr int kScanUnroll = 8;             // postings in flight per lane
constexpr int kMergeThreads = 512;
constexpr int kRerankThreads = 256;
constexpr int kRerankDocsPerBlock = 16;
constexpr int kHashSlots = 4096;           // query hash (load <= 1/2 for kMaxQueryTerms)
constexpr int kQueryTermLimit = kHashSlots / 2;

struct ScanArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    uint32_t g;                     // candidates kept per query (min(gamma or k, N))
    uint64_t* cand;                 // [queries][cand_cap]
    uint32_t* cand_count;           // [queries]
    unsigned long long* bound;      // [queries]
    uint32_t cand_cap;
};

template <int DT>
__device__ __forceinline__ float load_value(const void* pval, uint32_t p) {
    if (DT == SINDI_F32) {
        return __ldg(static_cast<const float*>(pval) + p);
    } else if (DT == SINDI_F16) {
        return __half2float(__ldg(static_cast<const __half*>(pval) + p));
    } else {
        __nv_fp8_storage_t c = __ldg(static_cast<const unsigned char*>(pval) + p);
        return __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
    }
}

// last t in [0, n) with pre[t] <= f (pre[0] = 0 <= f)
__device__ __forceinline__ int term_of(const uint32_t* pre, int n, uint32_t f) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int DT, bool QUERY_MAJOR>
__global__ void __launch_bounds__(kScanThreads) scan_window_kernel(ScanArgs a) {
    extern __shared__ float A[];                    // [lambda]
    __shared__ uint32_t t_start[kTermChunk];
    __shared__ uint32_t t_pre[kTermChunk + 1];
    __shared__ float t_w[kTermChunk];
    __shared__ uint32_t red[kScanWarps + 1];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t st[4];
    __shared__ unsigned long long s_bound;

    const DevIndex& ix = a.ix;
    const uint32_t w = QUERY_MAJOR ? blockIdx.y : blockIdx.x;
    const uint32_t y = QUERY_MAJOR ? blockIdx.x : blockIdx.y;
    const int64_t r = a.q_first + y;
    const uint32_t lambda = ix.lambda;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int64_t qb = a.q_indptr[r];
    const int nt = (int)(a.q_indptr[r + 1] - qb);

    for (uint32_t m = threadIdx.x; m < lambda; m += kScanThreads) A[m] = 0.0f;

    for (int c0 = 0; c0 < nt; c0 += kTermChunk) {
        const int nc = min(kTermChunk, nt - c0);
        __syncthreads();  // previous chunk fully consumed
        uint32_t len = 0;
        if ((int)threadIdx.x < nc) {
            const int32_t j = a.q_indices[qb + c0 + threadIdx.x];
            const float qv = a.q_values[qb + c0 + threadIdx.x];
            uint32_t start = 0;
            float wq = 0.0f;
            if (j >= 0 && j < ix.dim && isfinite(qv)) {
                const uint64_t s = (uint64_t)j * ix.sigma + w;
                start = ix.seg[s];
                len = ix.seg[s + 1] - start;
                wq = (DT == SINDI_F8E4M3) ? qv * ix.scale[j] : qv;
            } else if (w == 0) {
                atomicOr(ix.err, (j < 0 || j >= ix.dim) ? kErrQueryDim : kErrQueryValue);
            }
            t_start[threadIdx.x] = start;
            t_w[threadIdx.x] = wq;
        }
        uint32_t total;
        const uint32_t excl = block_exclusive_sum<uint32_t, kScanThreads>(len, &total, red);
        if ((int)threadIdx.x < nc) t_pre[threadIdx.x] = excl;
        __syncthreads();

        // scatter-add: lane-interleaved over the flattened postings of the chunk
        for (uint32_t base = (uint32_t)warp * 32u * kScanUnroll; base < total;
             base += (uint32_t)kScanWarps * 32u * kScanUnroll) {
            uint32_t id[kScanUnroll];
            float pr[kScanUnroll];
#pragma unroll
            for (int u = 0; u < kScanUnroll; u++) {
                const uint32_t f = base + (uint32_t)u * 32u + (uint32_t)lane;
                id[u] = 0xFFFFFFFFu;
                pr[u] = 0.0f;
                if (f < total) {
                    const int t = term_of(t_pre, nc, f);
                    const uint32_t p = t_start[t] + (f - t_pre[t]);
                    id[u] = __ldg(ix.pid + p);
                    pr[u] = t_w[t] * load_value<DT>(ix.pval, p);
                }
            }
#pragma unroll
            for (int u = 0; u < kScanUnroll; u++)
                if (id[u] != 0xFFFFFFFFu) atomicAdd(&A[id[u]], pr[u]);
        }
    }
    __syncthreads();

    // window top-g (Alg. 2 heap update), ids >= N are not candidates
    const int64_t gbase = (int64_t)w * lambda;
    const int64_t rest = ix.n_docs - gbase;
    const int n_eff = (int)(rest < (int64_t)lambda ? rest : (int64_t)lambda);
    const int g_w = (int)a.g < n_eff ? (int)a.g : n_eff;
    auto key_of = [&](int i) -> uint64_t { return result_key(A[i], (uint32_t)(gbase + i)); };
    uint64_t T = 0;
    if (n_eff > g_w) T = block_select_threshold<kScanThreads>(key_of, n_eff, g_w, hist, st);
    if (threadIdx.x == 0) {
        unsigned long long* bp = a.bound + y;
        unsigned long long B;
        if (g_w == (int)a.g) {
            unsigned long long old = atomicMax(bp, (unsigned long long)T);
            B = old > T ? old : T;
        } else {
            unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(bp);
            B = cur > T ? cur : T;
        }
        s_bound = B;
    }
    __syncthreads();
    const uint64_t B = s_bound;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t* cand = a.cand + (size_t)y * a.cand_cap;
    for (int base = 0; base < n_eff; base += kScanThreads) {
        const int i = base + threadIdx.x;
        uint64_t k = 0;
        bool ok = false;
        if (i < n_eff) {
            k = key_of(i);
            ok = k >= B;
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        uint32_t wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(a.cand_count + y, (uint32_t)__popc(bal));
        wbase = __shfl_sync(kFull, wbase, 0);
        if (ok) {
            const uint32_t pos = wbase + (uint32_t)__popc(bal & lt);
            if (pos < a.cand_cap) cand[pos] = k;
            else atomicOr(ix.err, kErrCandOverflow);
        }
    }
}

// ---------------------------------------------------------------------------
// Query checks shared by merge and rerank: an open-addressing hash of the
// query's dims in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_slot(int32_t j) { return ((uint32_t)j * 2654435761u) >> (32 - 12); }

template <int BLOCK>
__device__ void build_query_hash(const int32_t* qi, const float* qv, int nt, int32_t dim, int32_t* hk, float* hv,
                                 uint32_t* err, bool report) {
    for (int s = threadIdx.x; s < kHashSlots; s += BLOCK) hk[s] = -1;
    __syncthreads();
    if (nt > kQueryTermLimit) {
        if (report && threadIdx.x == 0) atomicOr(err, kErrQueryTooLong);
        return;
    }
    for (int t = threadIdx.x; t < nt; t += BLOCK) {
        const int32_t j = qi[t];
        const float v = qv[t];
        if (j < 0 || j >= dim) {
            if (report) atomicOr(err, kErrQueryDim);
            continue;
        }
        if (!isfinite(v)) {
            if (report) atomicOr(err, kErrQueryValue);
            continue;
        }
        uint32_t s = hash_slot(j);
        for (int probe = 0; probe < kHashSlots; probe++) {
            int32_t old = atomicCAS(&hk[s], -1, j);
            if (old == -1) {
                hv[s] = v;
                break;
            }
            if (old == j) {
                if (report) atomicOr(err, kErrQueryDup);
                break;
            }
            s = (s + 1) & (kHashSlots - 1);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float query_weight(const int32_t* hk, const float* hv, int32_t j) {
    uint32_t s = hash_slot(j);
    for (int probe = 0; probe < kHashSlots; probe++) {
        int32_t k = hk[s];
        if (k == j) return hv[s];
        if (k == -1) return 0.0f;
        s = (s + 1) & (kHashSlots - 1);
    }
    return 0.0f;
}

// Writes the selected keys (already gathered in s[0..cnt), cnt <= kMaxK) as
// sorted results of query row y: ids and scores, padded to k.
template <int BLOCK>
__device__ void write_sorted_results(uint64_t* s, int cnt, uint32_t k, uint32_t* out_ids, float* out_scores,
                                     int64_t y) {
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    for (int i = cnt + threadIdx.x; i < p2; i += BLOCK) s[i] = 0;
    __syncthreads();
    block_bitonic_sort_desc<BLOCK>(s, p2);
    for (uint32_t t = threadIdx.x; t < k; t += BLOCK) {
        uint32_t id = 0xFFFFFFFFu;
        float sc = -INFINITY;
        if ((int)t < cnt) {
            id = key_id(s[t]);
            sc = key_score(s[t]);
        }
        out_ids[(size_t)y * k + t] = id;
        out_scores[(size_t)y * k + t] = sc;
    }
}

struct MergeArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    uint32_t g;
    uint64_t* cand;
    uint32_t* cand_count;
    unsigned long long* bound;
    uint32_t cand_cap;
    int final_stage;           // 1: g = min(k, N) results are the answer
    uint32_t k;
    uint32_t* out_ids;         // rows indexed from q_first
    float* out_scores;
    uint64_t* top;             // [queries][top_cap] when final_stage == 0
    uint32_t* top_count;
    uint32_t top_cap;
};

__global__ void __launch_bounds__(kMergeThreads) merge_kernel(MergeArgs a) {
    __shared__ int32_t hk[kHashSlots];
    __shared__ float hv[kHashSlots];
    __shared__ uint64_t s[kMaxK];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_n;
    const uint32_t y = blockIdx.x;
    const int64_t r = a.q_first + y;
    const int64_t qb = a.q_indptr[r];
    const int nt = (int)(a.q_indptr[r + 1] - qb);
    build_query_hash<kMergeThreads>(a.q_indices + qb, a.q_values + qb, nt, a.ix.dim, hk, hv, a.ix.err, true);

    const uint32_t C = min(a.cand_count[y], a.cand_cap);
    const uint64_t* cand = a.cand + (size_t)y * a.cand_cap;
    const int g = (int)(a.g < C ? a.g : C);
    auto key_of = [&](int i) -> uint64_t { return cand[i]; };
    uint64_t T = 0;
    if ((int)C > g) T = block_select_threshold<kMergeThreads>(key_of, (int)C, g, hist, st);
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    for (uint32_t base = 0; base < C; base += kMergeThreads) {
        const uint32_t i = base + threadIdx.x;
        uint64_t k = 0;
        bool ok = false;
        if (i < C) {
            k = cand[i];
            ok = k >= T;
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        uint32_t wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(&s_n, (uint32_t)__popc(bal));
        wb = __shfl_sync(kFull, wb, 0);
        if (ok) {
            const uint32_t pos = wb + (uint32_t)__popc(bal & lt);
            if (a.final_stage) {
                if (pos < kMaxK) s[pos] = k;
            } else if (pos < a.top_cap) {
                a.top[(size_t)y * a.top_cap + pos] = k;
            }
        }
    }
    __syncthreads();
    if (a.final_stage) {
        write_sorted_results<kMergeThreads>(s, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores, r);
    } else if (threadIdx.x == 0) {
        a.top_count[y] = min(s_n, a.top_cap);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.cand_count[y] = 0;
        a.bound[y] = 0ull;
    }
}

struct RerankArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    const uint64_t* top;
    const uint32_t* top_count;
    uint32_t top_cap;
    uint64_t* rr;              // [queries][top_cap]
    uint32_t* done;            // [queries]
    uint32_t k;
    uint32_t* out_ids;
    float* out_scores;
};

__global__ void __launch_bounds__(kRerankThreads) rerank_kernel(RerankArgs a) {
    __shared__ int32_t hk[kHashSlots];
    __shared__ float hv[kHashSlots];
    __shared__ uint64_t s[kMaxK];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_n;
    __shared__ int s_last;
    const uint32_t y = blockIdx.y;
    const int64_t r = a.q_first + y;
    const int64_t qb = a.q_indptr[r];
    const int nt = (int)(a.q_indptr[r + 1] - qb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t g = min(a.top_count[y], a.top_cap);
    const uint32_t lo = blockIdx.x * kRerankDocsPerBlock;
    const uint32_t hi = g < lo + kRerankDocsPerBlock ? g : lo + kRerankDocsPerBlock;
    if (lo < hi) {
        build_query_hash<kRerankThreads>(a.q_indices + qb, a.q_values + qb, nt, a.ix.dim, hk, hv, a.ix.err, false);
        for (uint32_t idx = lo + warp; idx < hi; idx += kRerankThreads / 32) {
            const uint64_t key = a.top[(size_t)y * a.top_cap + idx];
            const uint32_t id = key_id(key);
            const int64_t b = a.ix.indptr[id], e = a.ix.indptr[id + 1];
            float acc = 0.0f;
            for (int64_t p = b + lane; p < e; p += 32) {
                const float qw = query_weight(hk, hv, __ldg(a.ix.indices + p));
                acc = fmaf(__ldg(a.ix.values + p), qw, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (lane == 0) a.rr[(size_t)y * a.top_cap + idx] = result_key(acc, id);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.done + y, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint64_t* rr = a.rr + (size_t)y * a.top_cap;
    const int kk = (int)(a.k < g ? a.k : g);
    auto key_of = [&](int i) -> uint64_t { return __ldcg(rr + i); };
    uint64_t T = 0;
    if ((int)g > kk) T = block_select_threshold<kRerankThreads>(key_of, (int)g, kk, hist, st);
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t base = 0; base < g; base += kRerankThreads) {
        const uint32_t i = base + threadIdx.x;
        uint64_t k = 0;
        bool ok = false;
        if (i < g) {
            k = __ldcg(rr + i);
            ok = k >= T;
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        uint32_t wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(&s_n, (uint32_t)__popc(bal));
        wb = __shfl_sync(kFull, wb, 0);
        if (ok && wb + __popc(bal & lt) < kMaxK) s[wb + __popc(bal & lt)] = k;
    }
    __syncthreads();
    write_sorted_results<kRerankThreads>(s, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores, r);
    if (threadIdx.x == 0) a.done[y] = 0;
}

// Rows of an empty index: every slot is padding.
__global__ void pad_results_kernel(uint32_t* out_ids, float* out_scores, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out_ids[i] = 0xFFFFFFFFu;
        out_scores[i] = -INFINITY;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int DT, bool QM>
static void launch_scan(const ScanArgs& a, uint32_t sigma, uint32_t nq, size_t smem, cudaStream_t s) {
    static bool configured = false;  // per instantiation; the attribute is per function
    if (!configured) {
        SINDI_CUDA(cudaFuncSetAttribute(scan_window_kernel<DT, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(kMaxWindow * sizeof(float))));
        configured = true;
    }
    dim3 grid = QM ? dim3(nq, sigma) : dim3(sigma, nq);
    scan_window_kernel<DT, QM><<<grid, kScanThreads, smem, s>>>(a);
    SINDI_CUDA(cudaGetLastError());
}

static void launch_scan_any(int dt, bool qm, const ScanArgs& a, uint32_t sigma, uint32_t nq, size_t smem,
                            cudaStream_t s) {
    if (dt == SINDI_F32) qm ? launch_scan<SINDI_F32, true>(a, sigma, nq, smem, s)
                            : launch_scan<SINDI_F32, false>(a, sigma, nq, smem, s);
    else if (dt == SINDI_F16) qm ? launch_scan<SINDI_F16, true>(a, sigma, nq, smem, s)
                                 : launch_scan<SINDI_F16, false>(a, sigma, nq, smem, s);
    else qm ? launch_scan<SINDI_F8E4M3, true>(a, sigma, nq, smem, s)
            : launch_scan<SINDI_F8E4M3, false>(a, sigma, nq, smem, s);
}

sindi_status search_impl(const IndexImpl& ix, const int64_t* q_indptr, const int32_t* q_indices,
                         const float* q_values, int64_t n_queries, const sindi_search_params& prm,
                         uint32_t* out_ids, float* out_scores, cudaStream_t stream) {
    const int64_t N = ix.n_docs;
    const uint32_t k = prm.k;
    if (n_queries == 0) return SINDI_OK;
    if (N == 0) {
        pad_results_kernel<<<256, 256, 0, stream>>>(out_ids, out_scores, n_queries * (int64_t)k);
        SINDI_CUDA(cudaGetLastError());
        ix.launches++;
        return SINDI_OK;
    }
    const bool final_stage = prm.gamma == 0;
    const uint32_t g = (uint32_t)std::min<int64_t>(final_stage ? k : prm.gamma, N);
    const uint32_t g_window = std::min<uint32_t>(g, ix.lambda);
    const uint32_t cand_cap = ix.sigma * g_window;
    const uint32_t top_cap = final_stage ? 1 : g;
    const size_t per_query = (size_t)cand_cap * 8 + 4 + 8 + (size_t)top_cap * 16 + 8;
    const bool batched = prm.mode == SINDI_MODE_BATCHED;
    int64_t chunk = 1;
    if (batched) {
        const size_t budget = (size_t)1 << 31;  // 2 GiB of candidate workspace per launch group
        chunk = std::max<int64_t>(1, std::min<int64_t>(n_queries, (int64_t)(budget / per_query)));
        chunk = std::min<int64_t>(chunk, 65535);
    }
    Pool P{ix.pool, stream};
    uint64_t* cand = P.alloc<uint64_t>((size_t)cand_cap * chunk);
    uint32_t* cand_count = P.alloc<uint32_t>(chunk);
    unsigned long long* bound = P.alloc<unsigned long long>(chunk);
    uint64_t* top = P.alloc<uint64_t>((size_t)top_cap * chunk);
    uint32_t* top_count = P.alloc<uint32_t>(chunk);
    uint64_t* rr = P.alloc<uint64_t>((size_t)top_cap * chunk);
    uint32_t* done = P.alloc<uint32_t>(chunk);
    SINDI_CUDA(cudaMemsetAsync(cand_count, 0, 4 * chunk, stream));
    SINDI_CUDA(cudaMemsetAsync(bound, 0, 8 * chunk, stream));
    SINDI_CUDA(cudaMemsetAsync(done, 0, 4 * chunk, stream));

    const DevIndex dix = ix.dev();
    const size_t scan_smem = (size_t)ix.lambda * sizeof(float);
    const bool timing = ix.timing.load() != 0;
    std::vector<cudaEvent_t> evs;

    for (int64_t q0 = 0; q0 < n_queries; q0 += chunk) {
        const uint32_t nq = (uint32_t)std::min<int64_t>(chunk, n_queries - q0);
        ScanArgs sa{dix, q_indptr, q_indices, q_values, q0, g, cand, cand_count, bound, cand_cap};
        if (timing) {
            cudaEvent_t e0, e1;
            SINDI_CUDA(cudaEventCreate(&e0));
            SINDI_CUDA(cudaEventCreate(&e1));
            evs.push_back(e0);
            evs.push_back(e1);
            SINDI_CUDA(cudaEventRecord(e0, stream));
        }
        // query-major grids put the queries of one window next to each other
        // (shared segments stay in L2); gridDim.y limits sigma to 65535 there
        launch_scan_any(ix.dtype, batched && ix.sigma <= 65535u, sa, ix.sigma, nq, scan_smem, stream);
        if (timing) SINDI_CUDA(cudaEventRecord(evs.back(), stream));
        MergeArgs ma{dix, q_indptr, q_indices, q_values, q0, g, cand, cand_count, bound, cand_cap,
                     final_stage ? 1 : 0, k, out_ids, out_scores, top, top_count, top_cap};
        merge_kernel<<<nq, kMergeThreads, 0, stream>>>(ma);
        SINDI_CUDA(cudaGetLastError());
        ix.launches += 2;
        ix.scan_launches += 1;
        if (!final_stage) {
            RerankArgs ra{dix, q_indptr, q_indices, q_values, q0, top, top_count, top_cap, rr, done, k,
                          out_ids, out_scores};
            dim3 grid(ceil_div_u32(g, kRerankDocsPerBlock), nq);
            rerank_kernel<<<grid, kRerankThreads, 0, stream>>>(ra);
            SINDI_CUDA(cudaGetLastError());
            ix.launches += 1;
        }
    }
    ix.queries += (uint64_t)n_queries;
    P.free(cand);
    P.free(cand_count);
    P.free(bound);
    P.free(top);
    P.free(top_count);
    P.free(rr);
    P.free(done);
    if (timing) {
        SINDI_CUDA(cudaStreamSynchronize(stream));
        double ms = 0.0;
        for (size_t i = 0; i + 1 < evs.size(); i += 2) {
            float t = 0.0f;
            SINDI_CUDA(cudaEventElapsedTime(&t, evs[i], evs[i + 1]));
            ms += t;
        }
        for (auto e : evs) cudaEventDestroy(e);
        std::lock_guard<std::mutex> lk(ix.tmu);
        ix.scan_ms += ms;
        ix.scan_timed += evs.size() / 2;
    }
    return SINDI_OK;
}

// ---------------------------------------------------------------------------
// Search without allocation (sindi_search_noalloc). The paper has no
// counterpart: this serves callers that may not allocate device memory while
// they run (their memory is fixed up front, or an allocation's implicit
// synchronisation is not allowed on their path). All working memory of the
// search comes from one file-scope device array, sized kNoAllocScratchBytes.
// Every call shares it: calls whose work overlaps on the GPU race.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device. Resolved once per
// device (cudaGetSymbolAddress, with that device current) and cached.
static cudaError_t noalloc_scratch_address(int device, unsigned char** out) {
    static std::mutex mu;
    static std::map<int, unsigned char*> addr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = addr.find(device);
    if (it != addr.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    unsigned char* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[device] = p;
    *out = p;
    return cudaSuccess;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

sindi_status search_noalloc_impl(const IndexImpl& ix, const int64_t* q_indptr, const int32_t* q_indices,
                                 const float* q_values, int64_t n_queries, const sindi_search_params& prm,
                                 uint32_t* out_ids, float* out_scores, cudaStream_t stream) {
    unsigned char* base = nullptr;
    cudaError_t ce = noalloc_scratch_address(ix.device, &base);
    if (ce != cudaSuccess) {
        set_last_error(std::string("sindi_search_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce));
        return SINDI_ERR_CUDA;
    }
    const int64_t N = ix.n_docs;
    const uint32_t k = prm.k;
    if (n_queries == 0) return SINDI_OK;
    if (N == 0) {
        pad_results_kernel<<<256, 256, 0, stream>>>(out_ids, out_scores, n_queries * (int64_t)k);
        SINDI_CUDA(cudaGetLastError());
        return SINDI_OK;
    }
    const bool final_stage = prm.gamma == 0;
    const uint32_t g = (uint32_t)std::min<int64_t>(final_stage ? k : prm.gamma, N);
    const uint32_t cand_cap = ix.sigma * std::min<uint32_t>(g, ix.lambda);
    const uint32_t top_cap = final_stage ? 1 : g;
    // scratch of a group of c queries: six arrays, each 256-byte aligned
    auto need = [&](int64_t c) {
        return align256((size_t)cand_cap * 8 * c) + align256(4 * (size_t)c) + align256(8 * (size_t)c) +
               align256((size_t)top_cap * 8 * c) + align256(4 * (size_t)c) + align256((size_t)top_cap * 8 * c) +
               align256(4 * (size_t)c);
    };
    if (need(1) > kNoAllocScratchBytes) {
        set_last_error("sindi_search_noalloc: one query needs " + std::to_string(need(1)) +
                       " bytes of scratch (n_windows * min(candidates, window) * 8 + ...), more than the " +
                       std::to_string(kNoAllocScratchBytes) + "-byte static scratch area; use sindi_search");
        return SINDI_ERR_UNSUPPORTED;
    }
    const bool batched = prm.mode == SINDI_MODE_BATCHED;
    int64_t chunk = 1;
    if (batched) {
        chunk = std::min<int64_t>(n_queries, 65535);
        while (chunk > 1 && need(chunk) > kNoAllocScratchBytes) chunk = std::max<int64_t>(1, chunk / 2);
    }
    unsigned char* q = base;
    auto carve = [&](size_t bytes) {
        unsigned char* r = q;
        q += align256(bytes);
        return r;
    };
    uint64_t* cand = reinterpret_cast<uint64_t*>(carve((size_t)cand_cap * 8 * chunk));
    uint32_t* cand_count = reinterpret_cast<uint32_t*>(carve(4 * (size_t)chunk));
    unsigned long long* bound = reinterpret_cast<unsigned long long*>(carve(8 * (size_t)chunk));
    uint64_t* top = reinterpret_cast<uint64_t*>(carve((size_t)top_cap * 8 * chunk));
    uint32_t* top_count = reinterpret_cast<uint32_t*>(carve(4 * (size_t)chunk));
    uint64_t* rr = reinterpret_cast<uint64_t*>(carve((size_t)top_cap * 8 * chunk));
    uint32_t* done = reinterpret_cast<uint32_t*>(carve(4 * (size_t)chunk));
    // the array keeps the previous call's contents: clear the counters the kernels start from
    SINDI_CUDA(cudaMemsetAsync(cand_count, 0, 4 * chunk, stream));
    SINDI_CUDA(cudaMemsetAsync(bound, 0, 8 * chunk, stream));
    SINDI_CUDA(cudaMemsetAsync(done, 0, 4 * chunk, stream));

    const DevIndex dix = ix.dev();
    const size_t scan_smem = (size_t)ix.lambda * sizeof(float);
    for (int64_t q0 = 0; q0 < n_queries; q0 += chunk) {
        const uint32_t nq = (uint32_t)std::min<int64_t>(chunk, n_queries - q0);
        ScanArgs sa{dix, q_indptr, q_indices, q_values, q0, g, cand, cand_count, bound, cand_cap};
        launch_scan_any(ix.dtype, batched && ix.sigma <= 65535u, sa, ix.sigma, nq, scan_smem, stream);
        MergeArgs ma{dix, q_indptr, q_indices, q_values, q0, g, cand, cand_count, bound, cand_cap,
                     final_stage ? 1 : 0, k, out_ids, out_scores, top, top_count, top_cap};
        merge_kernel<<<nq, kMergeThreads, 0, stream>>>(ma);
        SINDI_CUDA(cudaGetLastError());
        ix.launches += 2;
        ix.scan_launches += 1;
        if (!final_stage) {
            RerankArgs ra{dix, q_indptr, q_indices, q_values, q0, top, top_count, top_cap, rr, done, k,
                          out_ids, out_scores};
            dim3 grid(ceil_div_u32(g, kRerankDocsPerBlock), nq);
            rerank_kernel<<<grid, kRerankThreads, 0, stream>>>(ra);
            SINDI_CUDA(cudaGetLastError());
            ix.launches += 1;
        }
    }
    ix.queries += (uint64_t)n_queries;
    return SINDI_OK;
}

}  // namespace sindi

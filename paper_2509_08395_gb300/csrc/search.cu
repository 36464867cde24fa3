// Search on the device: Algorithm 4 per query, with Algorithm 2 as its coarse
// stage.
//
//   scan_window  (one block per (query, window)): the query's postings in the
//       window, I_{j,w} for every term j, are scatter-added into a score array
//       A[lambda] in shared memory (Alg. 2, the product + accumulation loops):
//       FP32 sums, or 32-bit fixed-point sums of the FP32 products (the default
//       when the search reorders; fixed_point.cuh), read as FP32 scores by the
//       cut. The block then histograms the window's scores on the top 12
//       bits of their order key and emits every slot in the bins at or above
//       the bin that holds its g-th best slot (the window's share of the heap
//       update of Alg. 2). When ties crowd that bin, an exact radix select
//       emits exactly the best g. Each block adds the histogram of what it
//       emitted to a per-query histogram H. Where earlier windows of the query
//       are complete (batched schedules: a snapshot taken at the block's
//       start; the plain schedule's second launch: H read after the
//       accumulation), a bin reached by g already emitted slots bounds what
//       can still enter the answer, and a window whose slots above that bound
//       fit its budget emits them in one pass, with no cut.
//   merge        (one block per query up to 16384 candidates, a few above):
//       from H, the bin of the global g-th best candidate; candidates below
//       it are dropped, the rest (about g) gathered and the exact best g
//       selected in shared memory (the heap H of Alg. 2 across windows).
//       With gamma = 0 these are the sorted results; otherwise they are the
//       gamma reorder candidates.
//   rerank       (one half-warp per candidate): delta(x_i, q) from the
//       unpruned document and the unpruned query (Alg. 4, the reorder loop);
//       the last block of a query sorts the scores and writes the top k.
//
// Order keys (common.cuh) make every comparison exact: (score desc, id asc).
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fixed_point.cuh"
#include "index.cuh"
#include "mass.cuh"
#include "primitives.cuh"

namespace sindi {

constexpr int kScanThreadsPlain = 512;     // two blocks per SM: the windows of concurrent queries interleave
constexpr int kScanThreadsBatched = 512;   // many windows: two blocks per SM overlap their phases
constexpr int kPlainLanes = 24;            // plain schedule: query chains in flight at once
constexpr uint32_t kPlainPipeItems = 6;    // plain schedule, pipelined scan: windows per block
constexpr uint32_t kSplitMinWindows = 8;   // plain schedule: a query of this many windows or more scans
constexpr uint32_t kSplitFraction = 8;     // its first 1/kSplitFraction windows first
constexpr int kMaxScanWarps = 1024 / 32;   // largest scan block
constexpr int kChunkTable = 2048;          // chunks mapped to their list by a table (then a search)
constexpr int kHistBits = 12;
constexpr int kHistBins = 1 << kHistBits;  // bins on the top 12 bits of a score key
constexpr int kKeyBinShift = 64 - kHistBits;
constexpr int kSubBits = 8;                // second-level bins inside the cut bin
constexpr int kSubBins = 1 << kSubBits;
constexpr int kRelBins = 256;              // window histogram bins below the window's top bin
constexpr int kMergeThreads = 512;
constexpr uint32_t kMergeOneBlock = 16384;  // candidates one merge block gathers alone
constexpr int kRerankThreads = 256;
constexpr int kRerankWarps = kRerankThreads / 32;
constexpr int kRerankU = 16;               // row entries per lane loaded at once
constexpr int kHashSlots = 4096;           // query hash (load <= 1/2 at the term limit)
constexpr int kQueryTermLimit = kHashSlots / 2;

// Working memory of a launch group of queries, all arrays [query][...].
struct Workspace {
    uint32_t* cand_count;   // window candidates appended so far
    uint32_t* fcount;       // merge: candidates kept by the filter
    uint32_t* mticket;      // merge: finished blocks
    uint32_t* rticket;      // rerank: finished blocks
    uint32_t* top_count;    // reorder candidates
    uint32_t* hist;         // [kHistBins] histogram of emitted candidates
    uint64_t* cand;         // [cand_cap]
    uint64_t* fbuf;         // [fcap]
    uint64_t* top;          // [top_cap]
    uint64_t* rr;           // [top_cap]
    uint32_t cand_cap, fcap, top_cap;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of a workspace for c queries, counters first (one memset clears them).
static size_t workspace_counter_bytes(int64_t c) { return align256((size_t)c * 4 * (5 + kHistBins)); }
static size_t workspace_bytes(int64_t c, uint32_t cand_cap, uint32_t fcap, uint32_t top_cap) {
    return workspace_counter_bytes(c) + align256((size_t)c * cand_cap * 8) + align256((size_t)c * fcap * 8) +
           2 * align256((size_t)c * top_cap * 8);
}

static Workspace carve_workspace(unsigned char* base, int64_t c, uint32_t cand_cap, uint32_t fcap, uint32_t top_cap) {
    Workspace w;
    uint32_t* u = reinterpret_cast<uint32_t*>(base);
    w.hist = u;  // first: every query's row starts 16-byte aligned
    w.cand_count = u + c * kHistBins;
    w.fcount = w.cand_count + c;
    w.mticket = w.cand_count + 2 * c;
    w.rticket = w.cand_count + 3 * c;
    w.top_count = w.cand_count + 4 * c;
    unsigned char* q = base + workspace_counter_bytes(c);
    w.cand = reinterpret_cast<uint64_t*>(q);
    q += align256((size_t)c * cand_cap * 8);
    w.fbuf = reinterpret_cast<uint64_t*>(q);
    q += align256((size_t)c * fcap * 8);
    w.top = reinterpret_cast<uint64_t*>(q);
    q += align256((size_t)c * top_cap * 8);
    w.rr = reinterpret_cast<uint64_t*>(q);
    w.cand_cap = cand_cap;
    w.fcap = fcap;
    w.top_cap = top_cap;
    return w;
}

// Floats a window array takes in shared memory: lambda rounded up to 4, so
// that every window starts 16-byte aligned and the cut reads it 4 slots at a
// time (the slots past lambda stay zero and are never candidates).
__host__ __device__ __forceinline__ uint32_t window_stride(uint32_t lambda) { return (lambda + 3u) & ~3u; }

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

// vmax[j] = the largest |stored value| of list I_j over all its windows
// (postings seg[j * sigma] .. seg[(j + 1) * sigma]), one warp per list. It
// bounds every product of term j, which sets the unit of the fixed-point
// window (window_scale_exp).
template <int DT>
__global__ void list_vmax_kernel(const uint32_t* seg, const void* pval, int32_t dim, uint32_t sigma, float* vmax) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < dim; j += warps) {
        const uint32_t lo = seg[(uint64_t)j * sigma], hi = seg[(uint64_t)(j + 1) * sigma];
        float m = 0.0f;
        for (uint32_t p = lo + lane; p < hi; p += 32) m = fmaxf(m, fabsf(load_value<DT>(pval, p)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) vmax[j] = m;
    }
}

void list_value_bounds(IndexImpl& ix, cudaStream_t stream) {
    if (!ix.vmax) {
        Pool P{ix.pool, stream};
        ix.vmax = P.alloc<float>(ix.dim > 0 ? ix.dim : 1);
    }
    if (ix.dim <= 0) return;
    const int64_t blocks = std::min<int64_t>(((int64_t)ix.dim + 7) / 8, 152 * 32);
    if (ix.dtype == SINDI_F32)
        list_vmax_kernel<SINDI_F32><<<(unsigned)blocks, 256, 0, stream>>>(ix.seg, ix.pval, ix.dim, ix.sigma, ix.vmax);
    else if (ix.dtype == SINDI_F16)
        list_vmax_kernel<SINDI_F16><<<(unsigned)blocks, 256, 0, stream>>>(ix.seg, ix.pval, ix.dim, ix.sigma, ix.vmax);
    else
        list_vmax_kernel<SINDI_F8E4M3><<<(unsigned)blocks, 256, 0, stream>>>(ix.seg, ix.pval, ix.dim, ix.sigma,
                                                                             ix.vmax);
    SINDI_CUDA(cudaGetLastError());
}

// Programmatic dependent launch. Kernels after the first of a search call are
// launched so that they may start while the previous kernel still runs; each
// waits here before it touches memory the previous kernels write, and lets
// the next kernel launch early.
__device__ __forceinline__ void wait_previous_kernels() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_kernel() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Eight consecutive postings p0 .. p0 + 7 (p0 a multiple of 8): their window
// ids (two per word) and values, read with aligned vector loads (the posting
// arrays are padded to a multiple of 8 entries).
__device__ __forceinline__ void load_ids8(const uint16_t* pid, uint32_t p0, uint32_t id2[4]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(pid + p0));
    id2[0] = u.x;
    id2[1] = u.y;
    id2[2] = u.z;
    id2[3] = u.w;
}

template <int DT>
__device__ __forceinline__ void load_values8(const void* pval, uint32_t p0, float v[8]) {
    if (DT == SINDI_F32) {
        const float4* f = reinterpret_cast<const float4*>(static_cast<const float*>(pval) + p0);
        const float4 a = __ldg(f), b = __ldg(f + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if (DT == SINDI_F16) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(static_cast<const __half*>(pval) + p0));
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w4[j]));
            v[2 * j] = f.x;
            v[2 * j + 1] = f.y;
        }
    } else {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned char*>(pval) + p0));
        const uint32_t w2[2] = {u.x, u.y};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w2[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
            const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
            const float2 f = __half22float2(__half2(h));
            v[2 * j] = f.x;
            v[2 * j + 1] = f.y;
        }
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

// One warp chunk of one query term's list in one window, in registers: the
// lane's postings are q0 + u (a long list) or q0 + 32 u (a short one), u <
// kChunkU; bit u of lm is set for those inside the segment.
struct Chunk {
    uint32_t id2[kChunkU / 2];  // window ids, two per word (low half first)
    float v[kChunkU];
    uint32_t lm;
    float wq;
    uint32_t vec;               // a long segment's chunk: every lane's 8 ids were loaded
};

// Loads the chunk at offset `off` (a multiple of kChunkLen) of the segment
// [ps, pe). A segment of at least kVecMin postings is tiled on 8-aligned
// groups, lane l owning the 8 consecutive postings of the chunk's l-th group
// (one vector load of ids, one or two of values); a shorter segment (always a
// single chunk) keeps the lanes interleaved, which keeps more of them busy.
// These are the positions the build's bank-aware order is laid out for.
template <int DT>
__device__ __forceinline__ void load_segment_chunk(const DevIndex& ix, uint32_t ps, uint32_t pe, uint32_t off,
                                                   int lane, Chunk& k) {
#pragma unroll
    for (int u = 0; u < kChunkU; u++) k.v[u] = 0.0f;
#pragma unroll
    for (int u = 0; u < kChunkU / 2; u++) k.id2[u] = 0;
    k.lm = 0;
    k.vec = 0;
    if (!checked(segment_in_bounds(ps, pe, ix.pcap), ix.err)) return;
    if (pe - ps >= kVecMin) {
        k.vec = 1;
        const uint32_t q0 = (ps & ~7u) + off + (uint32_t)lane * kChunkU;
        const uint32_t lo = ps > q0 ? ps - q0 : 0u;  // < 8: only the segment's first group
        const uint32_t hi = pe > q0 ? min(pe - q0, (uint32_t)kChunkU) : 0u;
        k.lm = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
        if (k.lm && !checked(group_in_bounds(q0, ix.pcap), ix.err)) k.lm = 0;
        if (k.lm) {
            load_ids8(ix.pid, q0, k.id2);
            load_values8<DT>(ix.pval, q0, k.v);
            if (k.lm != 0xFFu) {
                // a group at the segment's start or end: the postings outside it weigh 0
#pragma unroll
                for (int u = 0; u < kChunkU; u++)
                    if (!((k.lm >> u) & 1u)) k.v[u] = 0.0f;
            }
        }
    } else {
        const uint32_t q0 = ps + (uint32_t)lane;
        const uint32_t n = pe > q0 ? min((pe - q0 + 31u) >> 5, (uint32_t)kChunkU) : 0u;
        k.lm = (1u << n) - 1u;
#pragma unroll
        for (int u = 0; u < kChunkU; u++) {
            const uint32_t p = q0 + 32u * u;
            if (p < pe) {
                k.id2[u >> 1] |= (uint32_t)__ldg(ix.pid + p) << (16 * (u & 1));
                k.v[u] = load_value<DT>(ix.pval, p);
            }
        }
    }
}

// Loads chunk c of a term table (chunks of all its terms, in term order).
template <int DT>
__device__ __forceinline__ void load_chunk(const DevIndex& ix, const uint32_t* t_start, const uint32_t* t_end,
                                           const float* t_w, const uint32_t* c_pre, const uint16_t* c_term,
                                           int nc, uint32_t c, int lane, Chunk& k) {
    const int t = c < (uint32_t)kChunkTable ? (int)c_term[c] : term_of(c_pre, nc, c);
    k.wq = t_w[t];
    load_segment_chunk<DT>(ix, t_start[t], t_end[t], (c - c_pre[t]) * (uint32_t)kChunkLen, lane, k);
}

// The same from the term table's packed records: {start, end, first chunk,
// weight bits} per term, one 16-byte shared load.
template <int DT>
__device__ __forceinline__ void load_chunk_rec(const DevIndex& ix, const uint4* rec, const uint32_t* c_pre,
                                               const uint16_t* c_term, int nc, uint32_t c, int lane, Chunk& k) {
    const int t = c < (uint32_t)kChunkTable ? (int)c_term[c] : term_of(c_pre, nc, c);
    const uint4 r = rec[t];
    k.wq = __uint_as_float(r.w);
    load_segment_chunk<DT>(ix, r.x, r.y, (c - r.z) * (uint32_t)kChunkLen, lane, k);
}

__device__ __forceinline__ uint32_t chunk_slot(const Chunk& k, int u) {
    return (k.id2[u >> 1] >> (16 * (u & 1))) & 0xFFFFu;
}

// Adds a chunk with shared-memory atomics (segments of different terms may
// run at once and meet on a slot).
__device__ __forceinline__ void add_chunk(float* A, uint32_t lambda, uint32_t* err, const Chunk& k) {
#pragma unroll
    for (int u = 0; u < kChunkU; u++)
        if ((k.lm & (1u << u)) && checked(slot_in_bounds(chunk_slot(k, u), lambda), err))
            atomicAdd(&A[chunk_slot(k, u)], k.wq * k.v[u]);
}

// The same into a fixed-point window: each product (its weight already
// carries the window's 2^e) rounded to the nearest unit and added with a
// native shared-memory integer atomic. In a long segment's chunk every lane
// that loaded its group adds all 8 postings: the ones outside the segment
// have value 0 (load_segment_chunk) and add 0 at the slot their load
// returned (an id of a neighbouring segment, or the zero padding: a valid
// slot, and an integer + 0 changes nothing), so the adds need no branch and
// no select.
__device__ __forceinline__ void add_chunk_fixed(int32_t* A, uint32_t lambda, uint32_t* err, const Chunk& k) {
    if (k.vec && !kChecks) {
        if (k.lm) {
#pragma unroll
            for (int u = 0; u < kChunkU; u++)
                atomicAdd(&A[chunk_slot(k, u)], __float2int_rn(k.wq * k.v[u]));
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < kChunkU; u++)
        if ((k.lm & (1u << u)) && checked(slot_in_bounds(chunk_slot(k, u), lambda), err))
            atomicAdd(&A[chunk_slot(k, u)], __float2int_rn(k.wq * k.v[u]));
}

// Chunks of a segment of at least kVecMin postings.
__device__ __forceinline__ uint32_t long_segment_chunks(uint32_t ps, uint32_t pe) {
    return (((pe + 7u) & ~7u) - (ps & ~7u) + kChunkLen - 1) / kChunkLen;
}

// Block-wide: the bin holding the g-th largest element of a BINS-bin
// histogram read through `get`, counting from the top bin. Leaves the bin in
// st[0] (0 when the total is below g), the count strictly above it in st[1],
// its own count in st[2] and the histogram total in st[3]. red: [BLOCK/32 + 1].
template <int BINS, typename S, typename Get>
__device__ void group_find_bin(const Get& get, uint32_t g, uint32_t* red, uint32_t* st) {
    constexpr int BLOCK = S::kThreads;
    constexpr int BPT = (BINS + BLOCK - 1) / BLOCK;  // bins per thread, from the top
    const int tid = S::tid();
    uint32_t c[BPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < BPT; j++) {
        const int b = BINS - 1 - BPT * (int)tid - j;
        c[j] = b >= 0 ? get(b) : 0u;
        s += c[j];
    }
    uint32_t tot;
    const uint32_t ex = group_exclusive_sum<uint32_t, S>(s, &tot, red);
    if (tid == 0) {
        st[0] = 0;
        st[1] = tot;
        st[2] = 0;
        st[3] = tot;
    }
    S::sync();
    if (ex < g && g <= ex + s) {
        uint32_t above = ex;
#pragma unroll
        for (int j = 0; j < BPT; j++) {
            if (above < g && g <= above + c[j]) {
                st[0] = (uint32_t)(BINS - 1 - BPT * (int)tid - j);
                st[1] = above;
                st[2] = c[j];
            }
            above += c[j];
        }
    }
    S::sync();
}

template <int BINS, int BLOCK, typename Get>
__device__ void block_find_bin(const Get& get, uint32_t g, uint32_t* red, uint32_t* st) {
    group_find_bin<BINS, SyncBlock<BLOCK>>(get, g, red, st);
}

// 16-byte asynchronous copy global -> shared (through L2), and its completion.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct ScanArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    uint32_t g;             // candidates per query: min(gamma or k, N)
    uint32_t win_cap;       // most candidates one window may emit without an exact select
    int use_partial;        // read the per-query histogram before emitting: 0 no; 1 copied at the
                            // block's start (batched: earlier windows of the query are done); 2 read
                            // after the accumulation, once the previous launch (the query's first
                            // windows) is complete
    uint32_t w0;            // first window of this launch
    uint32_t nq;            // pipelined scan: query rows and windows of the launch's items
    uint32_t nwin;
    Workspace ws;
    int fixed;              // 1: the window accumulates in 32-bit fixed point (sindi_accumulator FIXED32)
};

// Shared-memory scratch of one window cut, owned by the threads that select.
struct CutScratch {
    uint32_t* hist;         // [kHistBins]
    uint32_t* hist2;        // [kSubBins]
    unsigned char* region;  // per-warp private histograms, then staged keys (16-byte aligned)
    uint32_t region_bytes;
    uint32_t* warp_off;     // [warps of the group]
    uint32_t* red;          // [warps of the group + 1]
    uint32_t* st;           // [4]
    uint32_t* s_staged;     // [1]
};

// ---------------------------------------------------------------------------
// The fixed-point window (sindi_accumulator FIXED32): the block-wide sums of
// B and of max |w_j| for one (query, window); fixed_point.cuh holds the rule
// that turns them into the unit 2^-e, and the integer bound of a bounded
// window.
// ---------------------------------------------------------------------------

// A warp's share of B and of max |w_j| (b, m: this thread's terms) into
// fred[warp] and fred[nw + warp]; every lane of the warp calls it.
__device__ __forceinline__ void fx_warp_partials(float b, float m, float* fred, int warp, int nw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b += __shfl_xor_sync(kFull, b, o);
        m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        fred[warp] = b;
        fred[nw + warp] = m;
    }
}

// e from the nw warps' partials (after a barrier). The warps are summed in a
// fixed order, so every thread gets the same e.
__device__ __forceinline__ int fx_exponent(const float* fred, int nw) {
    float B = 0.0f, M = 0.0f;
    for (int i = 0; i < nw; i++) {
        B += fred[i];
        M = fmaxf(M, fred[nw + i]);
    }
    return fx_exponent_from(B, M);
}

// This thread's part of B for term j of weight qv over window w.
template <int DT>
__device__ __forceinline__ void fx_term_bound(const DevIndex& ix, int32_t j, float qv, uint32_t len, float& b,
                                              float& m) {
    if (len == 0) return;
    const float wq = fabsf((DT == SINDI_F8E4M3) ? qv * ix.scale[j] : qv);
    b += wq * ix.vmax[j];
    m = fmaxf(m, wq);
}

// The term table of one query over one window, for terms c0 .. c0 + nc - 1
// of the query (nc <= the group's thread count): every term's posting range
// and weight, and the map from warp chunks to terms. Returns the number of
// chunks. Every thread of the group S calls it.
template <int DT, typename S>
__device__ uint32_t build_term_table(const ScanArgs& a, uint32_t w, int64_t qb, int c0, int nc, uint32_t* t_start,
                                     uint32_t* t_end, float* t_w, uint32_t* c_pre, uint16_t* c_term, uint32_t* red,
                                     uint32_t* negflag = nullptr, float* fred = nullptr, uint4* rec = nullptr) {
    const DevIndex& ix = a.ix;
    const int tid = S::tid();
    uint32_t nch = 0;
    float fb = 0.0f, fm = 0.0f;  // fixed-point window: this thread's part of B and of max |w_j|
    uint32_t r_start = 0, r_end = 0;  // the term's packed record (rec), once its first chunk is known
    float r_w = 0.0f;
    if (tid < nc) {
        const int32_t j = a.q_indices[qb + c0 + tid];
        const float qv = a.q_values[qb + c0 + tid];
        if (negflag && qv < 0.0f) *negflag = 1u;  // a negative query value (any thread may set it)
        uint32_t start = 0, len = 0;
        float wq = 0.0f;
        if (j >= 0 && j < ix.dim && isfinite(qv) && checked(list_in_bounds(j, w, ix.dim, ix.sigma), ix.err)) {
            const uint64_t sg = (uint64_t)j * ix.sigma + w;
            start = ix.seg[sg];
            len = ix.seg[sg + 1] - start;
            wq = (DT == SINDI_F8E4M3) ? qv * ix.scale[j] : qv;
        } else if (w == 0) {
            atomicOr(ix.err, (j < 0 || j >= ix.dim) ? kErrQueryDim : kErrQueryValue);
        }
        t_start[tid] = start;
        t_end[tid] = start + len;
        t_w[tid] = wq;
        r_start = start;
        r_end = start + len;
        r_w = wq;
        if (fred) fx_term_bound<DT>(ix, j, qv, len, fb, fm);
        // chunks of a long list tile its 8-aligned groups of postings
        nch = len >= kVecMin ? (((start + len + 7u) & ~7u) - (start & ~7u) + kChunkLen - 1) / kChunkLen
                             : (len ? 1u : 0u);
    }
    // (fred's partials are visible after the sum's barriers)
    if (fred) fx_warp_partials(fb, fm, fred, tid >> 5, S::kThreads / 32);
    uint32_t total;
    const uint32_t excl = group_exclusive_sum<uint32_t, S>(nch, &total, red);
    if (tid < nc) {
        c_pre[tid] = excl;
        if (rec) rec[tid] = make_uint4(r_start, r_end, excl, __float_as_uint(r_w));
        for (uint32_t c = excl; c < excl + nch && c < (uint32_t)kChunkTable; c++) c_term[c] = (uint16_t)tid;
    }
    S::sync();
    return total;
}

// Scatter-add of one term table into the window A (Alg. 2's product and
// accumulation loops): warp `warp` of NW takes chunks warp, warp + NW, ...;
// the next chunk's loads are issued before this chunk's adds.
template <int DT, int NW, bool FIXED = false>
__device__ __forceinline__ void accumulate_table(const DevIndex& ix, const uint32_t* t_start, const uint32_t* t_end,
                                                 const float* t_w, const uint32_t* c_pre, const uint16_t* c_term,
                                                 int nc, uint32_t total, int warp, int lane, float* A,
                                                 float wscale = 1.0f, const uint4* rec = nullptr) {
    // two chunks in registers, taking turns (no copy between them)
    uint32_t c = (uint32_t)warp;
    Chunk ka, kb;
    auto load = [&](uint32_t cc, Chunk& k) {
        if (rec) load_chunk_rec<DT>(ix, rec, c_pre, c_term, nc, cc, lane, k);
        else load_chunk<DT>(ix, t_start, t_end, t_w, c_pre, c_term, nc, cc, lane, k);
        if (FIXED) k.wq *= wscale;  // the fixed-point window's 2^e (exact)
    };
    auto add = [&](const Chunk& k) {
        if (FIXED) add_chunk_fixed(reinterpret_cast<int32_t*>(A), ix.lambda, ix.err, k);
        else add_chunk(A, ix.lambda, ix.err, k);
    };
    if (c < total) load(c, ka);
    while (c < total) {
        c += NW;
        if (c < total) load(c, kb);
        add(ka);
        if (c >= total) break;
        c += NW;
        if (c < total) load(c, ka);
        add(kb);
    }
}

// The fixed-point window's e for a query of more terms than one term table
// holds (its B must be known before the first table's adds): a pass over all
// of them. Every thread of the block calls it; fred: [2 * BLOCK / 32] floats,
// free on entry and on return.
template <int DT, int BLOCK>
__device__ int window_scale_exp(const ScanArgs& a, uint32_t w, int64_t qb, int nt, float* fred) {
    const DevIndex& ix = a.ix;
    float b = 0.0f, m = 0.0f;
    for (int t = threadIdx.x; t < nt; t += BLOCK) {
        const int32_t j = a.q_indices[qb + t];
        const float qv = a.q_values[qb + t];
        if (j >= 0 && j < ix.dim && isfinite(qv) && list_in_bounds(j, w, ix.dim, ix.sigma)) {
            const uint64_t sg = (uint64_t)j * ix.sigma + w;
            fx_term_bound<DT>(ix, j, qv, ix.seg[sg + 1] - ix.seg[sg], b, m);
        }
    }
    fx_warp_partials(b, m, fred, threadIdx.x >> 5, BLOCK / 32);
    __syncthreads();
    const int e = fx_exponent(fred, BLOCK / 32);
    __syncthreads();
    return e;
}

constexpr int kNoFx = 1 << 30;  // select_window: the window holds FP32 scores

// The fixed-point window's sums to FP32 scores in place: the rounded
// conversion times 2^-e (exact scaling). Every thread of the group S calls it.
template <typename S>
__device__ __forceinline__ void fx_window_to_float(float* A, uint32_t lambda, int e) {
    const float inv = pow2f(-e);
    int4* I4 = reinterpret_cast<int4*>(A);
    float4* F4 = reinterpret_cast<float4*>(A);
    for (uint32_t m = (uint32_t)S::tid(); m < window_stride(lambda) / 4; m += S::kThreads) {
        const int4 t = I4[m];
        F4[m] = make_float4((float)t.x * inv, (float)t.y * inv, (float)t.z * inv, (float)t.w * inv);
    }
}

// The least float whose order key is at least k: a slot's key is >= k
// exactly when its score is >= this value. -inf when every float's key is
// (k at or below the key of -inf); a NaN, which compares false with
// everything, when no finite float's key reaches k.
__device__ __forceinline__ float key_floor_float(uint32_t k) {
    if (k <= 0x007FFFFFu) return -INFINITY;
    if (k > 0xFF800000u) return __int_as_float(0x7FC00000);
    return order_bits_float(k);
}

// The cut of one accumulated window w of query row y: emits into the query's
// candidate list every slot that can still be among its best g, and adds what
// it emitted to the query's histogram H (ids >= N are not candidates).
// `bounded`: g candidates of the query already exist at or above bin pbin.
// Every thread of the group S (NW warps) calls it; the workspace must be free.
template <typename S, int NW, bool FX = false>
__device__ void select_window(const ScanArgs& a, float* A, uint32_t w, uint32_t y, bool bounded, uint32_t pbin,
                              const CutScratch& cs, bool skip_zero = false, int fx_e = kNoFx) {
    constexpr int NT = S::kThreads;
    const DevIndex& ix = a.ix;
    const int tid = S::tid();
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t* hist = cs.hist;
    uint32_t* hist2 = cs.hist2;
    uint32_t* warp_off = cs.warp_off;
    uint32_t* red = cs.red;
    uint32_t* st = cs.st;
    uint64_t* stage = reinterpret_cast<uint64_t*>(cs.region);
    const uint32_t stage_cap = cs.region_bytes / 8;
    uint32_t* H = a.ws.hist + (size_t)y * kHistBins;
    const uint32_t lambda = ix.lambda;
    const int64_t gbase = (int64_t)w * lambda;
    const int64_t rest = ix.n_docs - gbase;
    const int n_eff = (int)(rest < (int64_t)lambda ? rest : (int64_t)lambda);
    const uint32_t g_w = a.g < (uint32_t)n_eff ? a.g : (uint32_t)n_eff;
    // fx_e != kNoFx (only with FX, only for a bounded window): A holds the fixed-point sums in units of 2^-fx_e,
    // until a bounded window with too many slots at the bound converts them to FP32 for the full cut (fx
    // then turns false, and key_of reads the FP32 scores)
    bool fx = FX && fx_e != kNoFx;
    const float fx_inv = fx ? pow2f(-fx_e) : 1.0f;
    const int32_t* Ai = reinterpret_cast<const int32_t*>(A);
    auto key_of = [&](int i) -> uint64_t {
        return result_key(fx ? (float)Ai[i] * fx_inv : A[i], (uint32_t)(gbase + i));
    };
    uint64_t* cand = a.ws.cand + (size_t)y * a.ws.cand_cap;
    if (bounded) {
        // g candidates at or above bin pbin already exist, so only slots in
        // bins >= pbin can be in the answer. With skip_zero (every score of
        // the query is >= 0 and the earlier windows hold at least g slots, all
        // with scores >= 0 and lower ids), a slot whose score is exactly 0 can
        // never be either: when the bound reaches down to 0, only positive
        // slots count. When the slots that can count fit the window's budget,
        // emit all of them: no window histogram, no cut. One pass: every warp
        // stages its slots in its own share of the staging area (in order, no
        // atomics); then one reservation for the group.
        const unsigned lt = (1u << lane) - 1u;
        const uint32_t share = stage_cap / NW;
        uint64_t* mine_st = stage + (size_t)warp * share;
        // the window 4 slots per lane (one 16-byte load, one compare each against
        // the least score that can count); the per-slot work runs only for the
        // rare 128-slot spans that hold a candidate
        float thr = key_floor_float(pbin << (32 - kHistBits));
        if (skip_zero && thr <= 0.0f) thr = __int_as_float(1);  // the least positive float (NaN stays NaN)
        const int n4 = (n_eff + 3) >> 2;
        const float4* A4 = reinterpret_cast<const float4*>(A);
        const int4* I4 = reinterpret_cast<const int4*>(A);
        const int32_t ithr = fx ? fx_threshold(thr, fx_e) : 0;
        auto scan_bounded = [&](auto&& emit) -> uint32_t {
            uint32_t cnt = 0;
            for (int b4 = warp * 32; b4 < n4; b4 += NT) {
                const int i4 = b4 + lane;
                uint32_t m = 0;
                if (i4 < n4) {
                    if (fx) {
                        const int4 x = I4[i4];
                        m = (x.x >= ithr ? 1u : 0u) | (x.y >= ithr ? 2u : 0u) | (x.z >= ithr ? 4u : 0u) |
                            (x.w >= ithr ? 8u : 0u);
                    } else {
                        const float4 x = A4[i4];
                        m = (x.x >= thr ? 1u : 0u) | (x.y >= thr ? 2u : 0u) | (x.z >= thr ? 4u : 0u) |
                            (x.w >= thr ? 8u : 0u);
                    }
                    const int rem = n_eff - 4 * i4;
                    if (rem < 4) m &= (1u << rem) - 1u;
                }
                if (!__any_sync(kFull, m != 0u)) continue;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const bool ok = (m >> c) & 1u;
                    const unsigned bal = __ballot_sync(kFull, ok);
                    if (ok) emit(4 * i4 + c, cnt + (uint32_t)__popc(bal & lt));
                    cnt += (uint32_t)__popc(bal);
                }
            }
            return cnt;
        };
        const uint32_t cnt = scan_bounded([&](int i, uint32_t at) {
            if (at < share) mine_st[at] = key_of(i);
        });
        if (lane == 0) warp_off[warp] = cnt;
        S::sync();
        if (tid == 0) {
            uint32_t acc = 0, over = 0;
            for (int k = 0; k < NW; k++) {
                const uint32_t c = warp_off[k];
                over |= c > share ? 1u : 0u;
                warp_off[k] = acc;
                acc += c;
            }
            cs.s_staged[0] = acc;
            st[1] = over;
            st[0] = acc && acc <= a.win_cap ? atomicAdd(a.ws.cand_count + y, acc) : 0u;
        }
        S::sync();
        const uint32_t n_hi = cs.s_staged[0];
        if (n_hi <= a.win_cap) {
            const uint32_t at0 = st[0] + warp_off[warp];
            if (st[1] == 0) {
                // the staged keys out, each counted in the query's histogram
                for (uint32_t t = (uint32_t)lane; t < cnt; t += 32) {
                    const uint64_t key = mine_st[t];
                    if (at0 + t < a.ws.cand_cap) cand[at0 + t] = key;
                    else atomicOr(ix.err, kErrCandOverflow);
                    atomicAdd(H + (uint32_t)(key >> kKeyBinShift), 1u);
                }
            } else {
                // a warp had more slots than its share: read the window again
                (void)scan_bounded([&](int i, uint32_t at) {
                    const uint64_t key = key_of(i);
                    if (at0 + at < a.ws.cand_cap) cand[at0 + at] = key;
                    else atomicOr(ix.err, kErrCandOverflow);
                    atomicAdd(H + (uint32_t)(key >> kKeyBinShift), 1u);
                });
            }
            S::sync();  // warp_off, st and the staging area are reused by the caller's next cut
            return;
        }
        // too many: the cut below decides (group-uniform), on FP32 scores
        if (fx) {
            fx_window_to_float<S>(A, lambda, fx_e);
            S::sync();
            fx = false;
        }
    }
    // level 1: 12-bit bins of the score key. Each warp counts its slots in a
    // private histogram of the 256 bins below the window's top bin (no
    // contention between warps); the window histogram is their sum. When the
    // cut falls below that range, a full 4096-bin histogram is used instead.
    // the slot passes below read 4 slots per thread (thread t: slots 4 (t + k NT) .. + 3),
    // and a warp's slots are the same in every pass
    uint32_t* priv = reinterpret_cast<uint32_t*>(cs.region) + warp * kRelBins;
    const int n4w = (n_eff + 3) >> 2;
    const float4* A4w = reinterpret_cast<const float4*>(A);
    auto slots4 = [&](int i4, float v[4]) -> uint32_t {  // the group's scores; bit c: slot 4 i4 + c < n_eff
        const float4 x = A4w[i4];
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
        const int rem = n_eff - 4 * i4;
        return rem >= 4 ? 15u : (1u << rem) - 1u;
    };
    uint32_t top_key = 0;
    for (int i4 = tid; i4 < n4w; i4 += NT) {
        float v[4];
        const uint32_t ok = slots4(i4, v);
#pragma unroll
        for (int c = 0; c < 4; c++)
            if (ok & (1u << c)) top_key = max(top_key, float_order_bits(v[c]));
    }
    top_key = __reduce_max_sync(kFull, top_key);
    if (lane == 0) red[warp] = top_key;
    for (int b = tid; b < kSubBins; b += NT) hist2[b] = 0;
    S::sync();
    if (tid == 0) {
        uint32_t m = 0;
        for (int i = 0; i < NW; i++) m = max(m, red[i]);
        st[0] = m;
    }
    for (int b = lane; b < kRelBins; b += 32) priv[b] = 0;
    S::sync();
    const uint32_t top_bin = st[0] >> (32 - kHistBits);
    for (int i4 = tid; i4 < n4w; i4 += NT) {
        float v[4];
        const uint32_t ok = slots4(i4, v);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (ok & (1u << c)) {
                const uint32_t rel = top_bin - (float_order_bits(v[c]) >> (32 - kHistBits));
                atomicAdd(&priv[rel < (uint32_t)kRelBins ? rel : kRelBins - 1], 1u);
            }
        }
    }
    S::sync();
    for (int b = tid; b < kRelBins; b += NT) {
        uint32_t c = 0;
        for (int k = 0; k < NW; k++) c += reinterpret_cast<uint32_t*>(cs.region)[k * kRelBins + b];
        hist[b] = c;  // hist[rel] = slots in bin top_bin - rel (rel 255: that bin and all below)
    }
    S::sync();
    group_find_bin<kRelBins, S>([&](int b) { return hist[kRelBins - 1 - b]; }, g_w, red, st);
    const uint32_t rel_cut = kRelBins - 1 - st[0];
    uint32_t bw = top_bin - rel_cut;
    uint32_t above_bw = st[1];
    uint32_t c_bw = st[1] + st[2];  // slots in bins >= bw
    S::sync();
    const bool relative = rel_cut < (uint32_t)kRelBins - 1;
    if (!relative) {
        for (int b = tid; b < kHistBins; b += NT) hist[b] = 0;
        S::sync();
        for (int base = 0; base < n_eff; base += NT) {
            const int i = base + tid;
            const int bin = i < n_eff ? (int)(float_order_bits(A[i]) >> (32 - kHistBits)) : -1;
            const unsigned peers = __match_any_sync(kFull, bin);
            if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        S::sync();
        group_find_bin<kHistBins, S>([&](int b) { return hist[b]; }, g_w, red, st);
        bw = st[0];
        above_bw = st[1];
        c_bw = st[1] + st[2];
        S::sync();
    }
    // slots of the window in 12-bit bin b (b within the histogram kept above)
    auto bin_count = [&](uint32_t b) -> uint32_t {
        if (!relative) return hist[b];
        const uint32_t rel = top_bin - b;
        return rel < (uint32_t)kRelBins - 1 ? hist[rel] : 0u;
    };
    wait_previous_kernels();  // the workspace is free from here on
    uint32_t lo = bw;
    // g slots already emitted at or above a bin prove the answer lies there
    if (bounded && pbin > lo) lo = pbin;
    const bool staged = relative && c_bw <= stage_cap;  // slots >= bin lo fit in the staging area
    uint32_t n_src = (uint32_t)n_eff;
    if (staged) {
        // per-warp counts of slots at or above bin lo (from the private
        // histograms) give every warp its staging range: no atomics below
        uint32_t mine_w = 0;
        for (int b = lane; b < kRelBins - 1; b += 32)
            if (top_bin - (uint32_t)b >= lo) mine_w += priv[b];
        mine_w = __reduce_add_sync(kFull, mine_w);
        if (lane == 0) warp_off[warp] = mine_w;
        S::sync();
        if (tid == 0) {
            uint32_t acc = 0;
            for (int k = 0; k < NW; k++) {
                const uint32_t c = warp_off[k];
                warp_off[k] = acc;
                acc += c;
            }
            cs.s_staged[0] = acc;
        }
        S::sync();  // the private histograms are dead from here on
        uint32_t at = warp_off[warp];
        const unsigned lt = (1u << lane) - 1u;
        const float thr_lo = key_floor_float(lo << (32 - kHistBits));
        for (int b4 = warp * 32; b4 < n4w; b4 += NT) {
            const int i4 = b4 + lane;
            uint32_t m = 0;
            if (i4 < n4w) {
                float v[4];
                const uint32_t ok = slots4(i4, v);
#pragma unroll
                for (int c = 0; c < 4; c++) m |= (v[c] >= thr_lo ? 1u : 0u) << c;
                m &= ok;
            }
            if (!__any_sync(kFull, m != 0u)) continue;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const bool ok = (m >> c) & 1u;
                const unsigned bal = __ballot_sync(kFull, ok);
                if (ok) stage[at + __popc(bal & lt)] = key_of(4 * i4 + c);
                at += __popc(bal);
            }
        }
        S::sync();
        n_src = cs.s_staged[0];
    }
    // candidates: the staged keys, or the whole window
    auto src_key = [&](int i) -> uint64_t { return staged ? stage[i] : key_of(i); };
    uint64_t thr = (uint64_t)lo << kKeyBinShift;
    bool exact = false;
    if (lo == bw) {
        // level 2: the next 8 bits, inside bin bw only
        for (int i = tid; i < (int)n_src; i += NT) {
            const uint64_t k = src_key(i);
            if ((uint32_t)(k >> kKeyBinShift) == bw)
                atomicAdd(&hist2[(uint32_t)(k >> (kKeyBinShift - kSubBits)) & (kSubBins - 1)], 1u);
        }
        S::sync();
        group_find_bin<kSubBins, S>([&](int b) { return hist2[b]; }, g_w - above_bw, red, st);
        const uint32_t bw2 = st[0];
        const uint32_t c_cut = above_bw + st[1] + st[2];   // slots at or above the 20-bit cut
        S::sync();
        thr = ((uint64_t)((bw << kSubBits) | bw2)) << (kKeyBinShift - kSubBits);
        exact = c_cut > a.win_cap;
    }
    if (exact) {
        // ties crowd the cut: exact best g_w of the window
        thr = group_select_threshold<S>(src_key, (int)n_src, (int)g_w, hist2, st);
    }
    // emit keys >= thr: count, reserve the group's range with one atomic, write
    uint32_t mine = 0;
    for (int i = tid; i < (int)n_src; i += NT)
        if (src_key(i) >= thr) mine++;
    uint32_t total;
    uint32_t pos = group_exclusive_sum<uint32_t, S>(mine, &total, red);
    if (tid == 0) st[0] = total ? atomicAdd(a.ws.cand_count + y, total) : 0u;
    S::sync();
    pos += st[0];
    for (int i = tid; i < (int)n_src && mine; i += NT) {
        const uint64_t key = src_key(i);
        if (key >= thr) {
            if (pos < a.ws.cand_cap) cand[pos] = key;
            else atomicOr(ix.err, kErrCandOverflow);
            pos++;
            mine--;
        }
    }
    // what was emitted, per 12-bit bin, into the query's histogram: every
    // bin above the cut bin in full, the rest of the emitted slots in it
    const uint32_t tb = (uint32_t)(thr >> kKeyBinShift);
    uint32_t above_mine = 0;
    for (int b = tid; b < kHistBins; b += NT) {
        const uint32_t c = (uint32_t)b > tb ? bin_count((uint32_t)b) : 0u;
        if (c) {
            above_mine += c;
            atomicAdd(H + b, c);
        }
    }
    uint32_t above;
    (void)group_exclusive_sum<uint32_t, S>(above_mine, &above, red);
    if (tid == 0 && total > above) atomicAdd(H + tb, total - above);
    S::sync();  // hist, region and st are reused by the caller's next cut
}

// One block per (window, query): the term tables are staged in shared memory,
// the block's warps scatter-add every term's postings of the window into A,
// then the block cuts the window.
template <int DT, bool QUERY_MAJOR, int BLOCK, bool FX>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) scan_window_kernel(ScanArgs a) {
    constexpr int kScanThreads = BLOCK;
    constexpr int kScanWarps = BLOCK / 32;
    constexpr int kTermChunk = BLOCK;   // query terms staged per pass (one per thread)
    using S = SyncBlock<BLOCK>;
    // Shared memory: the window's scores, two histograms, and one region that
    // holds the term tables while postings are added and the staged
    // candidates of the window afterwards.
    constexpr int kTableBytes = 16 * kTermChunk + (((4 * kTermChunk + 1) * 4 + kChunkTable * 2 + 15) & ~15);
    constexpr int kPrivBytes = kScanWarps * kRelBins * 4;
    constexpr int kRegionBytes = kTableBytes > kPrivBytes ? kTableBytes : kPrivBytes;
    extern __shared__ float A[];                    // [lambda]
    __shared__ uint32_t hist[kHistBins];
    __shared__ uint32_t hist2[kSubBins];
    __shared__ __align__(16) unsigned char region[kRegionBytes];
    __shared__ uint32_t warp_off[kScanWarps];
    __shared__ uint32_t red[kScanWarps + 1];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_staged;
    __shared__ uint32_t s_qneg;  // the query has a negative value
    __shared__ float fred[2 * kScanWarps];  // fixed-point window: the warps' parts of B and of max |w_j|
    uint4* t_rec = reinterpret_cast<uint4*>(region);  // the terms' packed records, read once per chunk
    uint32_t* t_start = reinterpret_cast<uint32_t*>(region + 16 * kTermChunk);
    uint32_t* t_end = t_start + kTermChunk;
    uint32_t* c_pre = t_end + kTermChunk;
    float* t_w = reinterpret_cast<float*>(c_pre + kTermChunk + 1);
    uint16_t* c_term = reinterpret_cast<uint16_t*>(t_w + kTermChunk);

    const DevIndex& ix = a.ix;
    const uint32_t w = a.w0 + (QUERY_MAJOR ? blockIdx.y : blockIdx.x);
    const uint32_t y = QUERY_MAJOR ? blockIdx.x : blockIdx.y;
    const int64_t r = a.q_first + y;
    const uint32_t lambda = ix.lambda;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    uint32_t* H = a.ws.hist + (size_t)y * kHistBins;
    if (a.use_partial == 1) {
        // the query's histogram of what its earlier windows emitted, copied
        // while the window accumulates (a snapshot: H only grows during the
        // launch, so any snapshot bounds the answer)
        wait_previous_kernels();  // the workspace is free from here on
        for (int c = threadIdx.x; c < kHistBins / 4; c += kScanThreads) cp_async16(hist + 4 * c, H + 4 * c);
        cp_async_commit();
    }
    const int64_t qb = a.q_indptr[r];
    const int nt = (int)(a.q_indptr[r + 1] - qb);
    if (threadIdx.x == 0) s_qneg = 0;  // read after the term tables' barriers

    {
        float4* A4 = reinterpret_cast<float4*>(A);
        for (uint32_t m = threadIdx.x; m < window_stride(lambda) / 4; m += kScanThreads)
            A4[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    // fixed-point window: the unit 2^-e of this (query, window). B comes with the
    // term table when one table holds the query's terms, else from a pass of its own.
    int fx_e = 0;
    const bool fx_pre = FX && nt > kTermChunk;
    if (fx_pre) fx_e = window_scale_exp<DT, BLOCK>(a, w, qb, nt, fred);
    for (int c0 = 0; c0 < nt; c0 += kTermChunk) {
        const int nc = min(kTermChunk, nt - c0);
        __syncthreads();  // previous chunk fully consumed
        const uint32_t total = build_term_table<DT, S>(a, w, qb, c0, nc, t_start, t_end, t_w, c_pre, c_term, red,
                                                       &s_qneg, FX && !fx_pre ? fred : nullptr, t_rec);
        if (FX) {
            if (!fx_pre) fx_e = fx_exponent(fred, kScanWarps);
            accumulate_table<DT, kScanWarps, true>(ix, t_start, t_end, t_w, c_pre, c_term, nc, total, warp, lane, A,
                                                   pow2f(fx_e), t_rec);
        } else {
            accumulate_table<DT, kScanWarps>(ix, t_start, t_end, t_w, c_pre, c_term, nc, total, warp, lane, A,
                                             1.0f, t_rec);
        }
    }
    __syncthreads();

    // the next kernel may start its blocks now (they wait for this one where they
    // must); later than the block's start, so they do not sit idle through the
    // accumulation
    allow_next_kernel();

    uint32_t pbin = 0;  // bin of the g-th emitted candidate, when g have been emitted
    bool bounded = false;
    if (a.use_partial == 1) {
        cp_async_wait_all();
        __syncthreads();
        block_find_bin<kHistBins, kScanThreads>([&](int b) { return hist[b]; }, a.g, red, st);
        bounded = st[3] >= a.g;
        pbin = st[0];
        __syncthreads();
    } else if (a.use_partial == 2) {
        wait_previous_kernels();  // the first windows' candidates are all in H
        block_find_bin<kHistBins, kScanThreads>([&](int b) { return __ldcg(H + b); }, a.g, red, st);
        bounded = st[3] >= a.g;
        pbin = st[0];
        __syncthreads();
    }
    const CutScratch cs{hist, hist2, region, (uint32_t)kRegionBytes, warp_off, red, st, &s_staged};
    // zero-score slots cannot count once the earlier windows hold g slots, when no score can be negative
    const bool skip_zero = s_qneg == 0 && ix.nonneg && (uint64_t)w * lambda >= a.g;
    // a fixed-point window without a bound goes to FP32 for the full cut; a bounded one is read as integers
    if (FX && !bounded) {
        fx_window_to_float<S>(A, lambda, fx_e);
        S::sync();
    }
    select_window<S, kScanWarps, FX>(a, A, w, y, bounded, pbin, cs, skip_zero, FX && bounded ? fx_e : kNoFx);
}

// ---------------------------------------------------------------------------
// Pipelined window scan: one resident block per SM walks a list of (window,
// query) items with two window arrays in shared memory. Warps 0..23 scatter-
// add item i + 1 into one array while warps 24..31 cut item i in the other
// and build the term tables ahead, so the shared-memory scatter-add (the
// scan's bound) does not stop for the cut. Hardware named barriers hand the
// arrays and tables between the two groups:
//   ready[t]: table t holds the next stage's terms (cut group -> add group)
//   free[t]:  the add group is done with table t (add -> cut)
//   done[b]:  array b holds an item's complete scores (add -> cut)
//   empty[b]: array b is cut and zeroed again (cut -> add)
// An item with more terms than one table holds takes several stages.
// ---------------------------------------------------------------------------
constexpr int kPipeAddWarps = 24;
constexpr int kPipeCutWarps = 8;
constexpr int kPipeThreads = (kPipeAddWarps + kPipeCutWarps) * 32;
constexpr int kPipeTerms = kPipeCutWarps * 32;  // query terms per table (one per cutting thread)
constexpr int kPipeTableBytes = ((4 * kPipeTerms + 1) * 4 + kChunkTable * 2 + 15) & ~15;
constexpr int kPipeRegionBytes = 16384;         // cut scratch: 8 KiB private histograms / 2,048 staged keys
constexpr uint32_t kPipeMaxWindow = 16384;      // two window arrays of 64 KiB each
constexpr int kBarReady = 1, kBarFree = 3, kBarDone = 5, kBarEmpty = 7, kBarCut = 9;

__device__ __forceinline__ void named_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kPipeThreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "n"(kPipeThreads) : "memory");
}

static size_t pipe_smem_bytes(uint32_t lambda) {
    return (size_t)8 * window_stride(lambda) + 2 * (size_t)kPipeTableBytes + kPipeRegionBytes;
}

template <int DT>
__global__ void __launch_bounds__(kPipeThreads, 1) scan_pipe_kernel(ScanArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ uint32_t hist[kHistBins];
    __shared__ uint32_t hist2[kSubBins];
    __shared__ uint32_t warp_off[kPipeCutWarps];
    __shared__ uint32_t red[kPipeCutWarps + 1];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_staged;
    __shared__ uint32_t t_total[2];
    __shared__ int t_nc[2];
    using S = SyncGroup<kBarCut, kPipeCutWarps * 32, kPipeAddWarps * 32>;
    const DevIndex& ix = a.ix;
    const uint32_t lambda = ix.lambda;
    float* buf0 = reinterpret_cast<float*>(dsm);
    const uint32_t lam4 = window_stride(lambda);  // windows start 16-byte aligned
    unsigned char* tab = dsm + (size_t)8 * lam4;
    unsigned char* region = tab + 2 * kPipeTableBytes;
    auto t_start = [&](int t) { return reinterpret_cast<uint32_t*>(tab + t * kPipeTableBytes); };
    auto t_end = [&](int t) { return t_start(t) + kPipeTerms; };
    auto c_pre = [&](int t) { return t_start(t) + 2 * kPipeTerms; };
    auto t_w = [&](int t) { return reinterpret_cast<float*>(t_start(t) + 3 * kPipeTerms + 1); };
    auto c_term = [&](int t) { return reinterpret_cast<uint16_t*>(t_start(t) + 4 * kPipeTerms + 1); };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // items: k = blockIdx.x + it * gridDim.x; window w0 + k / nq, query row k % nq
    const uint32_t n_all = a.nq * a.nwin;
    const uint32_t n_my = blockIdx.x < n_all ? (n_all - blockIdx.x + gridDim.x - 1) / gridDim.x : 0u;
    auto item_y = [&](uint32_t it) { return (blockIdx.x + it * gridDim.x) % a.nq; };
    auto item_w = [&](uint32_t it) { return a.w0 + (blockIdx.x + it * gridDim.x) / a.nq; };
    auto passes = [&](uint32_t y) {
        const int64_t r = a.q_first + y;
        const int nt = (int)(a.q_indptr[r + 1] - a.q_indptr[r]);
        return nt > 0 ? (nt + kPipeTerms - 1) / kPipeTerms : 1;
    };

    for (uint32_t m = threadIdx.x; m < 2 * lam4; m += kPipeThreads) buf0[m] = 0.0f;
    __syncthreads();

    if (warp < kPipeAddWarps) {
        // ---- add group: scatter-add stage after stage
        int s = 0;
        for (uint32_t it = 0; it < n_my; it++) {
            const int np = passes(item_y(it));
            const int b = it & 1;
            for (int p = 0; p < np; p++, s++) {
                const int t = s & 1;
                named_sync(kBarReady + t);
                if (p == 0 && it >= 2) named_sync(kBarEmpty + b);
                accumulate_table<DT, kPipeAddWarps>(ix, t_start(t), t_end(t), t_w(t), c_pre(t), c_term(t), t_nc[t],
                                                    t_total[t], warp, lane, buf0 + (size_t)b * lam4);
                named_arrive(kBarFree + t);
                if (p == np - 1) named_arrive(kBarDone + b);
            }
        }
        allow_next_kernel();
        return;
    }

    // ---- cut group: tables ahead, then the cut of every accumulated item
    const CutScratch cs{hist, hist2, region, (uint32_t)kPipeRegionBytes, warp_off, red, st, &s_staged};
    uint32_t bi = 0;  // next stage to build: item bi, pass bp
    int bp = 0;
    auto build_next = [&](int t) {
        const uint32_t y = item_y(bi), w = item_w(bi);
        const int64_t r = a.q_first + y;
        const int64_t qb = a.q_indptr[r];
        const int nt = (int)(a.q_indptr[r + 1] - qb);
        const int c0 = bp * kPipeTerms;
        const int nc = nt - c0 < kPipeTerms ? (nt - c0 > 0 ? nt - c0 : 0) : kPipeTerms;
        const uint32_t total = build_term_table<DT, S>(a, w, qb, c0, nc, t_start(t), t_end(t), t_w(t), c_pre(t),
                                                       c_term(t), red);
        if (S::tid() == 0) {
            t_total[t] = total;
            t_nc[t] = nc;
        }
        const int np = nt > 0 ? (nt + kPipeTerms - 1) / kPipeTerms : 1;
        if (++bp == np) {
            bp = 0;
            bi++;
        }
    };
    if (bi < n_my) {
        build_next(0);
        named_arrive(kBarReady + 0);
    }
    if (bi < n_my) {
        build_next(1);
        named_arrive(kBarReady + 1);
    }
    int s = 0;
    for (uint32_t it = 0; it < n_my; it++) {
        const uint32_t y = item_y(it), w = item_w(it);
        const int np = passes(y);
        const int b = it & 1;
        for (int p = 0; p < np; p++, s++) {
            const int t = s & 1;
            named_sync(kBarFree + t);
            if (bi < n_my) {
                build_next(t);
                named_arrive(kBarReady + t);
            }
        }
        named_sync(kBarDone + b);
        // the workspace (and, for a query's later windows, H) is final from here on;
        // tables read only the index and the queries, so they were built before
        if (it == 0) wait_previous_kernels();
        if (it + 1 == n_my) allow_next_kernel();
        // the query's running bound: g candidates emitted at or above a bin
        const uint32_t* H = a.ws.hist + (size_t)y * kHistBins;
        group_find_bin<kHistBins, S>([&](int bb) { return __ldcg(H + bb); }, a.g, red, st);
        const bool bounded = st[3] >= a.g;
        const uint32_t pbin = st[0];
        S::sync();
        float* A = buf0 + (size_t)b * lam4;
        select_window<S, kPipeCutWarps>(a, A, w, y, bounded, pbin, cs);
        for (uint32_t m = (uint32_t)S::tid(); m < lam4 / 4; m += S::kThreads)
            reinterpret_cast<float4*>(A)[m] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (it + 2 < n_my) named_arrive(kBarEmpty + b);
    }
}

// ---------------------------------------------------------------------------
// Query-group window scan (batched schedule). One block owns window w for a
// group of up to Q queries and holds their Q score windows in shared memory.
// It walks the union of the group's query terms: each posting of a segment
// I_{j,w} is loaded once and added into the window of every query of the
// group that holds term j (Alg. 2's product and accumulation loops for Q
// queries at once). Each query's window is then cut as in scan_window_kernel.
//   union: the group's query entries, up to kGroupEntries per pass, go into a
//       shared-memory hash keyed by dim; an occupied slot is one union term
//       with the bit mask of the queries holding it and their weights. A dim
//       that reaches two passes is simply two terms (every (query, term)
//       entry is still added exactly once).
//   adds: a warp chunk is 256 postings of one segment (the geometry the
//       build's bank-aware order is laid out for); the ids are decoded once
//       and, for every holder, the 8 postings of a lane are added with FP32
//       shared-memory atomics under one 8-bit lane mask.
// Groups are consecutive query rows of the launch.
// ---------------------------------------------------------------------------
constexpr int kMaxGroup = (int)kMaxQueryGroup;
constexpr int kGroupEntries = 512;     // query entries hashed per pass (union terms per pass <= this)
constexpr int kGroupHash = 1024;       // hash slots (load <= 1/2)
constexpr int kGroupHashBits = 10;

// Shared-memory region of the group scan: the hash and term tables while
// postings are added (hash keys and values, term starts, ends, chunk prefix
// and holder masks, weights [kGroupEntries][kMaxGroup], the chunk -> term
// table), the cut's scratch afterwards (private histograms, staged keys).
constexpr size_t kGroupTableBytes = ((size_t)kGroupHash * 8 + (size_t)(4 * kGroupEntries + 1) * 4 +
                                     (size_t)kGroupEntries * kMaxGroup * 4 + (size_t)kChunkTable * 2 + 15) &
                                    ~(size_t)15;
__host__ __device__ constexpr size_t group_region_bytes(int block) {
    return kGroupTableBytes > (size_t)(block / 32) * kRelBins * 4 ? kGroupTableBytes
                                                                   : (size_t)(block / 32) * kRelBins * 4;
}
// Dynamic shared memory a group-scan block may take (the static arrays take the rest of the 227 KiB).
constexpr size_t kGroupDynSmemMax = (size_t)(227 - 20) * 1024;

static size_t group_smem_bytes(uint32_t lambda, uint32_t Q, int block) {
    return (size_t)Q * window_stride(lambda) * 4 + group_region_bytes(block);
}

struct GroupScanArgs {
    ScanArgs s;            // index, queries (rows q_first + y), g, win_cap, workspace, w0
    uint32_t Q;            // queries per group (1..kMaxGroup)
    uint32_t nq;           // query rows of the launch
};

// Adds a chunk of union term t into the window of every query of the group
// that holds the term (shared-memory atomics: chunks of different terms run
// at once and may meet on a slot).
__device__ __forceinline__ void add_chunk_holders(float* A, uint32_t stride, uint32_t lambda, uint32_t* err,
                                                  uint32_t mask, const float* w, const Chunk& k) {
    while (mask) {
        const int i = __ffs(mask) - 1;
        mask &= mask - 1u;
        const float wq = w[i];
        float* Ai = A + (size_t)i * stride;
#pragma unroll
        for (int u = 0; u < kChunkU; u++)
            if ((k.lm & (1u << u)) && checked(slot_in_bounds(chunk_slot(k, u), lambda), err))
                atomicAdd(Ai + chunk_slot(k, u), wq * k.v[u]);
    }
}

__device__ __forceinline__ uint32_t group_hash_slot(int32_t j) {
    return ((uint32_t)j * 2654435761u) >> (32 - kGroupHashBits);
}

template <int DT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) group_scan_kernel(GroupScanArgs a) {
    constexpr int NW = BLOCK / 32;
    using S = SyncBlock<BLOCK>;
    extern __shared__ __align__(16) unsigned char gsm[];
    __shared__ uint32_t hist[kHistBins];
    __shared__ uint32_t hist2[kSubBins];
    __shared__ uint32_t warp_off[NW];
    __shared__ uint32_t red[NW + 1];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_staged;
    __shared__ uint32_t mrow[kMaxGroup];        // query row (within the launch) of each member
    __shared__ uint32_t mpre[kMaxGroup + 1];    // prefix of the members' term counts
    __shared__ int64_t mqb[kMaxGroup];          // first entry of each member's query row
    __shared__ uint32_t s_negmask;              // bit i: member i has a negative query value
    const ScanArgs& sa = a.s;
    const DevIndex& ix = sa.ix;
    const uint32_t lambda = ix.lambda;
    const uint32_t Q = a.Q;
    const uint32_t grp = blockIdx.x;
    const uint32_t w = sa.w0 + blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t first = grp * Q;
    const uint32_t qn = min(Q, a.nq - first);  // members of this group

    float* A = reinterpret_cast<float*>(gsm);
    const uint32_t lam4 = window_stride(lambda);  // members' windows start 16-byte aligned
    unsigned char* region = gsm + (size_t)Q * lam4 * 4;
    int32_t* hkey = reinterpret_cast<int32_t*>(region);
    uint32_t* hval = reinterpret_cast<uint32_t*>(hkey + kGroupHash);  // holder mask | union index << 16
    uint32_t* t_start = hval + kGroupHash;
    uint32_t* t_end = t_start + kGroupEntries;
    uint32_t* c_pre = t_end + kGroupEntries;
    uint32_t* t_mask = c_pre + kGroupEntries + 1;
    float* t_w = reinterpret_cast<float*>(t_mask + kGroupEntries);
    uint16_t* c_term = reinterpret_cast<uint16_t*>(t_w + kGroupEntries * kMaxGroup);

    if (tid < (int)qn) {
        const uint32_t y = first + (uint32_t)tid;
        const int64_t r = sa.q_first + y;
        mrow[tid] = y;
        mqb[tid] = sa.q_indptr[r];
        mpre[tid + 1] = (uint32_t)(sa.q_indptr[r + 1] - sa.q_indptr[r]);
    }
    // zero the members' windows, 16 bytes per store
    {
        float4* A4 = reinterpret_cast<float4*>(A);
        const uint32_t n4 = (qn * lam4) >> 2;
        for (uint32_t m = tid; m < n4; m += BLOCK) A4[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (tid == 0) {
        mpre[0] = 0;
        for (uint32_t i = 0; i < qn; i++) mpre[i + 1] += mpre[i];
        s_negmask = 0;
    }
    __syncthreads();
    const uint32_t n_ent = mpre[qn];

    for (uint32_t e0 = 0; e0 < n_ent; e0 += kGroupEntries) {
        // ---- union of the entries e0 .. e0 + kGroupEntries - 1 in the hash
        for (int s = tid; s < kGroupHash; s += BLOCK) {
            hkey[s] = -1;
            hval[s] = 0;
        }
        __syncthreads();
        int my_slot = -1, my_i = 0;
        float my_w = 0.0f;
        if (tid < kGroupEntries && e0 + tid < n_ent) {
            const uint32_t e = e0 + (uint32_t)tid;
            int i = 0;
            while (i + 1 < (int)qn && mpre[i + 1] <= e) i++;
            const int64_t at = mqb[i] + (e - mpre[i]);
            const int32_t j = sa.q_indices[at];
            const float qv = sa.q_values[at];
            if (qv < 0.0f) atomicOr(&s_negmask, 1u << i);
            // entries the scan skips: dims out of range and non-finite values (the merge
            // reports them), zero weights (Definition 1: not entries)
            if (j >= 0 && j < ix.dim && isfinite(qv) && qv != 0.0f) {
                uint32_t s = group_hash_slot(j);
                for (int probe = 0; probe < kGroupHash; probe++) {
                    const int32_t old = atomicCAS(&hkey[s], -1, j);
                    if (old == -1 || old == j) break;
                    s = (s + 1) & (kGroupHash - 1);
                }
                my_slot = (int)s;
                my_i = i;
                my_w = (DT == SINDI_F8E4M3) ? qv * ix.scale[j] : qv;
                atomicOr(&hval[s], 1u << i);
            }
        }
        __syncthreads();
        // ---- occupied slots -> union terms 0 .. nu - 1 (slot order)
        constexpr int SPT = (kGroupHash + BLOCK - 1) / BLOCK;  // slots per thread
        uint32_t occ = 0;
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            const int s = tid * SPT + k;
            if (s < kGroupHash && hkey[s] >= 0) occ++;
        }
        uint32_t nu;
        uint32_t u = group_exclusive_sum<uint32_t, S>(occ, &nu, red);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            const int s = tid * SPT + k;
            if (s < kGroupHash && hkey[s] >= 0) {
                const uint32_t hv = hval[s];
                hval[s] = (hv & 0xFFFFu) | (u << 16);
                t_start[u] = (uint32_t)hkey[s];  // the dim, for now
                t_mask[u] = hv & 0xFFFFu;
                u++;
            }
        }
        for (uint32_t x = tid; x < nu * kMaxGroup; x += BLOCK) t_w[x] = 0.0f;
        __syncthreads();
        if (my_slot >= 0) t_w[(hval[my_slot] >> 16) * kMaxGroup + my_i] = my_w;
        // ---- the segment I_{j,w} of every union term, and the chunks that tile it
        uint32_t nch = 0;
        if (tid < (int)nu) {
            uint32_t start = 0, len = 0;
            if (checked(list_in_bounds((int32_t)t_start[tid], w, ix.dim, ix.sigma), ix.err)) {
                const uint64_t sg = (uint64_t)t_start[tid] * ix.sigma + w;
                start = ix.seg[sg];
                len = ix.seg[sg + 1] - start;
            }
            t_start[tid] = start;
            t_end[tid] = start + len;
            nch = len >= kVecMin ? long_segment_chunks(start, start + len) : (len ? 1u : 0u);
        }
        uint32_t n_chunks;
        const uint32_t excl = group_exclusive_sum<uint32_t, S>(nch, &n_chunks, red);
        if (tid < (int)nu) {
            c_pre[tid] = excl;
            for (uint32_t c = excl; c < excl + nch && c < (uint32_t)kChunkTable; c++) c_term[c] = (uint16_t)tid;
        }
        __syncthreads();
        // ---- scatter-add: warp `warp` takes chunks warp, warp + NW, ...; the next
        // chunk's loads are issued before this chunk's adds
        {
            auto load_c = [&](uint32_t c, Chunk& k) -> int {
                const int t = c < (uint32_t)kChunkTable ? (int)c_term[c] : term_of(c_pre, (int)nu, c);
                load_segment_chunk<DT>(ix, t_start[t], t_end[t], (c - c_pre[t]) * (uint32_t)kChunkLen, lane, k);
                return t;
            };
            uint32_t c = (uint32_t)warp;
            Chunk cur;
            int tc = 0;
            if (c < n_chunks) tc = load_c(c, cur);
            while (c < n_chunks) {
                const uint32_t cn = c + NW;
                Chunk nxt;
                int tn = 0;
                if (cn < n_chunks) tn = load_c(cn, nxt);
                add_chunk_holders(A, lam4, lambda, ix.err, t_mask[tc], t_w + (size_t)tc * kMaxGroup, cur);
                cur = nxt;
                tc = tn;
                c = cn;
            }
        }
        __syncthreads();  // tables and hash are reused by the next pass
    }

    allow_next_kernel();
    wait_previous_kernels();  // the workspace (candidates, H) is free from here on
    const CutScratch cs{hist, hist2, region, (uint32_t)group_region_bytes(BLOCK), warp_off, red, st, &s_staged};
    for (uint32_t i = 0; i < qn; i++) {
        const uint32_t y = mrow[i];
        // the query's running bound: g candidates emitted at or above some bin (H only
        // grows while the launch runs, so any read of it bounds the answer)
        const uint32_t* H = sa.ws.hist + (size_t)y * kHistBins;
        block_find_bin<kHistBins, BLOCK>([&](int b) { return __ldcg(H + b); }, sa.g, red, st);
        const bool bounded = st[3] >= sa.g;
        const uint32_t pbin = st[0];
        __syncthreads();
        // zero-score slots cannot count once the earlier windows hold g slots, when no score can be negative
        const bool skip_zero = !((s_negmask >> i) & 1u) && ix.nonneg && (uint64_t)w * lambda >= sa.g;
        select_window<S, NW>(sa, A + (size_t)i * lam4, w, y, bounded, pbin, cs, skip_zero);
    }
}

// ---------------------------------------------------------------------------
// Query hash in shared memory: dims -> weights (merge checks the query with
// it; rerank reads weights from it).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_slot(int32_t j) { return ((uint32_t)j * 2654435761u) >> (32 - 12); }

template <int BLOCK>
__device__ void build_query_hash(const int32_t* qi, const float* qv, int nt, int32_t dim, int32_t* hk, float* hv,
                                 uint32_t* err, bool report) {
    for (int s = threadIdx.x; s < kHashSlots; s += BLOCK) hk[s] = -1;
    __syncthreads();
    if (nt > kQueryTermLimit) {
        if (report && threadIdx.x == 0) atomicOr(err, kErrQueryTooLong);
        __syncthreads();
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
                if (hv) hv[s] = v;
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

// Sorts s[0..cnt) (cnt <= kMaxK) descending and writes the first k as the
// results of query row r, padded with id 0xFFFFFFFF / score -inf.
template <int BLOCK>
__device__ void write_sorted_results(uint64_t* s, int cnt, uint32_t k, uint32_t* out_ids, float* out_scores,
                                     int64_t r) {
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
        out_ids[(size_t)r * k + t] = id;
        out_scores[(size_t)r * k + t] = sc;
    }
}

// Gathers the keys >= T of key_of(0..n) into dst[0..cap) (block-wide, order
// arbitrary); *counter (shared, zero on entry) ends at the number found.
template <int BLOCK, typename KeyOf>
__device__ void gather_at_least(const KeyOf& key_of, uint32_t n, uint64_t T, uint64_t* dst, uint32_t cap,
                                uint32_t* counter) {
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    for (uint32_t base = 0; base < n; base += BLOCK) {
        const uint32_t i = base + threadIdx.x;
        uint64_t k = 0;
        bool ok = false;
        if (i < n) {
            k = key_of(i);
            ok = k >= T;
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        uint32_t wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(counter, (uint32_t)__popc(bal));
        wb = __shfl_sync(kFull, wb, 0);
        if (ok) {
            const uint32_t pos = wb + (uint32_t)__popc(bal & lt);
            if (pos < cap) dst[pos] = k;
        }
    }
    __syncthreads();
}

struct MergeArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    uint32_t g;
    int final_stage;           // 1: the g = min(k, N) results are the answer
    uint32_t k;
    uint32_t* out_ids;         // absolute query rows
    float* out_scores;
    Workspace ws;
};

__global__ void __launch_bounds__(kMergeThreads) merge_kernel(MergeArgs a) {
    extern __shared__ uint64_t sbuf[];          // [fcap]
    __shared__ uint64_t sel[kMaxK];
    __shared__ uint32_t red[kMaxScanWarps + 1];
    __shared__ uint32_t st[4];
    __shared__ uint32_t hist256[256];
    __shared__ uint32_t s_n;
    __shared__ int s_last;
    const Workspace& ws = a.ws;
    const uint32_t y = blockIdx.y;
    const int64_t r = a.q_first + y;
    if (blockIdx.x == 0) {
        // check the query (dims, values, repeats) while the scan still runs: the
        // query is an input of the call, no kernel of the search writes it
        const int64_t qb = a.q_indptr[r];
        const int nt = (int)(a.q_indptr[r + 1] - qb);
        build_query_hash<kMergeThreads>(a.q_indices + qb, a.q_values + qb, nt, a.ix.dim,
                                        reinterpret_cast<int32_t*>(sbuf), nullptr, a.ix.err, true);
    }
    wait_previous_kernels();
    const uint32_t C = min(ws.cand_count[y], ws.cand_cap);
    uint32_t* H = ws.hist + (size_t)y * kHistBins;
    // Every block takes one ticket on the query's way out, whatever path it takes; the last one leaves
    // the query's counters and H at zero for the next launch that uses this workspace. (A block must not
    // reset them while another block of the grid may still read H.)
    auto finish = [&]() {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(ws.mticket + y, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        for (int b = threadIdx.x; b < kHistBins; b += kMergeThreads) H[b] = 0;
        if (threadIdx.x == 0) {
            ws.cand_count[y] = 0;
            ws.fcount[y] = 0;
            ws.mticket[y] = 0;
        }
    };
    // S <= C: with C within both limits block 0 merges the query alone (below), the others have no work
    if (blockIdx.x != 0 && C <= kMergeOneBlock && C <= ws.fcap) {
        finish();
        return;
    }
    const uint32_t g = a.g < C ? a.g : C;
    const uint64_t* cand = ws.cand + (size_t)y * ws.cand_cap;

    // bin of the g-th best candidate; every candidate below it is out
    block_find_bin<kHistBins, kMergeThreads>([&](int b) { return __ldcg(H + b); }, g, red, st);
    const uint32_t bstar = st[0];
    const uint32_t S = st[1] + st[2];  // candidates in bins >= bstar
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    uint64_t* dst = a.final_stage ? sel : ws.top + (size_t)y * ws.top_cap;
    const uint32_t dcap = a.final_stage ? (uint32_t)kMaxK : ws.top_cap;
    if (C <= kMergeOneBlock && S <= ws.fcap) {
        // few candidates: block 0 alone gathers the survivors into shared
        // memory and selects; no filter buffer
        if (blockIdx.x != 0) {
            finish();
            return;
        }
        for (uint32_t base = 0; base < C; base += kMergeThreads * 4) {
            uint64_t kk[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t i = base + (uint32_t)(u * kMergeThreads) + threadIdx.x;
                kk[u] = i < C ? __ldcg(cand + i) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t i = base + (uint32_t)(u * kMergeThreads) + threadIdx.x;
                if (i < C && (uint32_t)(kk[u] >> kKeyBinShift) >= bstar &&
                    checked(doc_in_bounds(key_id(kk[u]), a.ix.n_docs), a.ix.err)) {
                    const uint32_t pos = atomicAdd(&s_n, 1u);
                    if (pos < ws.fcap) sbuf[pos] = kk[u];
                }
            }
        }
        __syncthreads();
        const uint32_t nf = min(s_n, ws.fcap);
        __syncthreads();
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        allow_next_kernel();  // the rerank may launch once the other block has taken its ticket and exited
        auto key_of = [&](int i) -> uint64_t { return sbuf[i]; };
        const uint64_t T = nf > g ? block_select_threshold<kMergeThreads>(key_of, (int)nf, (int)g, hist256, st) : 0ull;
        gather_at_least<kMergeThreads>(key_of, nf, T, dst, dcap, &s_n);
        if (a.final_stage) {
            write_sorted_results<kMergeThreads>(sel, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores,
                                                r);
        } else if (threadIdx.x == 0) {
            ws.top_count[y] = min(s_n, ws.top_cap);
        }
        finish();
        return;
    }
    {
        // this block's slice: survivors gathered in shared memory, then one
        // reservation in the query's filter buffer
        const uint32_t per = (C + gridDim.x - 1) / gridDim.x;
        const uint32_t lo = blockIdx.x * per, hi = min(C, lo + per);
        for (uint32_t base = lo; base < hi; base += kMergeThreads * 4) {
            uint64_t kk[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t i = base + (uint32_t)(u * kMergeThreads) + threadIdx.x;
                kk[u] = i < hi ? __ldcg(cand + i) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t i = base + (uint32_t)(u * kMergeThreads) + threadIdx.x;
                if (i < hi && (uint32_t)(kk[u] >> kKeyBinShift) >= bstar &&
                    checked(doc_in_bounds(key_id(kk[u]), a.ix.n_docs), a.ix.err)) {
                    const uint32_t pos = atomicAdd(&s_n, 1u);
                    if (pos < ws.fcap) sbuf[pos] = kk[u];
                }
            }
        }
        __syncthreads();
        const uint32_t n_local = min(s_n, ws.fcap);
        if (threadIdx.x == 0) st[0] = n_local ? atomicAdd(ws.fcount + y, n_local) : 0u;
        __syncthreads();
        const uint32_t at = st[0];
        uint64_t* fb = ws.fbuf + (size_t)y * ws.fcap;
        for (uint32_t i = threadIdx.x; i < n_local; i += kMergeThreads)
            if (at + i < ws.fcap) fb[at + i] = sbuf[i];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ws.mticket + y, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- last block of the query: exact best g
    allow_next_kernel();
    const uint32_t nf = min(__ldcg(ws.fcount + y), ws.fcap);
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (S <= ws.fcap) {
        const uint64_t* fb = ws.fbuf + (size_t)y * ws.fcap;
        for (uint32_t i = threadIdx.x; i < nf; i += kMergeThreads) sbuf[i] = __ldcg(fb + i);
        __syncthreads();
        auto key_of = [&](int i) -> uint64_t { return sbuf[i]; };
        const uint64_t T = nf > g ? block_select_threshold<kMergeThreads>(key_of, (int)nf, (int)g, hist256, st) : 0ull;
        gather_at_least<kMergeThreads>(key_of, nf, T, dst, dcap, &s_n);
    } else {
        // a crowded bin at the cut: select over every candidate
        auto key_of = [&](int i) -> uint64_t { return __ldcg(cand + i); };
        const uint64_t T = C > g ? block_select_threshold<kMergeThreads>(key_of, (int)C, (int)g, hist256, st) : 0ull;
        gather_at_least<kMergeThreads>(key_of, C, T, dst, dcap, &s_n);
    }
    if (a.final_stage) {
        write_sorted_results<kMergeThreads>(sel, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores, r);
    } else if (threadIdx.x == 0) {
        ws.top_count[y] = min(s_n, ws.top_cap);
    }
    __syncthreads();
    // leave the query's counters at zero for the next launch
    for (int b = threadIdx.x; b < kHistBins; b += kMergeThreads) H[b] = 0;
    if (threadIdx.x == 0) {
        ws.cand_count[y] = 0;
        ws.fcount[y] = 0;
        ws.mticket[y] = 0;
    }
}

// ---------------------------------------------------------------------------
// Merge of document-sharded result rows (sindi_merge_topk): shard s searched
// the documents from id_offset[s] on as an index of its own; its rows hold
// local ids. One block per query gathers every shard's row with ids made
// global, keeps the best k by the search's own order (score desc, id asc) and
// writes them sorted, padded like a search row.
// ---------------------------------------------------------------------------
struct MergeShardsArgs {
    const uint32_t* ids;      // [n_shards][n_queries][k_in]
    const float* scores;
    int64_t n_queries;
    uint32_t n_shards, k_in, k;
    uint32_t* out_ids;        // [n_queries][k]
    float* out_scores;
    int64_t offset[kMaxShards];
};

constexpr int kShardMergeThreads = 256;

__global__ void __launch_bounds__(kShardMergeThreads) merge_shards_kernel(MergeShardsArgs a) {
    extern __shared__ uint64_t sk[];          // [n_shards * k_in]
    __shared__ uint64_t sel[kMaxK];
    __shared__ uint32_t hist256[256];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_n;
    const int64_t q = blockIdx.x;
    const uint32_t n_all = a.n_shards * a.k_in;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    // every shard's valid entries, global ids, as order keys (padding dropped)
    for (uint32_t i = threadIdx.x; i < n_all; i += kShardMergeThreads) {
        const uint32_t sh = i / a.k_in, j = i - sh * a.k_in;
        const size_t at = ((size_t)sh * a.n_queries + q) * a.k_in + j;
        const uint32_t id = a.ids[at];
        if (id != 0xFFFFFFFFu) {
            const int64_t gid = (int64_t)id + a.offset[sh];
            sk[atomicAdd(&s_n, 1u)] = result_key(a.scores[at], (uint32_t)gid);
        }
    }
    __syncthreads();
    const uint32_t n = s_n;
    const uint32_t g = n < a.k ? n : a.k;
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    auto key_of = [&](int i) -> uint64_t { return sk[i]; };
    const uint64_t T = n > g ? block_select_threshold<kShardMergeThreads>(key_of, (int)n, (int)g, hist256, st) : 0ull;
    gather_at_least<kShardMergeThreads>(key_of, n, T, sel, kMaxK, &s_n);
    write_sorted_results<kShardMergeThreads>(sel, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores, q);
}

void merge_shards(const uint32_t* ids, const float* scores, uint32_t n_shards, int64_t n_queries, uint32_t k_in,
                  const int64_t* id_offset, uint32_t k, uint32_t* out_ids, float* out_scores, cudaStream_t stream) {
    static std::mutex mu;
    static std::vector<int> done;
    int device = 0;
    SINDI_CUDA(cudaGetDevice(&device));
    {
        std::lock_guard<std::mutex> lk(mu);
        if (std::find(done.begin(), done.end(), device) == done.end()) {
            SINDI_CUDA(cudaFuncSetAttribute(merge_shards_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(kMaxShardEntries * 8)));
            done.push_back(device);
        }
    }
    MergeShardsArgs a{ids, scores, n_queries, n_shards, k_in, k, out_ids, out_scores, {}};
    for (uint32_t s = 0; s < n_shards; s++) a.offset[s] = id_offset[s];
    const size_t smem = (size_t)n_shards * k_in * 8;
    merge_shards_kernel<<<(unsigned)n_queries, kShardMergeThreads, smem, stream>>>(a);
    SINDI_CUDA(cudaGetLastError());
}

struct RerankArgs {
    DevIndex ix;
    const int64_t* q_indptr;
    const int32_t* q_indices;
    const float* q_values;
    int64_t q_first;
    uint32_t k;
    uint32_t* out_ids;
    float* out_scores;
    Workspace ws;
};

__global__ void __launch_bounds__(kRerankThreads) rerank_kernel(RerankArgs a) {
    extern __shared__ uint64_t rk[];  // [top_cap]: the exact keys, in the query's last block
    __shared__ int32_t hk[kHashSlots];
    __shared__ float hv[kHashSlots];
    __shared__ uint64_t s[kMaxK];
    __shared__ uint32_t hist256[256];
    __shared__ uint32_t st[4];
    __shared__ uint32_t s_n;
    __shared__ int s_last;
    const Workspace& ws = a.ws;
    const uint32_t y = blockIdx.y;
    const int64_t r = a.q_first + y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    allow_next_kernel();
    {
        const int64_t qb = a.q_indptr[r];
        const int nt = (int)(a.q_indptr[r + 1] - qb);
        build_query_hash<kRerankThreads>(a.q_indices + qb, a.q_values + qb, nt, a.ix.dim, hk, hv, a.ix.err, false);
    }
    wait_previous_kernels();
    const uint32_t g = min(ws.top_count[y], ws.top_cap);
    uint64_t* rr = ws.rr + (size_t)y * ws.top_cap;
    // one half-warp per candidate: lanes 0-15 and 16-31 score two documents
    const int half = lane >> 4, hl = lane & 15;
    const unsigned hmask = half ? 0xFFFF0000u : 0x0000FFFFu;
    const uint32_t idx = (blockIdx.x * kRerankWarps + warp) * 2 + half;
    if (idx < g) {
        const uint64_t key = ws.top[(size_t)y * ws.top_cap + idx];
        const uint32_t id = key_id(key);
        const bool id_ok = checked(doc_in_bounds(id, a.ix.n_docs), a.ix.err);
        const int64_t b = id_ok ? a.ix.indptr[id] : 0, e0 = id_ok ? a.ix.indptr[id + 1] : 0;
        const int64_t e = checked(row_in_bounds(b, e0, a.ix.doc_nnz), a.ix.err) ? e0 : b;
        float acc = 0.0f;
        // the row's entries, up to 16 * kRerankU at a time, all loads issued before the first is used
        for (int64_t p0 = b; p0 < e; p0 += 16 * kRerankU) {
            int32_t jj[kRerankU];
            float xx[kRerankU];
#pragma unroll
            for (int u = 0; u < kRerankU; u++) {
                const int64_t p = p0 + u * 16 + hl;
                jj[u] = -1;
                xx[u] = 0.0f;
                if (p < e) {
                    jj[u] = __ldg(a.ix.indices + p);
                    xx[u] = __ldg(a.ix.values + p);
                }
            }
#pragma unroll
            for (int u = 0; u < kRerankU; u++)
                if (jj[u] >= 0) acc = fmaf(xx[u], query_weight(hk, hv, jj[u]), acc);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(hmask, acc, o);
        if (hl == 0) rr[idx] = result_key(acc, id);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ws.rticket + y, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    {
        // the best k of the g exact scores (copied to shared memory once), then sort only those
        for (uint32_t i = threadIdx.x; i < g; i += kRerankThreads) rk[i] = __ldcg(rr + i);
        __syncthreads();
        const uint32_t kk = a.k < g ? a.k : g;
        auto key_of = [&](int i) -> uint64_t { return rk[i]; };
        const uint64_t T = g > kk ? block_select_threshold<kRerankThreads>(key_of, (int)g, (int)kk, hist256, st) : 0ull;
        gather_at_least<kRerankThreads>(key_of, g, T, s, kMaxK, &s_n);
    }
    write_sorted_results<kRerankThreads>(s, (int)min(s_n, (uint32_t)kMaxK), a.k, a.out_ids, a.out_scores, r);
    if (threadIdx.x == 0) ws.rticket[y] = 0;
}

// beta-mass of every query (Alg. 4: q' = beta-mass(q), the alpha-mass rule
// with beta): one warp per query. Its kept entries go to the query's own
// positions of (pidx, pval), their count to kept[q]. Entries the scan would
// skip anyway (dim out of range, non-finite, zero) are not entries here.
constexpr int kPruneQueryWarps = 4;
constexpr size_t kPruneQuerySmem = (size_t)kPruneQueryWarps * kQueryTermLimit * sizeof(uint64_t);
__global__ void __launch_bounds__(kPruneQueryWarps * 32) prune_queries_kernel(
    const int64_t* qp, const int32_t* qi, const float* qv, int64_t nq, int32_t dim, double beta, uint32_t* kept,
    int32_t* pidx, float* pval) {
    extern __shared__ uint64_t qsm[];  // [warps][kQueryTermLimit]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* s = qsm + (size_t)warp * kQueryTermLimit;
    for (int64_t q = (int64_t)blockIdx.x * kPruneQueryWarps + warp; q < nq;
         q += (int64_t)gridDim.x * kPruneQueryWarps) {
        const int64_t b = qp[q];
        const int64_t m = qp[q + 1] - b;
        if (m > kQueryTermLimit) {  // refused: merge reports the query as too long
            if (lane == 0) kept[q] = 0;
            continue;
        }
        int p2 = 32;
        while (p2 < m) p2 <<= 1;
        int nz = 0;
        for (int t = lane; t < p2; t += 32) {
            uint64_t key = ~0ull;
            if (t < m) {
                const int32_t j = qi[b + t];
                const float v = qv[b + t];
                if (j >= 0 && j < dim && isfinite(v) && v != 0.0f) {
                    key = mass_key(j, v);
                    nz++;
                }
            }
            s[t] = key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(kFull, nz, o);
        __syncwarp();
        warp_bitonic_sort_asc(s, p2);
        int r = 0;
        if (lane == 0) r = alpha_mass_count(s, nz, beta);
        r = __shfl_sync(kFull, r, 0);
        for (int t = lane; t < r; t += 32) {
            pidx[b + t] = mass_key_dim(s[t]);
            pval[b + t] = mass_key_value(s[t]);
        }
        if (lane == 0) kept[q] = (uint32_t)r;
        __syncwarp();
    }
}

// Kept query entries -> compact CSR.
__global__ void compact_queries_kernel(const int64_t* qp, const int64_t* off, const int32_t* pidx, const float* pval,
                                       int64_t nq, int32_t* oidx, float* oval) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nq; q += warps) {
        const int64_t b = qp[q], o = off[q], r = off[q + 1] - o;
        for (int64_t t = lane; t < r; t += 32) {
            oidx[o + t] = pidx[b + t];
            oval[o + t] = pval[b + t];
        }
    }
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
// Sizes of one search: candidates per query and the buffers that follow.
struct Plan {
    bool final_stage;
    uint32_t g, win_cap, cand_cap, fcap, top_cap, merge_blocks, block;
    uint32_t group;  // batched scan: queries per block (1 = one block per (query, window))
    bool fixed;      // the one-block-per-window scan accumulates in fixed point
};

// Queries per block of the batched scan: as asked (0: one, the fastest shape
// measured on the 1M-document workload), at most kMaxGroup and at most what
// shared memory holds.
static uint32_t group_size(const IndexImpl& ix, uint32_t asked, uint32_t block) {
    const int bt = block == 1024 ? 1024 : 512;
    uint32_t q = asked ? asked : 1u;
    q = std::min<uint32_t>(q, (uint32_t)kMaxGroup);
    while (q > 1 && group_smem_bytes(ix.lambda, q, bt) > kGroupDynSmemMax) q--;
    return q;
}

static Plan make_plan(const IndexImpl& ix, const sindi_search_params& prm) {
    Plan p;
    p.final_stage = prm.gamma == 0;
    p.g = (uint32_t)std::min<int64_t>(p.final_stage ? prm.k : prm.gamma, ix.n_docs);
    const uint32_t gw = std::min<uint32_t>(p.g, ix.lambda);
    p.win_cap = 2 * gw;
    p.cand_cap = ix.sigma * p.win_cap;
    uint32_t f = 4096;
    while (f < 2 * p.g && f < 16384) f <<= 1;
    p.fcap = f;
    p.top_cap = p.final_stage ? 1 : p.g;
    // two blocks: a query's merge is one block unless its candidates crowd the cut, and every block of
    // the grid is resident (holding its shared memory) while the scan finishes
    p.merge_blocks = std::max<uint32_t>(1, std::min<uint32_t>(2, p.cand_cap / 8192));
    p.block = prm.block_threads;
    p.group = group_size(ix, prm.group, prm.block_threads);
    p.fixed = prm.accumulator == SINDI_ACCUM_FIXED32 || (prm.accumulator == SINDI_ACCUM_AUTO && !p.final_stage);
    return p;
}

// Launches `kern` on `stream`; with `pdl` the launch may begin while the
// previous kernel on the stream still runs (the kernel waits for it where it
// must, see wait_previous_kernels).
template <typename... Params, typename... Args>
static void launch_kernel(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream, bool pdl,
                          Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    SINDI_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

template <int DT, bool QM, int BLOCK>
static void allow_window_smem() {
    SINDI_CUDA(cudaFuncSetAttribute(scan_window_kernel<DT, QM, BLOCK, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxWindow * sizeof(float))));
    SINDI_CUDA(cudaFuncSetAttribute(scan_window_kernel<DT, QM, BLOCK, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxWindow * sizeof(float))));
}

template <int DT>
static void allow_window_smem_dt() {
    SINDI_CUDA(cudaFuncSetAttribute(scan_pipe_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pipe_smem_bytes(kPipeMaxWindow)));
    allow_window_smem<DT, false, 256>();
    allow_window_smem<DT, false, 512>();
    allow_window_smem<DT, false, 1024>();
    allow_window_smem<DT, true, 256>();
    allow_window_smem<DT, true, 512>();
    allow_window_smem<DT, true, 1024>();
}

// SMs of the device (once per device).
static int device_sms(int device) {
    static std::mutex mu;
    static std::map<int, int> sms;
    std::lock_guard<std::mutex> lk(mu);
    auto it = sms.find(device);
    if (it != sms.end()) return it->second;
    int n = 0;
    SINDI_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device));
    sms[device] = n;
    return n;
}

template <int DT>
static void launch_pipe_t(const ScanArgs& a, uint32_t blocks, size_t smem, cudaStream_t s, bool pdl) {
    launch_kernel(scan_pipe_kernel<DT>, dim3(blocks), dim3(kPipeThreads), smem, s, pdl, a);
}

static void launch_pipe(int dt, const ScanArgs& a, uint32_t blocks, size_t smem, cudaStream_t s, bool pdl) {
    if (dt == SINDI_F32) launch_pipe_t<SINDI_F32>(a, blocks, smem, s, pdl);
    else if (dt == SINDI_F16) launch_pipe_t<SINDI_F16>(a, blocks, smem, s, pdl);
    else launch_pipe_t<SINDI_F8E4M3>(a, blocks, smem, s, pdl);
}

template <int DT>
static void allow_group_smem() {
    SINDI_CUDA(cudaFuncSetAttribute(group_scan_kernel<DT, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kGroupDynSmemMax));
    SINDI_CUDA(cudaFuncSetAttribute(group_scan_kernel<DT, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kGroupDynSmemMax));
}

template <int DT, int BLOCK>
static void launch_group_scan_t(const GroupScanArgs& a, uint32_t n_groups, uint32_t nwin, size_t smem,
                                cudaStream_t s, bool pdl) {
    launch_kernel(group_scan_kernel<DT, BLOCK>, dim3(n_groups, nwin), dim3(BLOCK), smem, s, pdl, a);
}

static void launch_group_scan(int dt, uint32_t block, const GroupScanArgs& a, uint32_t n_groups, uint32_t nwin,
                              size_t smem, cudaStream_t s, bool pdl) {
    if (block == 1024) {
        if (dt == SINDI_F32) launch_group_scan_t<SINDI_F32, 1024>(a, n_groups, nwin, smem, s, pdl);
        else if (dt == SINDI_F16) launch_group_scan_t<SINDI_F16, 1024>(a, n_groups, nwin, smem, s, pdl);
        else launch_group_scan_t<SINDI_F8E4M3, 1024>(a, n_groups, nwin, smem, s, pdl);
    } else {
        if (dt == SINDI_F32) launch_group_scan_t<SINDI_F32, 512>(a, n_groups, nwin, smem, s, pdl);
        else if (dt == SINDI_F16) launch_group_scan_t<SINDI_F16, 512>(a, n_groups, nwin, smem, s, pdl);
        else launch_group_scan_t<SINDI_F8E4M3, 512>(a, n_groups, nwin, smem, s, pdl);
    }
}

// Shared-memory limits of every search kernel, set once per device before the
// first launch (and before any stream capture, where they cannot be set).
void configure_search_kernels(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return;
    allow_window_smem_dt<SINDI_F32>();
    allow_window_smem_dt<SINDI_F16>();
    allow_window_smem_dt<SINDI_F8E4M3>();
    allow_group_smem<SINDI_F32>();
    allow_group_smem<SINDI_F16>();
    allow_group_smem<SINDI_F8E4M3>();
    SINDI_CUDA(cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8));
    SINDI_CUDA(cudaFuncSetAttribute(rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxGamma * 8));
    SINDI_CUDA(cudaFuncSetAttribute(prune_queries_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kPruneQuerySmem));
    done.push_back(device);
}

template <int DT, bool QM, int BLOCK>
static void launch_scan_t(const ScanArgs& a, uint32_t sigma, uint32_t nq, size_t smem, cudaStream_t s, bool pdl) {
    dim3 grid = QM ? dim3(nq, sigma) : dim3(sigma, nq);
    if (a.fixed) launch_kernel(scan_window_kernel<DT, QM, BLOCK, true>, grid, dim3(BLOCK), smem, s, pdl, a);
    else launch_kernel(scan_window_kernel<DT, QM, BLOCK, false>, grid, dim3(BLOCK), smem, s, pdl, a);
}

// Plain schedules (one query) take window-major grids; batched schedules take
// query-major grids (window-major when sigma exceeds the grid's y limit). Both
// default to 512-thread blocks.
template <int DT, bool QM>
static void launch_scan_block(uint32_t block, const ScanArgs& a, uint32_t sigma, uint32_t nq, size_t smem,
                              cudaStream_t s, bool pdl) {
    if (block == 256) launch_scan_t<DT, QM, 256>(a, sigma, nq, smem, s, pdl);
    else if (block == 512) launch_scan_t<DT, QM, 512>(a, sigma, nq, smem, s, pdl);
    else launch_scan_t<DT, QM, 1024>(a, sigma, nq, smem, s, pdl);
}

template <int DT>
static void launch_scan_dt(uint32_t block, bool batched, bool qm, const ScanArgs& a, uint32_t sigma, uint32_t nq,
                           size_t smem, cudaStream_t s, bool pdl) {
    if (block == 0) block = batched ? kScanThreadsBatched : kScanThreadsPlain;
    if (qm) launch_scan_block<DT, true>(block, a, sigma, nq, smem, s, pdl);
    else launch_scan_block<DT, false>(block, a, sigma, nq, smem, s, pdl);
}

static void launch_scan_pdl(int dt, uint32_t block, bool batched, bool qm, const ScanArgs& a, uint32_t sigma,
                            uint32_t nq, size_t smem, cudaStream_t s, bool pdl) {
    if (dt == SINDI_F32) launch_scan_dt<SINDI_F32>(block, batched, qm, a, sigma, nq, smem, s, pdl);
    else if (dt == SINDI_F16) launch_scan_dt<SINDI_F16>(block, batched, qm, a, sigma, nq, smem, s, pdl);
    else launch_scan_dt<SINDI_F8E4M3>(block, batched, qm, a, sigma, nq, smem, s, pdl);
}

// The launches of one group of nq queries starting at row q0. `*chained` is
// false for the first launch of a search call (it follows the caller's work
// and must not overlap it) and true afterwards.
struct QueryCsr {
    const int64_t* indptr;
    const int32_t* indices;
    const float* values;
};

static void launch_group(const IndexImpl& ix, const Plan& pl, const Workspace& ws, const int64_t* q_indptr,
                         const int32_t* q_indices, const float* q_values, int64_t q0, uint32_t nq, bool batched,
                         uint32_t k, uint32_t* out_ids, float* out_scores, cudaStream_t stream, bool* chained,
                         cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, const QueryCsr* scan_q = nullptr) {
    configure_search_kernels(ix.device);
    const DevIndex dix = ix.dev();
    const size_t scan_smem = (size_t)window_stride(ix.lambda) * sizeof(float);
    // the coarse scan reads the beta-pruned queries when there are any (Alg. 4, the query-pruning step);
    // merge and rerank check and reorder with the full queries
    ScanArgs sa{dix, scan_q ? scan_q->indptr : q_indptr, scan_q ? scan_q->indices : q_indices,
                scan_q ? scan_q->values : q_values, q0, pl.g, pl.win_cap, batched ? 1 : 0, 0u, nq, ix.sigma, ws,
                pl.fixed ? 1 : 0};
    if (ev0) SINDI_CUDA(cudaEventRecord(ev0, stream));
    // the pipelined scan when asked for and its two window arrays fit; any
    // other shape is one block per window (block 0 or 1: the default size)
    const bool pipe = pl.block == SINDI_SCAN_PIPELINED && ix.lambda <= kPipeMaxWindow;
    const uint32_t block = pl.block == SINDI_SCAN_PIPELINED ? 0u : pl.block;
    const size_t pipe_smem = pipe_smem_bytes(ix.lambda);
    if (batched && !pipe && pl.group > 1 && ix.sigma <= 65535u) {
        // query groups: one block per (group, window); groups vary fastest, so the
        // blocks of one window run together and its lists stay in L2
        const uint32_t bt = pl.block == 1024 ? 1024u : 512u;
        const GroupScanArgs ga{sa, pl.group, nq};
        launch_group_scan(ix.dtype, bt, ga, (nq + pl.group - 1) / pl.group, ix.sigma,
                          group_smem_bytes(ix.lambda, pl.group, (int)bt), stream, *chained && !ev0);
    } else if (pipe && batched) {
        // one resident block per SM walks the (window, query) items in
        // window-major order, so a query's windows come one after another
        const uint64_t items = (uint64_t)nq * ix.sigma;
        const uint32_t blocks = (uint32_t)std::min<uint64_t>(items, (uint64_t)device_sms(ix.device));
        launch_pipe(ix.dtype, sa, blocks, pipe_smem, stream, *chained && !ev0);
    } else if (!batched && ix.sigma >= kSplitMinWindows) {
        // One query: its first windows run alone and fill the query's
        // histogram of candidates; the other windows then emit only what can
        // still enter the answer (the running bound of Alg. 2's heap, taken
        // from a block of windows instead of one window at a time).
        const uint32_t first = std::max<uint32_t>(2u, (ix.sigma + kSplitFraction - 1) / kSplitFraction);
        launch_scan_pdl(ix.dtype, block, false, false, sa, first, nq, scan_smem, stream, *chained && !ev0);
        ScanArgs sb = sa;
        sb.use_partial = 2;
        sb.w0 = first;
        sb.nwin = ix.sigma - first;
        if (pipe) {
            // a few blocks per query, each walking several windows
            const uint32_t blocks = (sb.nwin + kPlainPipeItems - 1) / kPlainPipeItems;
            launch_pipe(ix.dtype, sb, blocks, pipe_smem, stream, true);
        } else {
            launch_scan_pdl(ix.dtype, block, false, false, sb, ix.sigma - first, nq, scan_smem, stream, true);
        }
        ix.launches += 1;
        ix.scan_launches += 1;
    } else {
        // query-major grids put the queries of one window next to each other
        // (shared lists stay in L2); gridDim.y limits sigma to 65535 there
        launch_scan_pdl(ix.dtype, block, batched, batched && ix.sigma <= 65535u, sa, ix.sigma, nq, scan_smem,
                        stream, *chained && !ev0);
    }
    if (ev1) SINDI_CUDA(cudaEventRecord(ev1, stream));
    MergeArgs ma{dix, q_indptr, q_indices, q_values, q0, pl.g, pl.final_stage ? 1 : 0, k, out_ids, out_scores, ws};
    launch_kernel(merge_kernel, dim3(pl.merge_blocks, nq), dim3(kMergeThreads), (size_t)pl.fcap * 8, stream,
                  !ev1, ma);
    ix.launches += 2;
    ix.scan_launches += 1;
    if (!pl.final_stage) {
        RerankArgs ra{dix, q_indptr, q_indices, q_values, q0, k, out_ids, out_scores, ws};
        launch_kernel(rerank_kernel, dim3(ceil_div_u32(pl.g, 2 * kRerankWarps), nq), dim3(kRerankThreads),
                      (size_t)pl.top_cap * 8, stream, true, ra);
        ix.launches += 1;
    }
    *chained = true;
}

// The plain schedule's launches: query i's chain on lane i mod lanes. Every
// lane starts after the work already on `stream` (fork event) and `stream`
// continues after every lane (join events). The events go to `evs`; the
// caller destroys them once they are recorded (or once a capture ends).
static void enqueue_plain_lanes(const IndexImpl& ix, const Plan& pl, const std::vector<Workspace>& wss,
                                const int64_t* q_indptr, const int32_t* q_indices, const float* q_values,
                                int64_t n_queries, uint32_t k, uint32_t* out_ids, float* out_scores,
                                cudaStream_t stream, const std::vector<cudaStream_t>& ls, const QueryCsr* pruned,
                                std::vector<cudaEvent_t>& evs, bool chain_queries) {
    const int lanes = (int)ls.size();
    cudaEvent_t fork = nullptr;
    SINDI_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    evs.push_back(fork);
    SINDI_CUDA(cudaEventRecord(fork, stream));
    for (cudaStream_t l : ls) SINDI_CUDA(cudaStreamWaitEvent(l, fork, 0));
    std::vector<char> lane_chained(lanes, 0);
    for (int64_t q = 0; q < n_queries; q++) {
        const int l = (int)(q % lanes);
        // chain_queries: a lane's next query may start (programmatic dependent launch) while the previous
        // one's last kernel runs; otherwise it follows that kernel's completion in stream order
        bool c = chain_queries && lane_chained[l] != 0;
        launch_group(ix, pl, wss[l], q_indptr, q_indices, q_values, q, 1, false, k, out_ids, out_scores, ls[l], &c,
                     nullptr, nullptr, pruned);
        lane_chained[l] = c ? 1 : 0;
    }
    for (cudaStream_t l : ls) {
        cudaEvent_t join = nullptr;
        SINDI_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        evs.push_back(join);
        SINDI_CUDA(cudaEventRecord(join, l));
        SINDI_CUDA(cudaStreamWaitEvent(stream, join, 0));
    }
}

// Records the plain schedule of one call as a CUDA graph with workspaces of
// its own, on streams of its own (so no other search's streams are ever in
// capture). Replaces the index's previous graph. Caller holds ix.graph_mu.
static void capture_plain_graph(const IndexImpl& ix, const Plan& pl, const IndexImpl::PlainCall& call, int lanes,
                                const int64_t* q_indptr, const int32_t* q_indices, const float* q_values,
                                int64_t n_queries, uint32_t k, uint32_t* out_ids, float* out_scores) {
    configure_search_kernels(ix.device);  // attributes cannot be set during a capture
    if (ix.graph_exec) {
        SINDI_CUDA(cudaEventSynchronize(ix.graph_done));  // its last launch (and its workspaces) is done
        SINDI_CUDA(cudaGraphExecDestroy(ix.graph_exec));
        ix.graph_exec = nullptr;
    }
    if (!ix.graph_done) SINDI_CUDA(cudaEventCreateWithFlags(&ix.graph_done, cudaEventDisableTiming));
    if (ix.graph_ws) {
        SINDI_CUDA(cudaFree(ix.graph_ws));
        ix.graph_ws = nullptr;
    }
    const size_t ws_one = workspace_bytes(1, pl.cand_cap, pl.fcap, pl.top_cap);
    const size_t ws_stride = (ws_one + 255) & ~(size_t)255;
    unsigned char* mem = nullptr;
    SINDI_CUDA(cudaMalloc(&mem, ws_stride * lanes));
    ix.graph_ws = mem;
    std::vector<Workspace> wss;
    for (int l = 0; l < lanes; l++) wss.push_back(carve_workspace(mem + ws_stride * l, 1, pl.cand_cap, pl.fcap, pl.top_cap));
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> ls(lanes, nullptr);
    std::vector<cudaEvent_t> evs;
    cudaGraph_t graph = nullptr;
    const uint64_t l0 = ix.launches.load(), s0 = ix.scan_launches.load();
    bool capturing = false;
    try {
        SINDI_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        for (auto& l : ls) SINDI_CUDA(cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
        SINDI_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        for (int l = 0; l < lanes; l++)
            SINDI_CUDA(cudaMemsetAsync(mem + ws_stride * l, 0, workspace_counter_bytes(1), cap));
        enqueue_plain_lanes(ix, pl, wss, q_indptr, q_indices, q_values, n_queries, k, out_ids, out_scores, cap, ls,
                            nullptr, evs, true);
        capturing = false;
        SINDI_CUDA(cudaStreamEndCapture(cap, &graph));
        SINDI_CUDA(cudaGraphInstantiate(&ix.graph_exec, graph, 0));
    } catch (...) {
        if (capturing) {
            cudaGraph_t g = nullptr;
            (void)cudaStreamEndCapture(cap, &g);
            if (g) (void)cudaGraphDestroy(g);
        }
        if (graph) (void)cudaGraphDestroy(graph);
        for (cudaEvent_t e : evs) (void)cudaEventDestroy(e);
        for (cudaStream_t l : ls)
            if (l) (void)cudaStreamDestroy(l);
        if (cap) (void)cudaStreamDestroy(cap);
        ix.launches = l0;
        ix.scan_launches = s0;
        throw;
    }
    SINDI_CUDA(cudaGraphDestroy(graph));
    for (cudaEvent_t e : evs) SINDI_CUDA(cudaEventDestroy(e));
    for (cudaStream_t l : ls) SINDI_CUDA(cudaStreamDestroy(l));
    SINDI_CUDA(cudaStreamDestroy(cap));
    // the launches the capture counted happen at every graph launch instead
    ix.graph_launches = ix.launches.load() - l0;
    ix.graph_scan_launches = ix.scan_launches.load() - s0;
    ix.launches = l0;
    ix.scan_launches = s0;
    ix.graph_call = call;
}

sindi_status search_impl(const IndexImpl& ix, const int64_t* q_indptr, const int32_t* q_indices,
                         const float* q_values, int64_t n_queries, const sindi_search_params& prm,
                         uint32_t* out_ids, float* out_scores, cudaStream_t stream) {
    const uint32_t k = prm.k;
    if (n_queries == 0) return SINDI_OK;
    if (ix.n_docs == 0) {
        pad_results_kernel<<<256, 256, 0, stream>>>(out_ids, out_scores, n_queries * (int64_t)k);
        SINDI_CUDA(cudaGetLastError());
        ix.launches++;
        return SINDI_OK;
    }
    const Plan pl = make_plan(ix, prm);
    const bool batched = prm.mode == SINDI_MODE_BATCHED;
    int64_t chunk = 1;
    if (batched) {
        const size_t budget = (size_t)1 << 31;  // 2 GiB of workspace per launch group
        const size_t per_query = workspace_bytes(1, pl.cand_cap, pl.fcap, pl.top_cap);
        chunk = std::max<int64_t>(1, std::min<int64_t>(n_queries, (int64_t)(budget / per_query)));
        chunk = std::min<int64_t>(chunk, 65535);
    }
    const bool timing = ix.timing.load() != 0;
    // The plain schedule runs one launch chain (scan, merge, rerank) per query.
    // A chain is a few microseconds of dependent steps on few SMs after its
    // scan, so up to kPlainLanes chains run at once, each on its own stream
    // with its own workspace; query i takes lane i mod lanes. Timed runs keep
    // one lane, so that a scan's measured duration is its own.
    const int lanes = (batched || timing) ? 1 : (int)std::min<int64_t>(kPlainLanes, n_queries);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    SINDI_CUDA(cudaStreamIsCapturing(stream, &cst));
    if (lanes > 1 && prm.beta >= 1.0 && cst == cudaStreamCaptureStatusNone) {
        // A plain call is thousands of launches, which the host issues about as
        // fast as the GPU runs them. The second identical call (same buffers,
        // size and parameters) records them as a graph; identical calls after
        // it launch the graph.
        IndexImpl::PlainCall call;
        call.buf[0] = q_indptr;
        call.buf[1] = q_indices;
        call.buf[2] = q_values;
        call.buf[3] = out_ids;
        call.buf[4] = out_scores;
        call.n = n_queries;
        call.k = k;
        call.gamma = prm.gamma;
        call.block = prm.block_threads;
        call.accum = prm.accumulator;
        std::lock_guard<std::mutex> lk(ix.graph_mu);
        bool failed = false;
        if (!(ix.graph_exec && ix.graph_call == call) && ix.graph_seen == call) {
            try {
                capture_plain_graph(ix, pl, call, lanes, q_indptr, q_indices, q_values, n_queries, k, out_ids,
                                    out_scores);
            } catch (const CudaError&) {
                (void)cudaGetLastError();
                failed = true;  // launch directly, and do not try this call again
            }
        }
        if (ix.graph_exec && ix.graph_call == call) {
            SINDI_CUDA(cudaGraphLaunch(ix.graph_exec, stream));
            SINDI_CUDA(cudaEventRecord(ix.graph_done, stream));
            ix.launches += ix.graph_launches;
            ix.scan_launches += ix.graph_scan_launches;
            ix.queries += (uint64_t)n_queries;
            return SINDI_OK;
        }
        ix.graph_seen = failed ? IndexImpl::PlainCall{} : call;
    }
    Pool P{ix.pool, stream};
    const size_t ws_one = workspace_bytes(chunk, pl.cand_cap, pl.fcap, pl.top_cap);
    const size_t ws_stride = (ws_one + 255) & ~(size_t)255;
    unsigned char* mem = P.alloc<unsigned char>(ws_stride * lanes);
    std::vector<Workspace> wss;
    for (int l = 0; l < lanes; l++) {
        wss.push_back(carve_workspace(mem + ws_stride * l, chunk, pl.cand_cap, pl.fcap, pl.top_cap));
        SINDI_CUDA(cudaMemsetAsync(mem + ws_stride * l, 0, workspace_counter_bytes(chunk), stream));
    }
    const Workspace& ws = wss[0];
    QueryCsr pruned{nullptr, nullptr, nullptr};
    int64_t* pq_indptr = nullptr;
    int32_t* pq_idx = nullptr;
    float* pq_val = nullptr;
    int32_t* tq_idx = nullptr;
    float* tq_val = nullptr;
    uint32_t* pq_kept = nullptr;
    if (prm.beta < 1.0) {
        int64_t nnz = 0;
        SINDI_CUDA(cudaMemcpyAsync(&nnz, q_indptr + n_queries, 8, cudaMemcpyDeviceToHost, stream));
        SINDI_CUDA(cudaStreamSynchronize(stream));
        pq_kept = P.alloc<uint32_t>(n_queries);
        tq_idx = P.alloc<int32_t>(nnz);
        tq_val = P.alloc<float>(nnz);
        pq_indptr = P.alloc<int64_t>(n_queries + 1);
        pq_idx = P.alloc<int32_t>(nnz);
        pq_val = P.alloc<float>(nnz);
        configure_search_kernels(ix.device);  // the query-pruning kernel's shared-memory limit, per device
        const size_t qsmem = kPruneQuerySmem;
        const unsigned blocks = (unsigned)std::min<int64_t>((n_queries + kPruneQueryWarps - 1) / kPruneQueryWarps,
                                                            152 * 16);
        prune_queries_kernel<<<blocks, kPruneQueryWarps * 32, qsmem, stream>>>(q_indptr, q_indices, q_values,
                                                                               n_queries, ix.dim, prm.beta, pq_kept,
                                                                               tq_idx, tq_val);
        SINDI_CUDA(cudaGetLastError());
        exclusive_scan<uint32_t, int64_t>(pq_kept, pq_indptr, n_queries, P);
        compact_queries_kernel<<<blocks, 256, 0, stream>>>(q_indptr, pq_indptr, tq_idx, tq_val, n_queries, pq_idx,
                                                           pq_val);
        SINDI_CUDA(cudaGetLastError());
        ix.launches += 3;
        pruned = QueryCsr{pq_indptr, pq_idx, pq_val};
    }

    std::vector<cudaEvent_t> evs;
    bool chained = false;
    if (lanes > 1) {
        std::vector<cudaStream_t> ls;
        {
            std::lock_guard<std::mutex> lk(ix.lane_mu);
            while ((int)ix.lanes.size() < lanes) {
                cudaStream_t l = nullptr;
                SINDI_CUDA(cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
                ix.lanes.push_back(l);
            }
            ls.assign(ix.lanes.begin(), ix.lanes.begin() + lanes);
        }
        std::vector<cudaEvent_t> evs_lane;
        enqueue_plain_lanes(ix, pl, wss, q_indptr, q_indices, q_values, n_queries, k, out_ids, out_scores, stream, ls,
                            pruned.indptr ? &pruned : nullptr, evs_lane, false);
        for (cudaEvent_t e : evs_lane) SINDI_CUDA(cudaEventDestroy(e));
    }
    for (int64_t q0 = 0; lanes == 1 && q0 < n_queries; q0 += chunk) {
        const uint32_t nq = (uint32_t)std::min<int64_t>(chunk, n_queries - q0);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timing) {
            SINDI_CUDA(cudaEventCreate(&e0));
            SINDI_CUDA(cudaEventCreate(&e1));
            evs.push_back(e0);
            evs.push_back(e1);
        }
        launch_group(ix, pl, ws, q_indptr, q_indices, q_values, q0, nq, batched, k, out_ids, out_scores, stream,
                     &chained, e0, e1, pruned.indptr ? &pruned : nullptr);
    }
    ix.queries += (uint64_t)n_queries;
    P.free(mem);
    P.free(pq_kept);
    P.free(tq_idx);
    P.free(tq_val);
    P.free(pq_indptr);
    P.free(pq_idx);
    P.free(pq_val);
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

sindi_status search_noalloc_impl(const IndexImpl& ix, const int64_t* q_indptr, const int32_t* q_indices,
                                 const float* q_values, int64_t n_queries, const sindi_search_params& prm,
                                 uint32_t* out_ids, float* out_scores, cudaStream_t stream) {
    unsigned char* base = nullptr;
    cudaError_t ce = noalloc_scratch_address(ix.device, &base);
    if (ce != cudaSuccess) {
        set_last_error(std::string("sindi_search_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce));
        return SINDI_ERR_CUDA;
    }
    const uint32_t k = prm.k;
    if (n_queries == 0) return SINDI_OK;
    if (ix.n_docs == 0) {
        pad_results_kernel<<<256, 256, 0, stream>>>(out_ids, out_scores, n_queries * (int64_t)k);
        SINDI_CUDA(cudaGetLastError());
        return SINDI_OK;
    }
    const Plan pl = make_plan(ix, prm);
    const size_t one = workspace_bytes(1, pl.cand_cap, pl.fcap, pl.top_cap);
    if (one > kNoAllocScratchBytes) {
        set_last_error("sindi_search_noalloc: one query needs " + std::to_string(one) +
                       " bytes of scratch (n_windows * 2 * min(candidates, window) * 8 + ...), more than the " +
                       std::to_string(kNoAllocScratchBytes) + "-byte static scratch area; use sindi_search");
        return SINDI_ERR_UNSUPPORTED;
    }
    const bool batched = prm.mode == SINDI_MODE_BATCHED;
    int64_t chunk = 1;
    if (batched) {
        chunk = std::min<int64_t>(n_queries, 65535);
        while (chunk > 1 && workspace_bytes(chunk, pl.cand_cap, pl.fcap, pl.top_cap) > kNoAllocScratchBytes)
            chunk = std::max<int64_t>(1, chunk / 2);
    }
    const Workspace ws = carve_workspace(base, chunk, pl.cand_cap, pl.fcap, pl.top_cap);
    // the array keeps the previous call's contents: clear the counters the kernels start from
    SINDI_CUDA(cudaMemsetAsync(base, 0, workspace_counter_bytes(chunk), stream));
    bool chained = false;
    for (int64_t q0 = 0; q0 < n_queries; q0 += chunk) {
        const uint32_t nq = (uint32_t)std::min<int64_t>(chunk, n_queries - q0);
        launch_group(ix, pl, ws, q_indptr, q_indices, q_values, q0, nq, batched, k, out_ids, out_scores, stream,
                     &chained);
    }
    ix.queries += (uint64_t)n_queries;
    return SINDI_OK;
}

// ---------------------------------------------------------------------------
// Search in a workspace the caller owns (the serving loop keeps one per slot).
// ---------------------------------------------------------------------------
size_t search_workspace_bytes(const IndexImpl& ix, const sindi_search_params& prm, int64_t queries_per_launch) {
    const Plan pl = make_plan(ix, prm);
    return workspace_bytes(std::max<int64_t>(1, queries_per_launch), pl.cand_cap, pl.fcap, pl.top_cap);
}

sindi_status search_in_workspace(const IndexImpl& ix, const int64_t* q_indptr, const int32_t* q_indices,
                                 const float* q_values, int64_t n_queries, const sindi_search_params& prm,
                                 uint32_t* out_ids, float* out_scores, cudaStream_t stream, void* ws_base,
                                 size_t ws_bytes) {
    const uint32_t k = prm.k;
    if (n_queries == 0) return SINDI_OK;
    if (ix.n_docs == 0) {
        pad_results_kernel<<<256, 256, 0, stream>>>(out_ids, out_scores, n_queries * (int64_t)k);
        SINDI_CUDA(cudaGetLastError());
        return SINDI_OK;
    }
    const Plan pl = make_plan(ix, prm);
    if (workspace_bytes(1, pl.cand_cap, pl.fcap, pl.top_cap) > ws_bytes) {
        set_last_error("workspace too small for one query");
        return SINDI_ERR_OOM;
    }
    const bool batched = prm.mode == SINDI_MODE_BATCHED;
    int64_t chunk = 1;
    if (batched) {
        chunk = std::min<int64_t>(n_queries, 65535);
        while (chunk > 1 && workspace_bytes(chunk, pl.cand_cap, pl.fcap, pl.top_cap) > ws_bytes)
            chunk = std::max<int64_t>(1, chunk / 2);
    }
    unsigned char* base = static_cast<unsigned char*>(ws_base);
    const Workspace ws = carve_workspace(base, chunk, pl.cand_cap, pl.fcap, pl.top_cap);
    SINDI_CUDA(cudaMemsetAsync(base, 0, workspace_counter_bytes(chunk), stream));
    bool chained = false;
    for (int64_t q0 = 0; q0 < n_queries; q0 += chunk) {
        const uint32_t nq = (uint32_t)std::min<int64_t>(chunk, n_queries - q0);
        launch_group(ix, pl, ws, q_indptr, q_indices, q_values, q0, nq, batched, k, out_ids, out_scores, stream,
                     &chained);
    }
    ix.queries += (uint64_t)n_queries;
    return SINDI_OK;
}

}  // namespace sindi

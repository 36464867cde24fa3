// Shared device-side definitions of the SINDI GB300 path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "checks.cuh"
#include "sindi.h"

namespace sindi {

// ---------------------------------------------------------------------------
// Limits of this build.
// ---------------------------------------------------------------------------
constexpr uint32_t kMaxWindow = 32768;       // lambda: the window's 4-byte slots must fit one block's smem
constexpr uint32_t kDefaultWindow = 8192;
constexpr int64_t kMaxRowNnz = 16384;        // longest document row the build sorts on chip
constexpr uint32_t kMaxK = 1024;
constexpr uint32_t kMaxGamma = 8192;
constexpr int kMaxQueryTerms = 4096;         // per query (the smem term table holds them)
constexpr uint32_t kMaxShards = 64;          // sindi_merge_topk: shards per merge
constexpr uint32_t kMaxShardEntries = 8192;  // sindi_merge_topk: n_shards * k_in (one block's shared memory)

// Device error word bits (sticky until sindi_check clears them).
enum : uint32_t {
    kErrQueryDim = 1u << 0,        // a query dim outside [0, d)
    kErrQueryValue = 1u << 1,      // a non-finite query value
    kErrQueryDup = 1u << 2,        // a dim repeated within one query
    kErrQueryTooLong = 1u << 3,    // more than kMaxQueryTerms terms in one query
    kErrDocIndptr = 1u << 8,       // indptr[0] != 0 or decreasing
    kErrDocDim = 1u << 9,          // a document dim outside [0, d)
    kErrDocValue = 1u << 10,       // a non-finite document value
    kErrDocDup = 1u << 11,         // a dim repeated within one document
    kErrDocTooLong = 1u << 12,     // a document row longer than kMaxRowNnz
    kErrCandOverflow = 1u << 16,   // more window candidates than the buffer holds
    kErrBounds = 1u << 17,         // checked build: an offset or id out of bounds (access skipped)
    kErrTimeout = 1u << 24,        // a bounded wait gave up
};

// Everything a search kernel reads from the index.
struct DevIndex {
    int64_t n_docs;
    int32_t dim;
    uint32_t lambda;
    uint32_t sigma;
    int32_t dtype;
    const uint32_t* seg;     // [dim * sigma + 1]
    const uint16_t* pid;     // [P] i mod lambda
    const void* pval;        // [P] float | __half | e4m3 code
    const float* scale;      // [dim]
    const float* vmax;       // [dim] largest |stored value| of list I_j (all windows)
    uint64_t pcap;           // entries of pid / pval (postings rounded up to 8)
    int64_t doc_nnz;         // entries of the unpruned documents
    int32_t nonneg;          // 1: no stored posting value is negative
    const int64_t* indptr;   // unpruned documents (reordering)
    const int32_t* indices;
    const float* values;
    uint32_t* err;           // device error word
};

// The checked build's test of one bound: records a failure in the error word
// and returns false; the normal build returns true and the test compiles away.
#ifdef __CUDACC__
__device__ __forceinline__ bool checked(bool ok, uint32_t* err) {
    if (kChecks && !ok) {
        atomicOr(err, kErrBounds);
        return false;
    }
    return true;
}
#endif

// ---------------------------------------------------------------------------
// Ordering keys. A result (score s, document id i) maps to a 64-bit key that
// grows with s and, for equal s, falls with i, so "larger key" is exactly the
// result order (score desc, id asc) and every key is distinct.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t float_order_bits(float s) {
    s = s + 0.0f;  // -0.0 -> +0.0
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(s);
#else
    memcpy(&u, &s, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float order_bits_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

__host__ __device__ __forceinline__ uint64_t result_key(float s, uint32_t id) {
    return ((uint64_t)float_order_bits(s) << 32) | (uint64_t)(0xFFFFFFFFu - id);
}

__host__ __device__ __forceinline__ uint32_t key_id(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }
__host__ __device__ __forceinline__ float key_score(uint64_t k) { return order_bits_float((uint32_t)(k >> 32)); }

// ---------------------------------------------------------------------------
// Host-side error plumbing and tracing (SINDI_TRACE=1 in the environment
// prints every host step of build and search to stderr).
// ---------------------------------------------------------------------------
void set_last_error(const std::string& msg);
bool trace_on();

#define SINDI_TRACE_MSG(...)                          \
    do {                                              \
        if (::sindi::trace_on()) {                    \
            std::fprintf(stderr, "[sindi] " __VA_ARGS__); \
            std::fprintf(stderr, "\n");               \
            std::fflush(stderr);                      \
        }                                             \
    } while (0)

struct CudaError {
    cudaError_t code;
    std::string where;
};

#define SINDI_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) throw ::sindi::CudaError{e__, std::string(#call) + " at " + \
                                                         __FILE__ ":" + std::to_string(__LINE__)}; \
    } while (0)

inline uint32_t ceil_div_u32(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// How the window scan reads a list segment I_{j,w}, which the build's posting
// order follows: a warp chunk is 256 postings of one segment; a segment of at
// least kVecMin postings is tiled on 8-aligned groups (lane l of a chunk owns
// the l-th group of 8, one posting per add instruction u = 0..7); a shorter
// segment is one chunk whose lane l owns postings s + l + 32u.
constexpr int kChunkU = 8;                 // postings per lane in one warp chunk
constexpr int kChunkLen = 32 * kChunkU;    // postings of one warp chunk (one list only)
constexpr uint32_t kVecMin = 32;           // segments this long are read with vector loads

// sindi_search_params.block_threads: 0 (default), SINDI_SCAN_PIPELINED, 256, 512 or 1024.
inline bool valid_block_threads(uint32_t b) {
    return b == 0 || b == SINDI_SCAN_PIPELINED || b == 256 || b == 512 || b == 1024;
}

// sindi_search_params.group: queries per block of the batched scan, 0 (default) .. kMaxQueryGroup.
constexpr uint32_t kMaxQueryGroup = 8;

}  // namespace sindi

// Index construction on the device: Algorithm 3 (alpha-mass of every
// document, Sec. 4.1) followed by Algorithm 1 (value-storing inverted lists,
// Sec. 3.1) with the lists cut into windows of lambda ids (Sec. 3.3.1).
//
// Pipeline (one stream):
//   validate_indptr  -> prune_rows (warp per row) [+ prune_long_rows (block per row)]
//   -> exclusive scan of kept counts -> compact -> (window, dim) counts -> scan = seg
//   -> stable radix sort of kept entries by dim (input is in document order, so
//      equal dims stay in ascending document id: the order is (dim, doc))
//   -> [E4M3 per-list scales] -> pack (uint16 window-local id + value).
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "mass.cuh"
#include "primitives.cuh"

namespace sindi {

constexpr int kPruneWarps = 4;                 // warps per block in prune_rows (32 KiB static smem)
constexpr int kPruneRowCap = 1024;             // longest row a warp sorts (smem 8 KB / warp)

__global__ void validate_indptr_kernel(const int64_t* indptr, int64_t n, uint32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && indptr[0] != 0) atomicOr(err, kErrDocIndptr);
    if (i < n && indptr[i + 1] < indptr[i]) atomicOr(err, kErrDocIndptr);
}

void launch_validate_indptr(const int64_t* indptr, int64_t n, uint32_t* err, cudaStream_t stream) {
    const int64_t threads = n + 1;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    validate_indptr_kernel<<<blocks, 256, 0, stream>>>(indptr, n, err);
    SINDI_CUDA(cudaGetLastError());
}

// One warp per document. Validates the row (dims in range, finite values, no
// duplicate dim), computes r_i = |alpha-mass(x_i)| (or, when vn > 0, r_i =
// min(vn, nnz): Vector Number Pruning) and writes the kept entries (in pi
// order) to kdim/kval at the row's own input positions.
__global__ void __launch_bounds__(kPruneWarps * 32) prune_rows_kernel(
    const int64_t* indptr, const int32_t* indices, const float* values, int64_t n, int32_t dim, double alpha,
    uint32_t vn, uint32_t* kept, int32_t* kdim, float* kval, uint32_t* long_rows, uint32_t* n_long, uint32_t* err) {
    __shared__ uint64_t sm[kPruneWarps][kPruneRowCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* s = sm[warp];
    for (int64_t i = (int64_t)blockIdx.x * kPruneWarps + warp; i < n; i += (int64_t)gridDim.x * kPruneWarps) {
        const int64_t b = indptr[i];
        const int64_t m = indptr[i + 1] - b;
        if (m > kPruneRowCap) {
            if (lane == 0) {
                if (m > kMaxRowNnz) {
                    atomicOr(err, kErrDocTooLong);
                    kept[i] = 0;
                } else {
                    uint32_t slot = atomicAdd(n_long, 1u);
                    long_rows[slot] = (uint32_t)i;
                }
            }
            continue;
        }
        const int mm = (int)m;
        int p2 = 32;
        while (p2 < mm) p2 <<= 1;
        // 1) dims: range check, and duplicates unless the row is strictly ascending
        bool bad = false, ascending = true;
        for (int t = lane; t < p2; t += 32) {
            if (t < mm) {
                int32_t j = indices[b + t];
                float v = values[b + t];
                if (j < 0 || j >= dim) { bad = true; atomicOr(err, kErrDocDim); }
                if (!isfinite(v)) { bad = true; atomicOr(err, kErrDocValue); }
                if (t + 1 < mm && indices[b + t + 1] <= j) ascending = false;
                s[t] = ((uint64_t)(uint32_t)j << 32) | (uint32_t)t;
            } else {
                s[t] = ~0ull;
            }
        }
        bad = __any_sync(kFull, bad);
        ascending = __all_sync(kFull, ascending);
        __syncwarp();
        if (bad) {
            if (lane == 0) kept[i] = 0;
            continue;
        }
        if (!ascending) {
            warp_bitonic_sort_asc(s, p2);
            bool dup = false;
            for (int t = lane + 1; t < mm; t += 32)
                if ((s[t] >> 32) == (s[t - 1] >> 32)) dup = true;
            dup = __any_sync(kFull, dup);
            __syncwarp();
            if (dup) {
                if (lane == 0) {
                    atomicOr(err, kErrDocDup);
                    kept[i] = 0;
                }
                continue;
            }
        }
        // 2) the pi order; explicit zeros are not entries (Definition 1) and sort last
        int nz = 0;
        for (int t = lane; t < p2; t += 32) {
            uint64_t key = ~0ull;
            if (t < mm) {
                float v = values[b + t];
                if (v != 0.0f) {
                    key = mass_key(indices[b + t], v);
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
        if (lane == 0) r = vn ? (nz < (int)vn ? nz : (int)vn) : alpha_mass_count(s, nz, alpha);
        r = __shfl_sync(kFull, r, 0);
        for (int t = lane; t < r; t += 32) {
            kdim[b + t] = mass_key_dim(s[t]);
            kval[b + t] = mass_key_value(s[t]);
        }
        if (lane == 0) kept[i] = (uint32_t)r;
        __syncwarp();
    }
}

// One block per long row (kPruneRowCap < m <= kMaxRowNnz); same rules.
constexpr int kLongBlock = 512;
__global__ void __launch_bounds__(kLongBlock) prune_long_rows_kernel(
    const int64_t* indptr, const int32_t* indices, const float* values, const uint32_t* rows, int32_t dim,
    double alpha, uint32_t vn, uint32_t* kept, int32_t* kdim, float* kval, uint32_t* err) {
    extern __shared__ uint64_t s[];
    __shared__ int flags[2];
    __shared__ int s_r;
    const int64_t i = rows[blockIdx.x];
    const int64_t b = indptr[i];
    const int mm = (int)(indptr[i + 1] - b);
    int p2 = 32;
    while (p2 < mm) p2 <<= 1;
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; }
    __syncthreads();
    for (int t = threadIdx.x; t < p2; t += kLongBlock) {
        if (t < mm) {
            int32_t j = indices[b + t];
            float v = values[b + t];
            if (j < 0 || j >= dim) { flags[0] = 1; atomicOr(err, kErrDocDim); }
            if (!isfinite(v)) { flags[0] = 1; atomicOr(err, kErrDocValue); }
            s[t] = ((uint64_t)(uint32_t)j << 32) | (uint32_t)t;
        } else {
            s[t] = ~0ull;
        }
    }
    __syncthreads();
    if (flags[0]) {
        if (threadIdx.x == 0) kept[i] = 0;
        return;
    }
    // ascending sort of dims: reuse the descending sort on inverted keys
    for (int t = threadIdx.x; t < p2; t += kLongBlock) s[t] = ~s[t];
    __syncthreads();
    block_bitonic_sort_desc<kLongBlock>(s, p2);
    for (int t = threadIdx.x + 1; t < mm; t += kLongBlock)
        if (((~s[t]) >> 32) == ((~s[t - 1]) >> 32)) flags[1] = 1;
    __syncthreads();
    if (flags[1]) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrDocDup);
            kept[i] = 0;
        }
        return;
    }
    __shared__ int s_nz;
    if (threadIdx.x == 0) s_nz = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < p2; t += kLongBlock) {
        uint64_t key = ~0ull;
        if (t < mm) {
            float v = values[b + t];
            if (v != 0.0f) {
                key = mass_key(indices[b + t], v);
                atomicAdd(&s_nz, 1);
            }
        }
        s[t] = ~key;  // descending sort of inverted keys = ascending mass_key
    }
    __syncthreads();
    block_bitonic_sort_desc<kLongBlock>(s, p2);
    for (int t = threadIdx.x; t < p2; t += kLongBlock) s[t] = ~s[t];
    __syncthreads();
    if (threadIdx.x == 0) s_r = vn ? (s_nz < (int)vn ? s_nz : (int)vn) : alpha_mass_count(s, s_nz, alpha);
    __syncthreads();
    const int r = s_r;
    for (int t = threadIdx.x; t < r; t += kLongBlock) {
        kdim[b + t] = mass_key_dim(s[t]);
        kval[b + t] = mass_key_value(s[t]);
    }
    if (threadIdx.x == 0) kept[i] = (uint32_t)r;
}

// Kept entries of every row -> compact arrays in document order.
__global__ void compact_kernel(const int64_t* indptr, const int64_t* kept_off, const int32_t* kdim, const float* kval,
                               int64_t n, uint32_t* sdim, uint32_t* sdoc, uint32_t* sval) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t b = indptr[i], o = kept_off[i], r = kept_off[i + 1] - o;
        for (int64_t t = lane; t < r; t += 32) {
            sdim[o + t] = (uint32_t)kdim[b + t];
            sdoc[o + t] = (uint32_t)i;
            sval[o + t] = __float_as_uint(kval[b + t]);
        }
    }
}

// Count postings of every list I_{j,w}: cnt[j * sigma + w].
__global__ void list_count_kernel(const uint32_t* sdim, const uint32_t* sdoc, int64_t P, uint32_t lambda,
                                  uint32_t sigma, uint32_t* cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[(uint64_t)sdim[p] * sigma + sdoc[p] / lambda], 1u);
}

// Per-list E4M3 scale: max |x| over the list I_j (all windows) / 448.
__global__ void list_scale_kernel(const uint32_t* seg, const uint32_t* sval, int32_t dim, uint32_t sigma,
                                  float* scale) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < dim; j += warps) {
        const uint32_t lo = seg[(uint64_t)j * sigma], hi = seg[(uint64_t)(j + 1) * sigma];
        float amax = 0.0f;
        for (uint32_t p = lo + lane; p < hi; p += 32) amax = fmaxf(amax, fabsf(__uint_as_float(sval[p])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
        if (lane == 0) {
            float sc = __fdiv_rn(amax, 448.0f);
            scale[j] = sc > 0.0f ? sc : 1.0f;
        }
    }
}

// Window-local ids and stored values.
template <int DT>
__global__ void pack_kernel(const uint32_t* sdim, const uint32_t* sdoc, const uint32_t* sval, int64_t P,
                            uint32_t lambda, const float* scale, uint16_t* pid, void* pval) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        pid[p] = (uint16_t)(sdoc[p] % lambda);
        float v = __uint_as_float(sval[p]);
        if (DT == SINDI_F32) {
            static_cast<float*>(pval)[p] = v;
        } else if (DT == SINDI_F16) {
            static_cast<__half*>(pval)[p] = __float2half_rn(v);
        } else {
            float ratio = __fdiv_rn(v, scale[sdim[p]]);
            static_cast<__nv_fp8_storage_t*>(pval)[p] = __nv_cvt_float_to_fp8(ratio, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// List Pruning (Sec. 4.1): every list I_j keeps its `lp` entries of largest
// |x|, equal |x| by lower document id. Postings arrive in (dim, doc) order;
// a stable sort by (dim, |x| descending) then ranks every entry in its list.
// Sort keys: 0x7FFFFFFF - |x| bits (ascending = |x| descending), and the
// entry's position.
__global__ void lp_keys_kernel(const uint32_t* sval, int64_t P, uint32_t* inv, uint32_t* pos) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        inv[p] = 0x7FFFFFFFu - (sval[p] & 0x7FFFFFFFu);
        pos[p] = (uint32_t)p;
    }
}

// Entry t of the (dim, |x| desc, doc asc) order has rank t - start(list) in
// its list; the first lp survive. A dropped entry leaves its document's count.
__global__ void lp_mark_kernel(const uint32_t* dim_sorted, const uint32_t* pos_sorted, int64_t P, const uint32_t* seg,
                               uint32_t sigma, uint32_t lp, const uint32_t* sdoc, uint32_t* keep, uint32_t* kept) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = dim_sorted[t];
        const uint32_t p = pos_sorted[t];
        const bool k = (uint64_t)t - seg[(uint64_t)j * sigma] < lp;
        keep[p] = k ? 1u : 0u;
        if (!k) atomicSub(&kept[sdoc[p]], 1u);
    }
}

// Entries with keep[p] = 1 move to off[p] (exclusive scan of keep); the
// (dim, doc) order is kept.
__global__ void lp_compact_kernel(const uint32_t* keep, const uint32_t* off, int64_t P, const uint32_t* sdim,
                                  const uint32_t* sdoc, const uint32_t* sval, uint32_t* odim, uint32_t* odoc,
                                  uint32_t* oval) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        if (keep[p]) {
            const uint32_t o = off[p];
            odim[o] = sdim[p];
            odoc[o] = sdoc[p];
            oval[o] = sval[p];
        }
    }
}

// Posting order inside every list segment I_{j,w}, for the window scan's
// shared-memory scatter-add: the 32 postings one add instruction of a warp
// takes should sit in 32 different shared-memory banks (window slot mod 32),
// which makes the shared-memory atomicAdd conflict-free. One warp per segment:
//   1. every posting gets its bank b and a rank r among the segment's
//      postings of bank b; ordering the postings by (r, b) visits the banks
//      round robin, so any 32 consecutive ones hold 32 banks while every bank
//      still has postings;
//   2. that order is laid out over the positions of the segment in the order
//      the scan's add instructions visit them (see kVecMin), so each
//      instruction takes 32 consecutive ones.
// Any order of a segment gives the same scores up to FP32 rounding; this one
// only changes which bank each add of an instruction meets.
// scratch: uint32[P]; (sdoc, sval) in, (odoc, oval) out.
constexpr int kOrderWarps = 8;
__global__ void __launch_bounds__(kOrderWarps * 32) bank_order_kernel(const uint32_t* seg, int64_t S,
                                                                     const uint32_t* sdoc, const uint32_t* sval,
                                                                     uint32_t lambda, uint32_t* scratch,
                                                                     uint32_t* odoc, uint32_t* oval) {
    __shared__ uint32_t cnt[kOrderWarps][32];
    __shared__ uint32_t rnk[kOrderWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * kOrderWarps;
    for (int64_t sg = (int64_t)blockIdx.x * kOrderWarps + warp; sg < S; sg += warps) {
        const uint32_t s = seg[sg], e = seg[sg + 1], L = e - s;
        if (L <= 32) {
            // one add instruction takes the whole segment: nothing to gain
            if (lane < (int)L) {
                odoc[s + lane] = sdoc[s + lane];
                oval[s + lane] = sval[s + lane];
            }
            continue;
        }
        cnt[warp][lane] = 0;
        rnk[warp][lane] = 0;
        __syncwarp();
        for (uint32_t i = lane; i < L; i += 32) atomicAdd(&cnt[warp][(sdoc[s + i] % lambda) & 31u], 1u);
        __syncwarp();
        for (uint32_t i0 = 0; i0 < L; i0 += 32) {
            // rank = earlier postings of the same bank, in segment order (deterministic)
            const uint32_t i = i0 + (uint32_t)lane;
            const bool ok = i < L;
            const uint32_t b = ok ? (sdoc[s + i] % lambda) & 31u : 32u + (uint32_t)lane;
            const unsigned peers = __match_any_sync(kFull, b);
            const uint32_t r = ok ? rnk[warp][b] + (uint32_t)__popc(peers & lt) : 0u;
            __syncwarp();
            if (ok && (peers & lt) == 0) rnk[warp][b] += (uint32_t)__popc(peers);
            __syncwarp();
            if (ok) {
                // position of (r, b) in the (rank, bank) order
                uint32_t q = 0;
                for (uint32_t bb = 0; bb < 32; bb++) {
                    const uint32_t c = cnt[warp][bb];
                    q += c < r ? c : r;
                    q += (bb < b && c > r) ? 1u : 0u;
                }
                scratch[s + q] = s + i;
            }
        }
        __syncwarp();
        // the positions in the order the scan's add instructions take them
        uint32_t run = 0;
        if (L >= kVecMin) {
            const uint32_t g0 = s & ~7u, e8 = (e + 7u) & ~7u;
            for (uint32_t base = g0; base < e8; base += (uint32_t)kChunkLen) {
                for (int u = 0; u < kChunkU; u++) {
                    const uint32_t p = base + 8u * (uint32_t)lane + (uint32_t)u;
                    const bool ok = p >= s && p < e;
                    const unsigned bal = __ballot_sync(kFull, ok);
                    if (ok) {
                        const uint32_t src = scratch[s + run + (uint32_t)__popc(bal & lt)];
                        odoc[p] = sdoc[src];
                        oval[p] = sval[src];
                    }
                    run += (uint32_t)__popc(bal);
                }
            }
        } else {
            for (uint32_t u = 0; u * 32 < L; u++) {
                const uint32_t p = s + 32u * u + (uint32_t)lane;
                const bool ok = p < e;
                const unsigned bal = __ballot_sync(kFull, ok);
                if (ok) {
                    const uint32_t src = scratch[s + run + (uint32_t)__popc(bal & lt)];
                    odoc[p] = sdoc[src];
                    oval[p] = sval[src];
                }
                run += (uint32_t)__popc(bal);
            }
        }
        __syncwarp();
    }
}

__global__ void fill_u32_kernel(float* p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

static int grid_for(int64_t n, int block, int cap = 152 * 16) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

static uint32_t read_u32(const uint32_t* d, cudaStream_t s) {
    uint32_t h = 0;
    SINDI_CUDA(cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s));
    SINDI_CUDA(cudaStreamSynchronize(s));
    return h;
}

static int64_t read_i64(const int64_t* d, cudaStream_t s) {
    int64_t h = 0;
    SINDI_CUDA(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s));
    SINDI_CUDA(cudaStreamSynchronize(s));
    return h;
}

static std::string doc_error_text(uint32_t e) {
    std::string m;
    if (e & kErrDocIndptr) m += "indptr[0] != 0 or decreasing; ";
    if (e & kErrDocDim) m += "a document dim outside [0, dim); ";
    if (e & kErrDocValue) m += "a non-finite document value; ";
    if (e & kErrDocDup) m += "a dim repeated within a document; ";
    if (e & kErrDocTooLong) m += "a document row longer than 16384 entries; ";
    return m;
}

// Builds the lists of `ix`. Its documents are on the device and indptr has
// been validated (indptr[0] = 0, non-decreasing). Allocates the index arrays
// (seg, pid, pval, scale, kept) from the library pool; they belong to `ix`.
// Returns SINDI_OK or an error status with the message set.
sindi_status build_lists(IndexImpl& ix, cudaStream_t stream) {
    Pool P{ix.pool, stream};
    const int64_t n = ix.n_docs;
    const int32_t d = ix.dim;
    const uint32_t lambda = ix.lambda;
    const uint32_t sigma = ix.sigma;
    uint32_t e = 0;
    // the document stage: Vector Number Pruning keeps vn entries per row,
    // otherwise alpha-mass (alpha = 1 keeps every entry)
    const uint32_t vn = ix.prune == SINDI_PRUNE_VECTOR_NUMBER ? ix.prune_n : 0u;
    const uint32_t lp = (ix.prune == SINDI_PRUNE_LIST || ix.prune == SINDI_PRUNE_MASS_LIST) ? ix.prune_n : 0u;
    SINDI_TRACE_MSG("build_lists: enter");
    ix.kept = P.alloc<uint32_t>(n > 0 ? n : 1);
    ix.scale = P.alloc<float>(d);
    ix.seg = P.alloc<uint32_t>((size_t)d * sigma + 1);
    const int64_t nnz = ix.doc_nnz;
    uint32_t* kept = ix.kept;
    int32_t* kdim = P.alloc<int32_t>(nnz);
    float* kval = P.alloc<float>(nnz);
    uint32_t* long_rows = P.alloc<uint32_t>(n > 0 ? n : 1);
    uint32_t* n_long = P.alloc<uint32_t>(1);
    SINDI_CUDA(cudaMemsetAsync(n_long, 0, 4, stream));
    SINDI_TRACE_MSG("build_lists: launching prune_rows");
    if (n > 0) {
        prune_rows_kernel<<<grid_for(n, kPruneWarps, 152 * 32), kPruneWarps * 32, 0, stream>>>(
            ix.indptr, ix.indices, ix.values, n, d, ix.alpha, vn, kept, kdim, kval, long_rows, n_long, ix.err);
        SINDI_CUDA(cudaGetLastError());
    }
    uint32_t nl = n > 0 ? read_u32(n_long, stream) : 0;
    if (nl > 0) {
        size_t sm = (size_t)kMaxRowNnz * sizeof(uint64_t);
        SINDI_CUDA(cudaFuncSetAttribute(prune_long_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        prune_long_rows_kernel<<<nl, kLongBlock, sm, stream>>>(ix.indptr, ix.indices, ix.values, long_rows, d,
                                                                ix.alpha, vn, kept, kdim, kval, ix.err);
        SINDI_CUDA(cudaGetLastError());
    }
    e = read_u32(ix.err, stream);
    if (e) {
        P.free(kdim); P.free(kval); P.free(long_rows); P.free(n_long);
        set_last_error("malformed documents: " + doc_error_text(e));
        return (e & kErrDocTooLong) && !(e & ~kErrDocTooLong) ? SINDI_ERR_UNSUPPORTED : SINDI_ERR_INVALID_DATA;
    }
    P.free(long_rows);
    P.free(n_long);

    SINDI_TRACE_MSG("build_lists: pruning done");
    // --- compact kept entries (document order)
    int64_t* kept_off = P.alloc<int64_t>(n + 1);
    exclusive_scan<uint32_t, int64_t>(kept, kept_off, n, P);
    const int64_t Pn0 = read_i64(kept_off + n, stream);
    if (Pn0 > kMaxPostings) {
        P.free(kdim); P.free(kval); P.free(kept_off);
        set_last_error("more than 2^32 - 4096 kept entries");
        return SINDI_ERR_UNSUPPORTED;
    }
    int64_t Pn = Pn0;
    uint32_t* sdim = P.alloc<uint32_t>(Pn);
    uint32_t* sdoc = P.alloc<uint32_t>(Pn);
    uint32_t* sval = P.alloc<uint32_t>(Pn);
    if (n > 0) {
        compact_kernel<<<grid_for(n, 8, 152 * 32), 256, 0, stream>>>(ix.indptr, kept_off, kdim, kval, n, sdim, sdoc,
                                                                     sval);
        SINDI_CUDA(cudaGetLastError());
    }
    P.free(kdim);
    P.free(kval);
    P.free(kept_off);

    SINDI_TRACE_MSG("build_lists: compacted %lld kept entries", (long long)Pn);
    // --- offsets of every list I_{j,w}
    const int64_t S = (int64_t)d * sigma;
    uint32_t* cnt = P.alloc<uint32_t>(S > 0 ? S : 1);
    SINDI_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(S > 0 ? S : 1), stream));
    if (Pn > 0) {
        list_count_kernel<<<grid_for(Pn, 256), 256, 0, stream>>>(sdim, sdoc, Pn, lambda, sigma, cnt);
        SINDI_CUDA(cudaGetLastError());
    }
    exclusive_scan<uint32_t, uint32_t>(cnt, ix.seg, S, P);
    P.free(cnt);

    SINDI_TRACE_MSG("build_lists: list offsets done");
    // --- stable sort by dim: (dim, doc) order
    {
        uint32_t* kb = P.alloc<uint32_t>(Pn);
        uint32_t* db = P.alloc<uint32_t>(Pn);
        uint32_t* vb = P.alloc<uint32_t>(Pn);
        int bits = 0;
        while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)d) bits++;
        radix_sort_triples(sdim, sdoc, sval, kb, db, vb, Pn, bits, P);
        P.free(kb); P.free(db); P.free(vb);
    }

    SINDI_TRACE_MSG("build_lists: sort done");
    if (lp > 0 && Pn > 0) {
        // --- List Pruning on the lists built so far, then their offsets again
        uint32_t* inv = P.alloc<uint32_t>(Pn);
        uint32_t* dcp = P.alloc<uint32_t>(Pn);
        uint32_t* pos = P.alloc<uint32_t>(Pn);
        uint32_t* kb = P.alloc<uint32_t>(Pn);
        uint32_t* db = P.alloc<uint32_t>(Pn);
        uint32_t* vb = P.alloc<uint32_t>(Pn);
        lp_keys_kernel<<<grid_for(Pn, 256), 256, 0, stream>>>(sval, Pn, inv, pos);
        SINDI_CUDA(cudaGetLastError());
        SINDI_CUDA(cudaMemcpyAsync(dcp, sdim, sizeof(uint32_t) * (size_t)Pn, cudaMemcpyDeviceToDevice, stream));
        radix_sort_triples(inv, dcp, pos, kb, db, vb, Pn, 31, P);  // by |x| descending (stable)
        int bits = 0;
        while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)d) bits++;
        radix_sort_triples(dcp, inv, pos, kb, db, vb, Pn, bits, P);  // then by dim (stable)
        uint32_t* keep = kb;  // scratch reuse
        uint32_t* off = P.alloc<uint32_t>(Pn + 1);
        lp_mark_kernel<<<grid_for(Pn, 256), 256, 0, stream>>>(dcp, pos, Pn, ix.seg, sigma, lp, sdoc, keep, kept);
        SINDI_CUDA(cudaGetLastError());
        exclusive_scan<uint32_t, uint32_t>(keep, off, Pn, P);
        const int64_t Pk = read_u32(off + Pn, stream);
        uint32_t* odim = P.alloc<uint32_t>(Pk > 0 ? Pk : 1);
        uint32_t* odoc = P.alloc<uint32_t>(Pk > 0 ? Pk : 1);
        uint32_t* oval = P.alloc<uint32_t>(Pk > 0 ? Pk : 1);
        lp_compact_kernel<<<grid_for(Pn, 256), 256, 0, stream>>>(keep, off, Pn, sdim, sdoc, sval, odim, odoc, oval);
        SINDI_CUDA(cudaGetLastError());
        P.free(inv); P.free(dcp); P.free(pos); P.free(kb); P.free(db); P.free(vb); P.free(off);
        P.free(sdim); P.free(sdoc); P.free(sval);
        sdim = odim;
        sdoc = odoc;
        sval = oval;
        Pn = Pk;
        uint32_t* cnt2 = P.alloc<uint32_t>(S > 0 ? S : 1);
        SINDI_CUDA(cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * (size_t)(S > 0 ? S : 1), stream));
        if (Pn > 0) {
            list_count_kernel<<<grid_for(Pn, 256), 256, 0, stream>>>(sdim, sdoc, Pn, lambda, sigma, cnt2);
            SINDI_CUDA(cudaGetLastError());
        }
        exclusive_scan<uint32_t, uint32_t>(cnt2, ix.seg, S, P);
        P.free(cnt2);
        SINDI_TRACE_MSG("build_lists: list pruning kept %lld postings", (long long)Pn);
    }
    ix.postings = Pn;
    // posting arrays padded to a multiple of 8 entries: the scan reads aligned groups of 8
    const int64_t Pp = (Pn + 7) & ~(int64_t)7;
    ix.pid = P.alloc<uint16_t>(Pp);
    ix.pval = P.alloc<uint8_t>((size_t)Pp * ix.value_bytes());
    if ((reinterpret_cast<uintptr_t>(ix.pid) | reinterpret_cast<uintptr_t>(ix.pval)) & 15)
        throw CudaError{cudaErrorMisalignedAddress, "posting arrays are not 16-byte aligned"};
    if (Pp > Pn) {
        SINDI_CUDA(cudaMemsetAsync(ix.pid + Pn, 0, sizeof(uint16_t) * (size_t)(Pp - Pn), stream));
        SINDI_CUDA(cudaMemsetAsync(static_cast<uint8_t*>(ix.pval) + (size_t)Pn * ix.value_bytes(), 0,
                                   (size_t)(Pp - Pn) * ix.value_bytes(), stream));
    }
    // --- values and window-local ids
    if (ix.dtype == SINDI_F8E4M3) {
        if (d > 0) {
            list_scale_kernel<<<grid_for(d, 8, 152 * 32), 256, 0, stream>>>(ix.seg, sval, d, sigma, ix.scale);
            SINDI_CUDA(cudaGetLastError());
        }
    } else if (d > 0) {
        fill_u32_kernel<<<grid_for(d, 256), 256, 0, stream>>>(ix.scale, d, 1.0f);
        SINDI_CUDA(cudaGetLastError());
    }
    if (Pn > 0) {
        // bank-aware order inside every segment (the scan's scatter-add)
        uint32_t* scratch = P.alloc<uint32_t>(Pn);
        uint32_t* odoc = P.alloc<uint32_t>(Pn);
        uint32_t* oval = P.alloc<uint32_t>(Pn);
        bank_order_kernel<<<grid_for(S, kOrderWarps, 152 * 16), kOrderWarps * 32, 0, stream>>>(
            ix.seg, S, sdoc, sval, lambda, scratch, odoc, oval);
        SINDI_CUDA(cudaGetLastError());
        P.free(scratch);
        P.free(sdoc);
        P.free(sval);
        sdoc = odoc;
        sval = oval;
        if (ix.dtype == SINDI_F32)
            pack_kernel<SINDI_F32><<<grid_for(Pn, 256), 256, 0, stream>>>(sdim, sdoc, sval, Pn, lambda, ix.scale,
                                                                          ix.pid, ix.pval);
        else if (ix.dtype == SINDI_F16)
            pack_kernel<SINDI_F16><<<grid_for(Pn, 256), 256, 0, stream>>>(sdim, sdoc, sval, Pn, lambda, ix.scale,
                                                                          ix.pid, ix.pval);
        else
            pack_kernel<SINDI_F8E4M3><<<grid_for(Pn, 256), 256, 0, stream>>>(sdim, sdoc, sval, Pn, lambda,
                                                                             ix.scale, ix.pid, ix.pval);
        SINDI_CUDA(cudaGetLastError());
    }
    P.free(sdim);
    P.free(sdoc);
    P.free(sval);
    list_value_bounds(ix, stream);
    ix.nonneg = postings_nonnegative(ix, stream);  // synchronises the stream
    return SINDI_OK;
}

// Sets *flag when a stored posting value has its sign bit set (FP32, binary16
// or E4M3 alike: the top bit of the stored word).
__global__ void negative_values_kernel(const unsigned char* pval, int64_t P, int vbytes, uint32_t* flag) {
    bool neg = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P && !neg;
         p += (int64_t)gridDim.x * blockDim.x)
        neg = (pval[p * vbytes + vbytes - 1] & 0x80u) != 0;  // little-endian: the sign is in the last byte
    if (__syncthreads_or(neg) && threadIdx.x == 0) atomicOr(flag, 1u);
}

bool postings_nonnegative(const IndexImpl& ix, cudaStream_t stream) {
    Pool P{ix.pool, stream};
    uint32_t* flag = P.alloc<uint32_t>(1);
    SINDI_CUDA(cudaMemsetAsync(flag, 0, 4, stream));
    if (ix.postings > 0) {
        negative_values_kernel<<<grid_for(ix.postings, 256), 256, 0, stream>>>(
            static_cast<const unsigned char*>(ix.pval), ix.postings, (int)ix.value_bytes(), flag);
        SINDI_CUDA(cudaGetLastError());
    }
    uint32_t h = 0;
    SINDI_CUDA(cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, stream));
    P.free(flag);
    SINDI_CUDA(cudaStreamSynchronize(stream));
    return h == 0;
}

}  // namespace sindi

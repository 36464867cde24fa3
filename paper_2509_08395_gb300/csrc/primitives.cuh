// Device-wide and block-wide primitives of the SINDI GB300 path:
//   - exclusive prefix sum over an array (three-phase, recursive on tile sums);
//   - stable LSD radix sort of (key, doc, value) triples by an unsigned key;
//   - block-level radix selection of the g largest distinct 64-bit keys;
//   - block-level bitonic sort of 64-bit keys in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sindi {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Stream-ordered scratch memory from the library pool.
// ---------------------------------------------------------------------------
struct Pool {
    cudaMemPool_t pool;
    cudaStream_t stream;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        SINDI_CUDA(cudaMallocFromPoolAsync(&p, bytes, pool, stream));
        return static_cast<T*>(p);
    }
    void free(void* p) {
        if (p) SINDI_CUDA(cudaFreeAsync(p, stream));
    }
};

cudaMemPool_t library_pool(int device);

// ---------------------------------------------------------------------------
// Exclusive scan: out[0] = 0, out[i] = in[0] + ... + in[i-1], out[n] = total.
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = (int64_t)kScanBlock * kScanItems;

// Who cooperates in a collective below, and how they synchronise: the whole
// block (__syncthreads), or a warp-aligned group of NT threads starting at
// thread FIRST that meets at hardware barrier BAR (bar.sync; barrier 0 is the
// block's own). tid() is the thread's index inside the group.
template <int NT>
struct SyncBlock {
    static constexpr int kThreads = NT;
    __device__ static __forceinline__ void sync() { __syncthreads(); }
    __device__ static __forceinline__ int tid() { return (int)threadIdx.x; }
};

template <int BAR, int NT, int FIRST>
struct SyncGroup {
    static constexpr int kThreads = NT;
    static_assert(NT % 32 == 0 && FIRST % 32 == 0 && BAR > 0 && BAR < 16, "warp-aligned group, barriers 1..15");
    __device__ static __forceinline__ void sync() { asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory"); }
    __device__ static __forceinline__ int tid() { return (int)threadIdx.x - FIRST; }
};

// Group-wide exclusive sum of one value per thread; *total gets the group sum.
// smem: [S::kThreads / 32 + 1] elements. Group size <= 1024.
template <typename T, typename S>
__device__ __forceinline__ T group_exclusive_sum(T v, T* total, T* smem) {
    constexpr int W = S::kThreads / 32;
    const int lane = S::tid() & 31, warp = S::tid() >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    S::sync();
    if (warp == 0) {
        T w = lane < W ? smem[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < W) smem[lane] = w;  // inclusive warp totals
        if (lane == W - 1) smem[W] = w;
    }
    S::sync();
    T warp_excl = warp > 0 ? smem[warp - 1] : T(0);
    *total = smem[W];
    T r = warp_excl + x - v;
    S::sync();
    return r;
}

// The same over the whole block of BLOCK threads.
template <typename T, int BLOCK = kScanBlock>
__device__ __forceinline__ T block_exclusive_sum(T v, T* total, T* smem) {
    return group_exclusive_sum<T, SyncBlock<BLOCK>>(v, total, smem);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanBlock) scan_tile_sums_kernel(const TI* in, int64_t n, TO* sums) {
    __shared__ TO sm[kScanBlock / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    TO acc = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        int64_t i = base + t;
        if (i < n) acc += (TO)in[i];
    }
    TO total;
    (void)block_exclusive_sum<TO>(acc, &total, sm);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanBlock) scan_tile_apply_kernel(const TI* in, int64_t n, const TO* tile_off,
                                                                   TO* out) {
    __shared__ TO sm[kScanBlock / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    TI v[kScanItems];
    TO acc = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        int64_t i = base + t;
        v[t] = i < n ? in[i] : TI(0);
        acc += (TO)v[t];
    }
    TO total;
    TO run = block_exclusive_sum<TO>(acc, &total, sm) + tile_off[blockIdx.x];
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        int64_t i = base + t;
        if (i < n) out[i] = run;
        run += (TO)v[t];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanBlock - 1) out[n] = run;
}

// out must hold n + 1 elements.
template <typename TI, typename TO>
void exclusive_scan(const TI* in, TO* out, int64_t n, Pool& P) {
    if (n == 0) {
        SINDI_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), P.stream));
        return;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    TO* offs = P.alloc<TO>(tiles + 1);
    TO* sums = nullptr;
    if (tiles == 1) {
        // one tile: its offset is zero (base case of the recursion on tile sums)
        SINDI_CUDA(cudaMemsetAsync(offs, 0, sizeof(TO) * 2, P.stream));
    } else {
        sums = P.alloc<TO>(tiles);
        scan_tile_sums_kernel<TI, TO><<<(unsigned)tiles, kScanBlock, 0, P.stream>>>(in, n, sums);
        SINDI_CUDA(cudaGetLastError());
        exclusive_scan<TO, TO>(sums, offs, tiles, P);
    }
    scan_tile_apply_kernel<TI, TO><<<(unsigned)tiles, kScanBlock, 0, P.stream>>>(in, n, offs, out);
    SINDI_CUDA(cudaGetLastError());
    P.free(sums);
    P.free(offs);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort by key (8-bit digits), carrying doc (u32) and value (u32
// bit pattern). Each tile of kSortTile items is split into per-warp contiguous
// runs; within a run items are ranked in order with __match_any_sync, so the
// scatter keeps the input order of equal digits.
// ---------------------------------------------------------------------------
constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortRounds = 16;                              // rounds of 32 items per warp
constexpr int kSortTile = kSortBlock * kSortRounds;          // 4096 items per tile

static __global__ void __launch_bounds__(kSortBlock) radix_hist_kernel(const uint32_t* key, int64_t n, int shift,
                                                              uint32_t* tile_hist, uint32_t n_tiles) {
    __shared__ uint32_t h[256];
    for (int b = threadIdx.x; b < 256; b += kSortBlock) h[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int t = threadIdx.x; t < kSortTile; t += kSortBlock) {
        int64_t i = base + t;
        int dig = i < n ? (int)((key[i] >> shift) & 255u) : -1;
        unsigned peers = __match_any_sync(kFull, dig);
        if (dig >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[dig], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += kSortBlock) tile_hist[(int64_t)b * n_tiles + blockIdx.x] = h[b];
}

static __global__ void __launch_bounds__(kSortBlock) radix_scatter_kernel(
    const uint32_t* key, const uint32_t* doc, const uint32_t* val, int64_t n, int shift, const uint32_t* tile_off,
    uint32_t n_tiles, uint32_t* key_out, uint32_t* doc_out, uint32_t* val_out) {
    __shared__ uint32_t wcount[kSortWarps][256];
    __shared__ uint32_t base_of[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = lane; b < 256; b += 32) wcount[warp][b] = 0;
    for (int b = threadIdx.x; b < 256; b += kSortBlock) base_of[b] = tile_off[(int64_t)b * n_tiles + blockIdx.x];
    __syncwarp();
    const int64_t run = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortRounds);
    const unsigned lt = (1u << lane) - 1u;
    // pass 1: per-warp digit counts
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = run + r * 32 + lane;
        int dig = i < n ? (int)((key[i] >> shift) & 255u) : -1;
        unsigned peers = __match_any_sync(kFull, dig);
        if (dig >= 0 && lane == __ffs(peers) - 1) wcount[warp][dig] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for every digit
    for (int b = threadIdx.x; b < 256; b += kSortBlock) {
        uint32_t acc = base_of[b];
        for (int w = 0; w < kSortWarps; w++) {
            uint32_t c = wcount[w][b];
            wcount[w][b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    // pass 2: ranked scatter
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = run + r * 32 + lane;
        bool ok = i < n;
        uint32_t k = ok ? key[i] : 0u;
        int dig = ok ? (int)((k >> shift) & 255u) : -1;
        unsigned peers = __match_any_sync(kFull, dig);
        uint32_t pos = 0;
        if (ok) pos = wcount[warp][dig] + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcount[warp][dig] += (uint32_t)__popc(peers);
        __syncwarp();
        if (ok) {
            key_out[pos] = k;
            doc_out[pos] = doc[i];
            val_out[pos] = val[i];
        }
    }
}

// Sorts n triples by key[0..n) (keys < 2^key_bits). Buffers *_a hold the input
// and receive the sorted output; *_b are scratch of the same size.
inline void radix_sort_triples(uint32_t* key_a, uint32_t* doc_a, uint32_t* val_a, uint32_t* key_b, uint32_t* doc_b,
                               uint32_t* val_b, int64_t n, int key_bits, Pool& P) {
    if (n <= 1 || key_bits <= 0) return;
    const uint32_t n_tiles = ceil_div_u32((uint64_t)n, kSortTile);
    uint32_t* hist = P.alloc<uint32_t>((size_t)256 * n_tiles);
    uint32_t* off = P.alloc<uint32_t>((size_t)256 * n_tiles + 1);
    int passes = (key_bits + 7) / 8;
    uint32_t *ka = key_a, *da = doc_a, *va = val_a, *kb = key_b, *db = doc_b, *vb = val_b;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        radix_hist_kernel<<<n_tiles, kSortBlock, 0, P.stream>>>(ka, n, shift, hist, n_tiles);
        SINDI_CUDA(cudaGetLastError());
        exclusive_scan<uint32_t, uint32_t>(hist, off, (int64_t)256 * n_tiles, P);
        radix_scatter_kernel<<<n_tiles, kSortBlock, 0, P.stream>>>(ka, da, va, n, shift, off, n_tiles, kb, db, vb);
        SINDI_CUDA(cudaGetLastError());
        uint32_t* t;
        t = ka; ka = kb; kb = t;
        t = da; da = db; db = t;
        t = va; va = vb; vb = t;
    }
    if (ka != key_a) {
        SINDI_CUDA(cudaMemcpyAsync(key_a, ka, n * 4, cudaMemcpyDeviceToDevice, P.stream));
        SINDI_CUDA(cudaMemcpyAsync(doc_a, da, n * 4, cudaMemcpyDeviceToDevice, P.stream));
        SINDI_CUDA(cudaMemcpyAsync(val_a, va, n * 4, cudaMemcpyDeviceToDevice, P.stream));
    }
    P.free(hist);
    P.free(off);
}

// ---------------------------------------------------------------------------
// Block radix selection. Given n distinct 64-bit keys (key_of(i), i < n) and
// 1 <= g <= n, returns T such that exactly g keys are >= T. The leading bits
// all keys share are found first (one max/min reduction) and skipped; 8-bit
// digits then go from the highest differing bit down, and a digit bucket that
// holds exactly the remainder ends the search early.
//   hist: shared uint32[256]; st: shared uint32[4].
// Every thread of the group must call it (it synchronises).
// ---------------------------------------------------------------------------
template <typename S, typename KeyOf>
__device__ uint64_t group_select_threshold(const KeyOf& key_of, int n, int g, uint32_t* hist, uint32_t* st) {
    constexpr int BLOCK = S::kThreads;
    constexpr int W = BLOCK / 32;
    static_assert(2 * W * 2 <= 256, "scratch for the reduction lives in hist");
    const int tid = S::tid();
    const int lane = tid & 31, warp = tid >> 5;
    // shared prefix: highest bit where the largest and smallest key differ
    uint64_t mx = 0, mn = ~0ull;
    for (int i = tid; i < n; i += BLOCK) {
        const uint64_t k = key_of(i);
        mx = k > mx ? k : mx;
        mn = k < mn ? k : mn;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(kFull, mx, o), b = __shfl_xor_sync(kFull, mn, o);
        mx = a > mx ? a : mx;
        mn = b < mn ? b : mn;
    }
    uint64_t* red64 = reinterpret_cast<uint64_t*>(hist);
    S::sync();  // hist may still be read by the caller's previous use
    if (lane == 0) {
        red64[warp] = mx;
        red64[W + warp] = mn;
    }
    S::sync();
    if (tid == 0) {
        uint64_t a = 0, b = ~0ull;
        for (int i = 0; i < W; i++) {
            a = red64[i] > a ? red64[i] : a;
            b = red64[W + i] < b ? red64[W + i] : b;
        }
        red64[0] = a;
        red64[1] = b;
    }
    S::sync();
    const uint64_t kmax = red64[0], diff = kmax ^ red64[1];
    S::sync();
    if (diff == 0) return kmax;  // a single key
    const int hb = 63 - __clzll((long long)diff);
    uint64_t mask = hb >= 63 ? 0ull : ~((2ull << hb) - 1ull);  // bits every key shares
    uint64_t prefix = kmax & mask;
    uint32_t remaining = (uint32_t)g;
    for (int shift = hb - 7 > 0 ? hb - 7 : 0;; shift = shift - 8 > 0 ? shift - 8 : 0) {
        for (int b = tid; b < 256; b += BLOCK) hist[b] = 0;
        S::sync();
        for (int base = 0; base < n; base += BLOCK) {
            int i = base + tid;
            int dig = -1;
            if (i < n) {
                uint64_t k = key_of(i);
                if ((k & mask) == prefix) dig = (int)((k >> shift) & 255u);
            }
            unsigned peers = __match_any_sync(kFull, dig);
            if (dig >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[dig], (uint32_t)__popc(peers));
        }
        S::sync();
        if (warp == 0) {
            // lane l owns bins 255-8l .. 248-8l (from the top)
            uint32_t c[8];
            uint32_t s = 0;
#pragma unroll
            for (int t = 0; t < 8; t++) {
                c[t] = hist[255 - 8 * lane - t];
                s += c[t];
            }
            uint32_t incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t excl = incl - s;
            if (excl < remaining && remaining <= incl) {
                uint32_t above = excl;
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    if (above < remaining && remaining <= above + c[t]) {
                        st[0] = (uint32_t)(255 - 8 * lane - t);
                        st[1] = above;
                        st[2] = c[t];
                        above = 0xFFFFFFFFu;  // found; stop matching
                    } else if (above != 0xFFFFFFFFu) {
                        above += c[t];
                    }
                }
            }
        }
        S::sync();
        const uint32_t bin = st[0], above = st[1], cnt = st[2];
        S::sync();
        remaining -= above;
        prefix = (prefix & ~((uint64_t)0xFF << shift)) | ((uint64_t)bin << shift);
        mask |= (uint64_t)0xFF << shift;
        // the whole bucket is in: the threshold is the bucket's lowest key
        if (cnt == remaining) return prefix;
        if (shift == 0) return prefix;
    }
}

template <int BLOCK, typename KeyOf>
__device__ uint64_t block_select_threshold(const KeyOf& key_of, int n, int g, uint32_t* hist, uint32_t* st) {
    return group_select_threshold<SyncBlock<BLOCK>>(key_of, n, g, hist, st);
}

// Bitonic sort of n (power of two) 64-bit keys in shared memory, descending.
template <int BLOCK>
__device__ void block_bitonic_sort_desc(uint64_t* s, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += BLOCK) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = s[i], b = s[ixj];
                    bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Warp-level bitonic sort of n (power of two, >= 32) 64-bit keys, ascending.
__device__ __forceinline__ void warp_bitonic_sort_asc(uint64_t* s, int n) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = s[i], b = s[ixj];
                    bool asc = (i & k) == 0;
                    if (asc ? (a > b) : (a < b)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace sindi

// Throughput probe for the window scan's inner operation: FP32 atomicAdd into
// a shared-memory window at random slots. The scan's scatter-add (Alg. 2: the
// per-window accumulator A[i mod lambda] += q_j * v) issues exactly this
// operation once per posting; this probe measures how many of them an SM can
// retire per second when nothing else runs, which is the roofline the scan's
// accumulation phase is held against. Measurement infrastructure only: the
// search path does not call it.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void scatter_probe_kernel(uint32_t window, uint32_t iters, float* sink) {
    extern __shared__ float A[];
    for (uint32_t i = threadIdx.x; i < window; i += blockDim.x) A[i] = 0.0f;
    __syncthreads();
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            x = x * 1664525u + 1013904223u;              // LCG step (Numerical Recipes constants)
            atomicAdd(&A[__umulhi(x, window)], 1.0f);    // slot in [0, window)
        }
    }
    __syncthreads();
    float s = 0.0f;
    for (uint32_t i = threadIdx.x; i < window; i += blockDim.x) s += A[i];
    if (s < 0.0f) atomicAdd(sink, s);  // never taken (counts are >= 0); keeps the adds live
}

// The same scatter in five forms, for comparing the scan's FP32 atomicAdd
// with what an exclusive owner of the slots could do instead:
//   0 FP32 atomicAdd, random slot of the window
//   1 FP32 atomicAdd, the 32 lanes of a warp on 32 different banks
//   2 plain load-add-store, random slot of the warp's own 1/warps of the window
//   3 plain load-add-store, warp's own slots, 32 different banks
//   4 uint32 atomicAdd, random slot of the window
// (forms 2 and 3 lose the adds of two lanes that meet on a slot; only their
// rate is measured).
template <int MODE>
__global__ void scatter_mode_kernel(uint32_t window, uint32_t iters, float* sink) {
    extern __shared__ float A[];
    for (uint32_t i = threadIdx.x; i < window; i += blockDim.x) A[i] = 0.0f;
    __syncthreads();
    const uint32_t nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sub = window / nw;  // slots a warp owns (window and warps are powers of two)
    const uint32_t base = warp * sub;
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    uint32_t xr = (blockIdx.x * nw + warp) * 2246822519u + 777u;  // one stream per warp
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            x = x * 1664525u + 1013904223u;
            xr = xr * 1664525u + 1013904223u;
            if (MODE == 0) {
                atomicAdd(&A[__umulhi(x, window)], 1.0f);
            } else if (MODE == 1) {
                atomicAdd(&A[(__umulhi(xr, window >> 5) << 5) + lane], 1.0f);
            } else if (MODE == 2) {
                volatile float* p = &A[base + __umulhi(x, sub)];
                *p = *p + 1.0f;
            } else if (MODE == 3) {
                volatile float* p = &A[base + (__umulhi(xr, sub >> 5) << 5) + lane];
                *p = *p + 1.0f;
            } else {
                atomicAdd(reinterpret_cast<uint32_t*>(&A[__umulhi(x, window)]), 1u);
            }
        }
    }
    __syncthreads();
    float s = 0.0f;
    for (uint32_t i = threadIdx.x; i < window; i += blockDim.x) s += A[i];
    if (s < 0.0f) atomicAdd(sink, s);
}

}  // namespace

// Runs the probe on the current device with `block`-thread blocks, each
// holding a `window`-float shared-memory array, as many blocks as fit on every
// SM at once. Each thread adds 8 * iters times. Writes the adds per second and
// the kernel's duration (CUDA events, second of two launches).
// Returns 0, or the cudaError_t of the first failing call; 1 for bad arguments
// (window 1..32768, block a multiple of 32 in 32..1024, iters >= 1).
extern "C" int sindi_probe_scatter_peak(uint32_t window, uint32_t block, uint32_t iters, double* adds_per_s,
                                        double* ms) {
    if (window == 0 || window > 32768 || block < 32 || block > 1024 || block % 32 || iters == 0 || !adds_per_s)
        return 1;
    cudaError_t e;
    int dev = 0, sms = 0, per_sm = 0;
    const size_t smem = (size_t)window * sizeof(float);
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
    if ((e = cudaFuncSetAttribute(scatter_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return (int)e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scatter_probe_kernel, (int)block, smem)) !=
        cudaSuccess)
        return (int)e;
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)(sms * per_sm);
    float* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float t = 0.0f;
    if ((e = cudaMalloc(&sink, sizeof(float))) != cudaSuccess) return (int)e;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) goto done;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) goto done;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0, s);
        scatter_probe_kernel<<<grid, block, smem, s>>>(window, iters, sink);
        cudaEventRecord(e1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) goto done;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) goto done;
    }
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) goto done;
    *adds_per_s = (double)grid * block * iters * 8.0 / ((double)t * 1e-3);
    if (ms) *ms = t;
done:
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return (int)e;
}

// Rate of scatter form `mode` (0..4, see scatter_mode_kernel) with `block`-thread
// blocks holding a `window`-float array, as many blocks per SM as fit. window and
// block / 32 must be powers of two with window >= 32 * (block / 32). Returns 0,
// the cudaError_t of the first failing call, or 1 for bad arguments.
extern "C" int sindi_probe_scatter_mode(uint32_t mode, uint32_t window, uint32_t block, uint32_t iters,
                                        double* adds_per_s) {
    const uint32_t nw = block / 32;
    if (mode > 4 || window == 0 || window > 32768 || (window & (window - 1)) || block < 32 || block > 1024 ||
        block % 32 || (nw & (nw - 1)) || window < 32 * nw || iters == 0 || !adds_per_s)
        return 1;
    void (*kern)(uint32_t, uint32_t, float*) =
        mode == 0 ? scatter_mode_kernel<0>
                  : mode == 1 ? scatter_mode_kernel<1>
                              : mode == 2 ? scatter_mode_kernel<2> : mode == 3 ? scatter_mode_kernel<3>
                                                                               : scatter_mode_kernel<4>;
    cudaError_t e;
    int dev = 0, sms = 0, per_sm = 0;
    const size_t smem = (size_t)window * sizeof(float);
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return (int)e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)block, smem)) != cudaSuccess)
        return (int)e;
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)(sms * per_sm);
    float* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float t = 0.0f;
    if ((e = cudaMalloc(&sink, sizeof(float))) != cudaSuccess) return (int)e;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) goto done;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) goto done;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0, s);
        kern<<<grid, block, smem, s>>>(window, iters, sink);
        cudaEventRecord(e1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) goto done;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) goto done;
    }
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) goto done;
    *adds_per_s = (double)grid * block * iters * 8.0 / ((double)t * 1e-3);
done:
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return (int)e;
}

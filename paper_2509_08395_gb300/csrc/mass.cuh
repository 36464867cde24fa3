// The alpha-mass subvector (Sec. 4.1, Definitions "Mass of a Vector" and
// "alpha-Mass Subvector") on the device: the sort key of the order pi and the
// FP64 rule that picks the kept count. Documents use it at build time
// (alpha), queries at search time (beta, Alg. 4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sindi {

// Sort key for the alpha-mass order pi: |x| descending, then dim ascending.
// High word: bit-inverted |x| (positive floats order like their bit patterns).
// Low word: dim << 1 | sign of x, so the signed value can be rebuilt.
__device__ __forceinline__ uint64_t mass_key(int32_t j, float v) {
    uint32_t a = __float_as_uint(fabsf(v));
    uint32_t lo = ((uint32_t)j << 1) | (__float_as_uint(v) >> 31);
    return ((uint64_t)(~a) << 32) | lo;
}

__device__ __forceinline__ float mass_key_abs(uint64_t k) { return __uint_as_float(~(uint32_t)(k >> 32)); }
__device__ __forceinline__ int32_t mass_key_dim(uint64_t k) { return (int32_t)((uint32_t)k >> 1); }
__device__ __forceinline__ float mass_key_value(uint64_t k) {
    float a = mass_key_abs(k);
    return ((uint32_t)k & 1u) ? -a : a;
}

// The alpha-mass rule on a row already sorted by mass_key (m_nz non-zero
// entries first). FP64, sequential in pi order, exactly as the definition
// reads: mass = sum |x|, r = smallest r with prefix_r >= alpha * mass.
__device__ __forceinline__ int alpha_mass_count(const uint64_t* s, int m_nz, double alpha) {
    if (m_nz == 0) return 0;
    if (alpha >= 1.0) return m_nz;
    double mass = 0.0;
    for (int t = 0; t < m_nz; t++) mass = __dadd_rn(mass, (double)mass_key_abs(s[t]));
    const double target = __dmul_rn(alpha, mass);
    double prefix = 0.0;
    for (int t = 0; t < m_nz; t++) {
        prefix = __dadd_rn(prefix, (double)mass_key_abs(s[t]));
        if (prefix >= target) return t + 1;
    }
    return m_nz;
}

}  // namespace sindi

// The arithmetic of the fixed-point score window (sindi_accumulator FIXED32):
// the exponent e of one (query, window)'s unit 2^-e, and the integer bound a
// window that has the query's running bound is compared with. Plain functions
// of floats and integers, so that the host tests run the same code.
//
// For one (query, window): B = the sum of |w_j| * vmax_j over the terms whose
// list I_{j,w} is not empty (w_j = q_j, times the list scale for E4M3; vmax_j
// = the largest |stored value| of list I_j), e = 30 - x with 2^(x-1) <= B <
// 2^x, clamped so that every |w_j| * 2^e < 2^127 and to [-126, 126]; 0 when
// B = 0. The window holds integers in units of 2^-e, and every sum stays below
// 2^31 (B * 2^e < 2^30, plus half a unit per product).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "checks.cuh"  // SINDI_HD

namespace sindi {

SINDI_HD uint32_t fx_float_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

SINDI_HD float fx_bits_float(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// x with 2^(x-1) <= f < 2^x for a finite f > 0 (from the exponent field; a
// subnormal f gets x = -126, an upper bound); inf: the bound of a sum of at
// most 4096 (kMaxQueryTerms) values below 2^128.
SINDI_HD int exponent_bound(float f) {
    const int E = (int)((fx_float_bits(f) >> 23) & 0xFFu);
    return E == 0xFF ? 128 + 12 : (E == 0 ? -126 : E - 126);
}

// 2^e as a float, |e| <= 126.
SINDI_HD float pow2f(int e) { return fx_bits_float((uint32_t)(e + 127) << 23); }

// e from B (the sum) and M (the largest |w_j|) of one (query, window).
SINDI_HD int fx_exponent_from(float B, float M) {
    if (!(B > 0.0f)) return 0;
    int e = 30 - exponent_bound(B);
    if (M > 0.0f) {
        const int em = 127 - exponent_bound(M);
        e = e < em ? e : em;
    }
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

// An integer t such that every sum n of a fixed-point window (unit 2^-e, |n| <
// 2^31) whose FP32 score float(n) * 2^-e is >= thr has n >= t: the exact least
// such n when |thr * 2^e| < 2^24 (where the conversion is exact), else up to
// 128 below it (the conversion's rounding at |n| < 2^31), so a few slots just
// under the bound may also be emitted, which the merge drops. NaN: none; -inf:
// all; thr > 0: at least 1 (a zero sum scores 0).
SINDI_HD int32_t fx_threshold(float thr, int e) {
    if (thr != thr) return INT32_MAX;
    if (thr == -INFINITY) return INT32_MIN;
    const float X = thr * pow2f(e);
    int32_t t;
    if (X > 2147483648.0f) t = INT32_MAX;  // above every float(n) (float(n) <= 2^31)
    else if (X < -2147483648.0f) t = INT32_MIN;
    else if (fabsf(X) < 16777216.0f) t = (int32_t)ceilf(X);  // every sum next to X is exact in FP32
    else {
        const int64_t t64 = (int64_t)floorf(X) - 128;  // 64-bit: near -2^31 the margin would wrap in 32 bits
        t = t64 < (int64_t)INT32_MIN ? INT32_MIN : (int32_t)t64;
    }
    return thr > 0.0f ? (t > 1 ? t : 1) : t;
}

}  // namespace sindi

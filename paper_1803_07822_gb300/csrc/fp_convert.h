// Conversions between IEEE 754 binary64 and binary32 done on the integer
// units, written from the two formats' bit fields.  On GB300 a hardware
// conversion between FP64 and FP32 issues on the FP64 pipe, which runs at a
// small fraction of the FP32 rate; the metric and transformation kernels
// convert tens of values per node, and these keep that work off the FP64
// pipe.  Host and device share the code (the host build serves the CPU test
// of the rounding against a reference conversion).
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define CSLBM_HD __host__ __device__ __forceinline__
#else
#define CSLBM_HD inline
#endif

namespace cslbm {

// binary64 -> binary32, round to nearest with ties to even.  Results in the
// binary32 normal range are exact roundings; results below it are flushed to
// a zero of the same sign and results above it (and NaN) become infinity.
CSLBM_HD float f64_to_f32_rn(double x)
{
    uint64_t u;
    memcpy(&u, &x, 8);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // binary32 biased exponent
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the 23 kept fraction bits
    const uint32_t rest = lo & 0x1fffffffu;                  // the 29 dropped ones
    // a carry out of the fraction moves into the exponent, as rounding wants
    uint32_t r = ((uint32_t)(e > 0 ? e : 0) << 23) + m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    if (e <= 0) r = 0u;
    if (e >= 255 || r >= 0x7f800000u) r = 0x7f800000u;
    r |= sign;
    float f;
    memcpy(&f, &r, 4);
    return f;
}

// binary32 -> binary64 (exact for normal numbers and zeros; subnormal
// binary32 inputs become zero)
CSLBM_HD double f32_to_f64(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    uint64_t u = (uint64_t)(b & 0x80000000u) << 32;
    if (e == 255u) u |= 0x7ff0000000000000ull | ((uint64_t)m << 29);
    else if (e != 0u) u |= ((uint64_t)(e - 127u + 1023u) << 52) | ((uint64_t)m << 29);
    double x;
    memcpy(&x, &u, 8);
    return x;
}

}  // namespace cslbm

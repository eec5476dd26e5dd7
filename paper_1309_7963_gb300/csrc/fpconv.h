// Conversions between float and double built from the IEEE-754 bit fields with integer
// instructions.
//
// GB300 runs float<->double conversions (F2F) on its FP64 pipe, at the cost of an FP64
// operation: one warp instruction per 16 SM cycles whatever the number of active lanes
// (measured). The FP32-mode kernels convert often (FP32 momenta into the FP64 boosts and
// bookkeeping and back), so they use these instead, which run on the integer pipes.
//
//   f2d: exact for every normal float, zero, infinity and NaN; subnormal floats (which
//        --use_fast_math flushes anyway) become signed zero.
//   d2f: round to nearest, ties to even; results below the smallest normal float become
//        signed zero (the flush-to-zero conversion of fast-math), overflow becomes infinity,
//        NaN stays NaN.
//
// Plain C++ as well, so that the host tests can check them bit for bit against the
// hardware conversion of the CPU.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PNUC_HD __host__ __device__ __forceinline__
#else
#define PNUC_HD inline
#endif

namespace pnuc {

PNUC_HD uint32_t fbits(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}
PNUC_HD float bitsf(uint32_t b)
{
    float f;
    memcpy(&f, &b, 4);
    return f;
}
PNUC_HD uint64_t dbits(double d)
{
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
}
PNUC_HD double bitsd(uint64_t b)
{
    double d;
    memcpy(&d, &b, 8);
    return d;
}

PNUC_HD double f2d(float f)
{
    const uint32_t b = fbits(f);
    const uint32_t mag = b & 0x7fffffffu;
    // exponent rebias 127 -> 1023 is an add of 896 << 20 to the shifted field
    uint32_t hi = (mag >> 3) + 0x38000000u;
    uint32_t lo = b << 29;
    if (mag >= 0x7f800000u) hi = 0x7ff00000u | ((mag >> 3) & 0x000fffffu);  // inf, NaN
    if (mag < 0x00800000u) hi = lo = 0u;                                    // zero, subnormal
    return bitsd(((uint64_t)(hi | (b & 0x80000000u)) << 32) | lo);
}

PNUC_HD float d2f(double d)
{
    const uint64_t b = dbits(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t E = (hi >> 20) & 0x7ffu;
    const int e = (int)E - 896;  // biased float exponent
    // 23 mantissa bits: 20 from the high word, 3 from the low word; 29 bits dropped
    uint32_t r = ((uint32_t)e << 23) + (((hi & 0x000fffffu) << 3) | (lo >> 29));
    const uint32_t rem = lo & 0x1fffffffu;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry bumps the exponent
    if (e >= 255) r = 0x7f800000u;                                          // overflow
    if (e <= 0) r = 0u;                                                     // below FLT_MIN
    if (E == 0x7ffu) r = ((hi & 0x000fffffu) | lo) ? 0x7fc00000u : 0x7f800000u;
    return bitsf(r | sign);
}

}  // namespace pnuc

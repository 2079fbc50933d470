// Conversions between binary64 and binary32 from the IEEE 754 bit fields,
// with integer operations: on this GPU the conversion instructions share the
// FP64 pipe, which bounds the refinement residual kernels (measured: -8 % for
// the cell-centred, -20 % for the nodal residual).  In kernels that are not
// FP64-bound the 64-bit integer work costs more than it saves (the solution
// update, the strain-rate kernel), so they keep the instructions.  Each
// function gives the same bits as the conversion it replaces (nearest, ties
// to even; exact widening) and falls back to that conversion outside the
// normal ranges.
#pragma once

#include <cuda_runtime.h>

namespace ebv {

// ---- binary64 -> binary32 by the IEEE 754 bit fields (integer operations:
// on this GPU the conversion instructions share the slow FP64 pipe).
// v (0 <= v < 2^62) times 2^scale rounded to binary32 (nearest, ties to
// even); false if the result is not a normal binary32 or zero.
__device__ inline bool u64_to_f32(unsigned long long v, int scale, float &out)
{
    if (v == 0) { out = 0.f; return true; }
    const int L = 63 - __clzll((long long)v);          // index of the leading bit
    unsigned long long q;
    int e = L + scale;                                 // exponent of the leading bit
    if (L <= 23) {
        q = v << (23 - L);
    } else {
        const int sh = L - 23;
        q = v >> sh;
        const unsigned long long r = v & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (r > half || (r == half && (q & 1))) q++;
        if (q == (1ull << 24)) { q >>= 1; e++; }
    }
    if (e < -126 || e > 127) return false;
    out = __uint_as_float((unsigned)(e + 127) << 23 | (unsigned)(q & 0x7fffffu));
    return true;
}

// x 2^k (k the exponent of sc, a power of two) rounded to binary32: the
// scaling is exact, so this is the rounding of x's significand at the shifted
// exponent (the same bits as (float)(x * sc)), falling back to that
// expression when the result leaves the normal binary32 range.
__device__ inline float f64_to_f32_pow2(double x, double sc)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    const int k = (int)(((unsigned long long)__double_as_longlong(sc) >> 52) & 0x7ff) - 1023;
    if ((b << 1) == 0) return (b >> 63) ? -0.f : 0.f;
    float f;
    if (E == 0 || E == 2047 || !u64_to_f32((b & 0xfffffffffffffull) | (1ull << 52), E - 1075 + k, f))
        return __double2float_rn(x * sc);
    return (b >> 63) ? -f : f;
}

}  // namespace ebv

// FP64 tanh for the double-precision kernels: a table of degree-10 Taylor
// expansions on intervals of width 1/16 (coefficients from the derivative
// recurrence of tanh, computed in 60-digit arithmetic by gen_tanh_table.py),
// evaluated with 11 FP64 operations (the interval and its offset are found
// with integer instructions) instead of a general-purpose routine, because
// FP64 issue slots are the scarce resource of the GB300 (FP64 runs at 1/64
// of the FP32 rate).  Odd symmetry gives negative arguments; |x| >= 16,
// infinities and NaN take the library tanh.  Error: within 0.77 ulp before
// the rounding of the Horner steps, measured within a few ulp of CUDA's tanh
// by the GPU tests.
#pragma once

#include <cuda_runtime.h>

#include "tanh_table.inc"

namespace dp {

__device__ __forceinline__ double tanh_f64(double x)
{
    const long long bits = __double_as_longlong(x);
    const long long abits = bits & 0x7fffffffffffffffLL;
    if (abits >= 0x4030000000000000LL) return tanh(x);   // |x| >= 16, inf, NaN
    // k = round(16 |x|) (ties up) and k/16 from the bits with integer instructions: 16 |x| is the
    // significand shifted right by 1071 - exponent (45 .. 53 bits for 1/32 <= |x| < 16)
    const int ex = (int)(abits >> 52);
    int k = 0;
    double kd = 0.0;
    if (ex >= 1018) {
        const unsigned long long mant = ((unsigned long long)abits & ((1ULL << 52) - 1)) | (1ULL << 52);
        const int sh = 1071 - ex;
        k = (int)((mant + (1ULL << (sh - 1))) >> sh);
        const int msb = 31 - __clz(k);                     // k/16 as a double: 2^(msb - 4) (k / 2^msb)
        kd = __longlong_as_double(((long long)(msb - 4 + 1023) << 52) |
                                  ((long long)((unsigned)k ^ (1u << msb)) << (52 - msb)));
    }
    const double d = __longlong_as_double(abits) - kd;      // |x| - k/16, exact, |d| <= 1/32
    const double *c = kTanhTab + k;
    double y = __ldg(c + kTanhDeg * kTanhK);
#pragma unroll
    for (int n = kTanhDeg - 1; n >= 0; --n) y = fma(y, d, __ldg(c + n * kTanhK));
    return __longlong_as_double(__double_as_longlong(y) ^ (bits & (long long)0x8000000000000000ULL));   // sign of x
}

}  // namespace dp

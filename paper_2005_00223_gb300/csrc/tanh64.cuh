// FP64 tanh for the double-precision kernels: a table of degree-10 Taylor
// expansions on intervals of width 1/16 (coefficients from the derivative
// recurrence of tanh, computed in 60-digit arithmetic by gen_tanh_table.py),
// evaluated with 7 FP64 operations instead of a general-purpose routine:
// the interval and its offset are found with integer instructions, and the
// terms of degree 6..10 (below 2^-31 of the result) are summed in FP32,
// because FP64 issue slots are the scarce resource of the GB300 (FP64 runs
// at 1/64 of the FP32 rate).  Odd symmetry gives negative arguments; |x| >= 16,
// infinities and NaN take the library tanh.  Error: within 0.77 ulp before
// the rounding of the Horner steps, measured within a few ulp of CUDA's tanh
// by the GPU tests.
#pragma once

#include <cuda_runtime.h>

#include "tanh_table.inc"

namespace dp {

constexpr int kTanhF = 6;   // coefficients kTanhF .. kTanhDeg are evaluated in FP32


// double -> float by truncation, and float -> double (exact), on the integer
// pipe; magnitudes below the float normal range become 0.
__device__ __forceinline__ float d2f_int(double v)
{
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (ex <= 0) return 0.0f;
    return __uint_as_float((unsigned)((unsigned long long)b >> 32 & 0x80000000u) | ((unsigned)ex << 23) |
                           (unsigned)(((unsigned long long)b >> 29) & 0x7fffffu));
}

__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const int ex = (int)((u >> 23) & 0xff);
    if (ex == 0) return 0.0;
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)(ex - 127 + 1023) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

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
    // the terms of degree kTanhF and above in FP32: they are below 2^-31 of the result, so their
    // FP32 rounding stays within about 2^-53 of it, under the rounding of the FP64 Horner steps
    // (a CPU emulation of this routine gives the same error distribution, at most 1 ulp, as with
    // the degree-6 term in FP64); the rest by Horner in FP64
    const float df = d2f_int(d);
    float tf = d2f_int(__ldg(c + kTanhDeg * kTanhK));
#pragma unroll
    for (int n = kTanhDeg - 1; n >= kTanhF; --n) tf = fmaf(tf, df, d2f_int(__ldg(c + n * kTanhK)));
    double y = f2d_int(tf);
#pragma unroll
    for (int n = kTanhF - 1; n >= 0; --n) y = fma(y, d, __ldg(c + n * kTanhK));
    return __longlong_as_double(__double_as_longlong(y) ^ (bits & (long long)0x8000000000000000ULL));   // sign of x
}

}  // namespace dp

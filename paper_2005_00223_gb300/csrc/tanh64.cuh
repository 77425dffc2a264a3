// FP64 tanh for the double-precision kernels: a table of degree-10 Taylor
// expansions on intervals of width 1/16 (coefficients from the derivative
// recurrence of tanh, computed in 60-digit arithmetic by gen_tanh_table.py),
// evaluated with 13 FP64 operations instead of a general-purpose routine,
// because FP64 issue slots are the scarce resource of the GB300 (FP64 runs
// at 1/64 of the FP32 rate).  Odd symmetry gives negative arguments; |x| >= 16,
// infinities and NaN take the library tanh.  Error: within 0.77 ulp before
// the rounding of the Horner steps, measured within a few ulp of CUDA's tanh
// by the GPU tests.
#pragma once

#include <cuda_runtime.h>

#include "tanh_table.inc"

namespace dp {

__device__ __forceinline__ double tanh_f64(double x)
{
    const double ax = fabs(x);
    if (__double2hiint(ax) >= 0x40300000) return tanh(x);   // |x| >= 16, inf, NaN
    // k = round(16 |x|) from the low word of 16 |x| + 1.5 * 2^52 (ulp 1 there)
    const double t = fma(ax, 16.0, 0x1.8p52);
    const int k = __double2loint(t);
    const double d = fma(t - 0x1.8p52, -0.0625, ax);        // |x| - k/16, exact, |d| <= 1/32
    const double *c = kTanhTab + k;
    double y = __ldg(c + kTanhDeg * kTanhK);
#pragma unroll
    for (int n = kTanhDeg - 1; n >= 0; --n) y = fma(y, d, __ldg(c + n * kTanhK));
    return copysign(y, x);
}

}  // namespace dp

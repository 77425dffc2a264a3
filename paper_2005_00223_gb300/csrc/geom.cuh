// Periodic-box geometry shared by the device kernels: orthorhombic box and
// the minimum-image difference with explicitly rounded FP64 operations.
#pragma once

#include <cuda_runtime.h>

#include "dp_internal.cuh"

namespace dp {

// Packed position (x, y, z, type as a double), one 32-byte load per atom.
struct __align__(32) Pos4 {
    double x, y, z, w;
};

struct BoxDev {
    double L[3], invL[3];
    float invLf[3];       // (float) invL: the FP32 estimate of the image index in min_image_r
    int nc[3];
    int ncell_f;          // cells of one frame
    int64_t frame_n;      // atoms per frame (frame of atom i = i / frame_n)
};

inline BoxDev make_box(const dp_nlist *nl)
{
    BoxDev b;
    for (int k = 0; k < 3; ++k) {
        b.L[k] = nl->L[k];
        b.invL[k] = 1.0 / nl->L[k];
        b.invLf[k] = (float)b.invL[k];
        b.nc[k] = nl->nc[k];
    }
    b.ncell_f = (int)nl->ncell_frame;
    b.frame_n = nl->frame_n > 0 ? nl->frame_n : 1;
    return b;
}

// dk - L rint(dk invL) with the FP64 operations of min_image_r, taking the image index from an FP32
// estimate where that is safe.  The estimate xf = dk' invLf, dk' = dk truncated to its leading 20
// mantissa bits by integer operations (no FP64 instruction), is within 2^-19 |x| of x = dk invL; for
// |xf| <= 2 that is below 4e-6, so where xf is more than 1e-5 away from a half-integer rint(x) =
// rintf(xf) exactly, and the index 0 or +-1 gives the FP64 result with at most one subtraction
// (L (+-1) is exact).  Near a half-integer, for larger indices, and for huge or non-finite dk the FP64
// operations run as written.
__device__ __forceinline__ double min_image_k(double dk, double L, double invL, float invLf)
{
    const int hi = __double2hiint(dk);
    const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;   // FP32 exponent field of dk
    if (e < 140) {                                       // |dk| < 2^13 (and not inf / nan)
        const float xf = e > 0 ? __int_as_float((hi & (int)0x80000000) | (e << 23) | ((hi & 0xfffff) << 3)) * invLf
                               : 0.f;
        const float nf = rintf(xf);
        if (fabsf(xf) <= 2.f && fabsf(fabsf(xf - nf) - 0.5f) > 1e-5f) {
            // index 0: dk itself, except -0, which the FP64 form turns into +0 (-0 - -0 = +0)
            if (nf == 0.f) return __double_as_longlong(dk) == (long long)0x8000000000000000ULL ? 0.0 : dk;
            if (nf == 1.f) return __dsub_rn(dk, L);
            if (nf == -1.f) return __dadd_rn(dk, L);
        }
    }
    return __dsub_rn(dk, __dmul_rn(L, rint(__dmul_rn(dk, invL))));
}

// d = r_b - r_a under minimum image: d_k = (b_k - a_k) - L_k rint((b_k - a_k) / L_k)
// with 1/L_k precomputed; returns r = sqrt((dx dx + dy dy) + dz dz).  Every
// operation is individually rounded (no contraction into multiply-adds); the
// image index comes from an FP32 estimate where that gives the same result
// (min_image_k).
__device__ __forceinline__ double min_image_r(const Pos4 a, const Pos4 b, const BoxDev &bx, double d[3])
{
    const double pa[3] = {a.x, a.y, a.z};
    const double pb[3] = {b.x, b.y, b.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = min_image_k(__dsub_rn(pb[k], pa[k]), bx.L[k], bx.invL[k], bx.invLf[k]);
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    return __dsqrt_rn(r2);
}

// FP32 copy of a position wrapped into [0, L) in FP64 (so its rounding error
// is bounded by the box, whatever the raw coordinate), type bits in w.
__device__ __forceinline__ float4 wrapped_f32(const double *x, int32_t type, const BoxDev &bx)
{
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = (float)(x[k] - bx.L[k] * floor(x[k] * bx.invL[k]));
    return make_float4(w[0], w[1], w[2], __int_as_float(type));
}

// 1/r for 2^-126 < r < 2^126 by two Newton-Raphson steps y <- y + y (1 - r y) in FP64 from the FP32
// hardware reciprocal estimate (relative error about 2^-23, then 2^-46, then below the FP64 rounding):
// four FP64 operations instead of a correctly rounded FP64 division (within an ulp of it).  The FP32
// argument is r truncated to 24 bits and the estimate is widened exactly, with integer instructions.
__device__ __forceinline__ double recip_nr(double r)
{
    const long long b = __double_as_longlong(r);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    const float rf = __uint_as_float((unsigned)((unsigned long long)b >> 32 & 0x80000000u) | ((unsigned)ex << 23) |
                                     (unsigned)(((unsigned long long)b >> 29) & 0x7fffffu));
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(rf));
    const unsigned u = __float_as_uint(yf);
    double y = __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                                ((unsigned long long)(((u >> 23) & 0xffu) - 127 + 1023) << 52) |
                                                ((unsigned long long)(u & 0x7fffffu) << 29)));
    y = fma(y, fma(-r, y, 1.0), y);
    return fma(y, fma(-r, y, 1.0), y);
}

// Switching function of the environment matrix: s = 1/r below r_cs,
// (1/r)(u^3(-6u^2 + 15u - 10) + 1) with u = (r - r_cs)/(r_c - r_cs) up to
// r_c, 0 beyond; *ds = ds/dr.  The quintic is twice continuously
// differentiable at both ends (order-2 smoothness of Sec. 2).  ir = 1/r,
// inv_sw = 1/(r_c - r_cs).
__device__ __forceinline__ double switch_fn(double r, double ir, double rcs, double rc, double inv_sw, double *ds)
{
    if (r < rcs) {
        *ds = -ir * ir;
        return ir;
    }
    if (r < rc) {
        double u = (r - rcs) * inv_sw;
        double u2 = u * u;
        double poly = u2 * u * (-6.0 * u2 + 15.0 * u - 10.0) + 1.0;
        double dpoly = -30.0 * u2 * (u - 1.0) * (u - 1.0) * inv_sw;
        *ds = (dpoly - poly * ir) * ir;
        return poly * ir;
    }
    *ds = 0.0;
    return 0.0;
}

// Environment-matrix row R = (s, s dx/r, s dy/r, s dz/r) and its Jacobian
// J[c][k] = dR_c / dd_k (row-major 4 x 3); inv_sw = 1/(r_c - r_cs).
__device__ __forceinline__ void env_row(const double d[3], double r, double rcs, double rc, double inv_sw, double R[4],
                                        double J[12])
{
    double ds;
    const double ir = recip_nr(r);
    double s = switch_fn(r, ir, rcs, rc, inv_sw, &ds);
    double sr = s * ir;
    double dsr = (ds - sr) * ir;          // d(s/r)/dr
    R[0] = s;
#pragma unroll
    for (int k = 0; k < 3; ++k) R[1 + k] = sr * d[k];
    double u[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
#pragma unroll
    for (int k = 0; k < 3; ++k) J[k] = ds * u[k];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) J[3 * (1 + a) + k] = (a == k ? sr : 0.0) + d[a] * dsr * u[k];
}

}  // namespace dp

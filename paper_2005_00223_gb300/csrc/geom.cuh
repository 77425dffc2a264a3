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
        b.nc[k] = nl->nc[k];
    }
    b.ncell_f = (int)nl->ncell_frame;
    b.frame_n = nl->frame_n > 0 ? nl->frame_n : 1;
    return b;
}

// d = r_b - r_a under minimum image: d_k = (b_k - a_k) - L_k rint((b_k - a_k) / L_k)
// with 1/L_k precomputed; returns r = sqrt((dx dx + dy dy) + dz dz).  Every
// operation is individually rounded (no contraction into multiply-adds).
__device__ __forceinline__ double min_image_r(const Pos4 a, const Pos4 b, const BoxDev &bx, double d[3])
{
    const double pa[3] = {a.x, a.y, a.z};
    const double pb[3] = {b.x, b.y, b.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double dk = __dsub_rn(pb[k], pa[k]);
        double nk = rint(__dmul_rn(dk, bx.invL[k]));
        d[k] = __dsub_rn(dk, __dmul_rn(bx.L[k], nk));
    }
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

// Switching function of the environment matrix: s = 1/r below r_cs,
// (1/r)(u^3(-6u^2 + 15u - 10) + 1) with u = (r - r_cs)/(r_c - r_cs) up to
// r_c, 0 beyond; *ds = ds/dr.  The quintic is twice continuously
// differentiable at both ends (order-2 smoothness of Sec. 2).
__device__ __forceinline__ double switch_fn(double r, double rcs, double rc, double *ds)
{
    if (r < rcs) {
        double ir = 1.0 / r;
        *ds = -ir * ir;
        return ir;
    }
    if (r < rc) {
        double ir = 1.0 / r;
        double u = (r - rcs) / (rc - rcs);
        double u2 = u * u;
        double poly = u2 * u * (-6.0 * u2 + 15.0 * u - 10.0) + 1.0;
        double dpoly = -30.0 * u2 * (u - 1.0) * (u - 1.0) / (rc - rcs);
        *ds = (dpoly - poly * ir) * ir;
        return poly * ir;
    }
    *ds = 0.0;
    return 0.0;
}

// Environment-matrix row R = (s, s dx/r, s dy/r, s dz/r) and its Jacobian
// J[c][k] = dR_c / dd_k (row-major 4 x 3).
__device__ __forceinline__ void env_row(const double d[3], double r, double rcs, double rc, double R[4], double J[12])
{
    double ds;
    double s = switch_fn(r, rcs, rc, &ds);
    double ir = 1.0 / r;
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

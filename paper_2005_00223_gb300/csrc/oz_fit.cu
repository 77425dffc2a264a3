// Hidden layers of the double-precision fitting net (Sec. 2, Fig. 1(d,g))
// with every product as an FP64 product on the tensor cores by error-free
// splitting (ozaki.cuh, ozaki.cu), for the common shape of three hidden
// layers of one width F (a first layer without skip, two with y = x + t) and
// a linear output.  Given z1 = D W1 + b1 of a type's atoms, the chain
//   stage 0  t1 = tanh(z1), x1 = t1, digits of x1
//   GEMM     z2 = x1 W2 + b2
//   stage 1  t2 = tanh(z2), x2 = x1 + t2, digits of x2
//   GEMM     z3 = x2 W3 + b3
//   stage 2  t3 = tanh(z3), x3 = x2 + t3, E_i = x3 . w_out + b_out,
//            dE/dx3 = w_out, dz3 = w_out (1 - t3^2) and its digits
//   GEMM     g = dz3 W3^T
//   stage 3  dE/dx2 = g + w_out (skip), dz2 = dE/dx2 (1 - t2^2), digits
//   GEMM     g = dz2 W2^T
//   stage 4  dE/dx1 = g + dE/dx2 (skip), dz1 = dE/dx1 (1 - t1^2)
// leaves dz1 for the first layer's input gradient dE/dD = dz1 W1^T.  The
// stages run one warp per atom (columns strided over the lanes, E_i summed
// by a fixed shuffle tree); tanh is the FP64 table routine of the other
// FP64 kernels.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "ozaki.cuh"
#include "tanh64.cuh"

namespace dp {
namespace {

constexpr int kS = 9, kBeta = 6, kNC = 48, kKC = 16;   // 240-wide products: 9 digits of 6 bits
constexpr int kMaxJ = 8;                               // columns per lane (F <= 256)

// One warp per row r < rows_pad (rows >= count get zero digits).  Z: the
// stage's input [count][F]; X, DY, T1, T2 [count][F] as listed above; the
// digits of the stage's output row go to dig (tiled for 128-row tiles and
// K chunks of 16) with its scale ex[r]; stage 4 writes dz1 [count][F].
__global__ void __launch_bounds__(256) k_fit_stage(int stage, ModelDev md, int ti, const int32_t *__restrict__ order,
                                                   int64_t pos_begin, int64_t count, int64_t rows_pad,
                                                   const double *__restrict__ Z, double *__restrict__ X,
                                                   double *__restrict__ DY, double *__restrict__ T1,
                                                   double *__restrict__ T2, __half *__restrict__ dig,
                                                   int *__restrict__ ex, double *__restrict__ E_atom,
                                                   double *__restrict__ dz1)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows_pad) return;
    const int F = md.fit.wout[0];
    const bool live = r < count;
    const double *net = md.p + md.fit_base + (int64_t)ti * md.fit.size;
    const double *wout = net + md.fit.W[md.n_fit];
    double v[kMaxJ];   // the value whose digits this stage writes, per owned column
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
        const int k = lane + 32 * j;
        v[j] = 0.0;
        if (!live || k >= F) continue;
        const int64_t q = r * F + k;
        const double z = Z[q];
        if (stage == 0) {
            const double t = tanh_f64(z);
            T1[q] = t;
            X[q] = t;
            v[j] = t;
        } else if (stage == 1) {
            const double t = tanh_f64(z);
            T2[q] = t;
            const double x = X[q] + t;
            X[q] = x;
            v[j] = x;
        } else if (stage == 2) {
            const double t = tanh_f64(z);
            const double x = X[q] + t;
            X[q] = x;                                  // x3, for E_i below
            v[j] = wout[k] * (1.0 - t * t);            // dz3
        } else if (stage == 3) {
            const double dy = z + wout[k];             // dE/dx2
            DY[q] = dy;
            const double t = T2[q];
            v[j] = dy * (1.0 - t * t);                 // dz2
        } else {
            const double dy = z + DY[q];               // dE/dx1
            const double t = T1[q];
            dz1[q] = dy * (1.0 - t * t);
        }
        mx = oz::amax(mx, v[j]);
    }
    if (stage == 2) {
        // E_i = x3 . w_out + b_out
        double e = 0.0;
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
            const int k = lane + 32 * j;
            if (live && k < F) e += X[r * F + k] * wout[k];
        }
        for (int s = 16; s > 0; s >>= 1) e += __shfl_xor_sync(0xffffffffu, e, s);
        if (lane == 0 && live) E_atom[order[pos_begin + r]] = e + net[md.fit.b[md.n_fit]];
    }
    if (stage == 4) return;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = oz::row_exp(mx);
    if (lane == 0) ex[r] = e;
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
        const int k = lane + 32 * j;
        if (k >= F) continue;
        int d[kS];
        oz::digits<kS, kBeta>(v[j], e, d);
#pragma unroll
        for (int i = 0; i < kS; ++i) dig[oz::tiled(r, k, i, kS, 128, kKC, F)] = __int2half_rn(d[i]);
    }
}

size_t weight_halves(const ModelDev &md)
{
    const int F = md.fit.wout[0];
    return (size_t)kS * F * F;   // one product's weight digits
}

}  // namespace

bool oz_fit_chain_ok(const ModelDev &md)
{
    if (md.n_fit != 3) return false;
    const int F = md.fit.wout[0], nd = md.desc_dim;
    return md.fit.wout[1] == F && md.fit.wout[2] == F && F % kNC == 0 && F <= 32 * kMaxJ && nd != F && 2 * nd != F &&
           (long long)kS * F * (1LL << (2 * kBeta - 2)) <= (1LL << 24);
}

// Digits of W2^T, W3^T (rows: output channel; for z = x W) and of W3, W2
// (rows: input; for the input gradients) per type.
dp_status oz_fit_chain_refresh(dp_model *m, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int F = md.fit.wout[0];
    const size_t per = weight_halves(md);
    if (!m->d_ozw_fit) {
        DP_CUDA(cudaMalloc(&m->d_ozw_fit, sizeof(__half) * 4 * per * md.ntypes));
        DP_CUDA(cudaMalloc((void **)&m->d_oze_fit, sizeof(int) * 4 * (size_t)F * md.ntypes));
        ++m->epoch;
        m->oz_fit_stale = true;
    }
    if (!m->oz_fit_stale) return DP_OK;
    for (int t = 0; t < md.ntypes; ++t) {
        __half *w = (__half *)m->d_ozw_fit + 4 * per * t;
        int *e = m->d_oze_fit + 4 * (size_t)F * t;
        const int64_t base = md.fit_base + (int64_t)t * md.fit.size;
        DP_TRY((oz_split<kS, kBeta>(md.pT + base + md.fit.W[1], F, F, F, F, F, kNC, kKC, w, e, st)));
        DP_TRY((oz_split<kS, kBeta>(md.pT + base + md.fit.W[2], F, F, F, F, F, kNC, kKC, w + per, e + F, st)));
        DP_TRY((oz_split<kS, kBeta>(md.p + base + md.fit.W[2], F, F, F, F, F, kNC, kKC, w + 2 * per, e + 2 * F, st)));
        DP_TRY((oz_split<kS, kBeta>(md.p + base + md.fit.W[1], F, F, F, F, F, kNC, kKC, w + 3 * per, e + 3 * F, st)));
    }
    m->oz_fit_stale = false;
    return DP_OK;
}

size_t oz_fit_chain_bytes(const ModelDev &md, int64_t count)
{
    const int64_t rows = (count + 127) / 128 * 128;
    const int F = md.fit.wout[0];
    return sizeof(__half) * rows * kS * F + sizeof(int) * rows + sizeof(double) * count * F * 5 + 8 * 256;
}

// From z1 [count][F] (bias included) of type ti's atoms at positions
// [pos_begin, pos_begin + count): E_i, and dz1 [count][F].
dp_status oz_fit_chain(dp_model *m, int ti, const int32_t *order, int64_t pos_begin, int64_t count,
                       const double *z1, double *dz1, double *E_atom, char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int F = md.fit.wout[0];
    const int64_t rows_pad = (count + 127) / 128 * 128;
    auto carve = [&](size_t bytes) {
        char *p = scratch;
        scratch += (bytes + 255) & ~(size_t)255;
        return p;
    };
    __half *dig = (__half *)carve(sizeof(__half) * rows_pad * kS * F);
    int *ex = (int *)carve(sizeof(int) * rows_pad);
    double *Z = (double *)carve(sizeof(double) * count * F);
    double *X = (double *)carve(sizeof(double) * count * F);
    double *DY = (double *)carve(sizeof(double) * count * F);
    double *T1 = (double *)carve(sizeof(double) * count * F);
    double *T2 = (double *)carve(sizeof(double) * count * F);
    const size_t per = weight_halves(md);
    const __half *w = (const __half *)m->d_ozw_fit + 4 * per * ti;
    const int *e = m->d_oze_fit + 4 * (size_t)F * ti;
    const double *net = md.p + md.fit_base + (int64_t)ti * md.fit.size;
    const unsigned blocks = (unsigned)((rows_pad * 32 + 255) / 256);
    auto stage = [&](int s, const double *in) -> dp_status {
        k_fit_stage<<<blocks, 256, 0, st>>>(s, md, ti, order, pos_begin, count, rows_pad, in, X, DY, T1, T2, dig, ex,
                                            E_atom, dz1);
        DP_CUDA(cudaGetLastError());
        return DP_OK;
    };
    DP_TRY(stage(0, z1));
    DP_TRY((oz_gemm<kS, kBeta, kNC, kKC>(m, count, F, F, dig, ex, rows_pad, w, e, net + md.fit.b[1], Z, F, st)));
    DP_TRY(stage(1, Z));
    DP_TRY((oz_gemm<kS, kBeta, kNC, kKC>(m, count, F, F, dig, ex, rows_pad, w + per, e + F, net + md.fit.b[2], Z, F,
                                         st)));
    DP_TRY(stage(2, Z));
    DP_TRY((oz_gemm<kS, kBeta, kNC, kKC>(m, count, F, F, dig, ex, rows_pad, w + 2 * per, e + 2 * F, nullptr, Z, F, st)));
    DP_TRY(stage(3, Z));
    DP_TRY((oz_gemm<kS, kBeta, kNC, kKC>(m, count, F, F, dig, ex, rows_pad, w + 3 * per, e + 3 * F, nullptr, Z, F, st)));
    return stage(4, Z);
}

}  // namespace dp

// The fitting net (Fig. 1(d,g)) over the atoms of one center type as tiled GEMMs, shared by the
// MIX-32 evaluation (simt.cu: E_i and dE/dD) and the parameter gradient (grad.cu: the primal and the
// forward-mode tangent along v, E_i, Edot_i and their reverse).  A kernel per layer instead of a CTA
// per atom (or a few atoms), which would stream every weight row from L2 once per CTA.
//
// Per hidden layer k, with TAN the tangent rows X' (and Z', Y', their adjoints) beside the primal:
//   forward  Z = X W + b (Z' = X' W), X = D for k = 0, else the layer input stored in rec; then per
//            entry t = tanh(z), y = skip(x) + t (y' = skip(x') + (1 - t^2) z') -> rec;
//   k_fit_out  E_i = y . w + b (Edot_i = y' . w) and the output adjoints alpha w (beta w) of the last
//            hidden layer (alpha = beta = the loss weights in the gradient, alpha = 1 in an evaluation);
//   k_fit_zbar z_bar = (y_bar + y'_bar z' (-2 t)) (1 - t^2), z'_bar = y'_bar (1 - t^2) (without TAN:
//            z_bar = y_bar (1 - t^2));
//   reverse  X_bar = Z_bar W^T + skip^T(Y_bar) (X'_bar likewise) -> the other adjoint buffer of rec,
//            or D_bar (D'_bar) for k = 0.
// rec holds, per atom, every layer's input, t, z', z_bar and z'_bar (FitRec), which the weight
// gradient (grad.cu) reads.  Tiles of 32 atoms x 64 columns, 128 threads of 4 x 4 (primal and tangent
// share every B element), K staged 16 at a time in shared memory.  Per-atom buffers (D, rec, D_bar)
// are indexed by the atom's position minus row0 (a batch's first position); order[] by the position.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "tanh64.cuh"

namespace dp {
namespace fitg {

// Layout of the per-atom record: for hidden layer k (0-based) the offsets of its input x and x'
// (layer 0 reads D and D' instead), t, z', z_bar, z'_bar; then the last hidden output y and y' and
// two adjoint ping-pong vectors.
struct FitRec {
    int x[kMaxFit + 1], xd[kMaxFit + 1], t[kMaxFit + 1], zd[kMaxFit + 1], zb[kMaxFit + 1], zdb[kMaxFit + 1];
    int yl, yld, a0, a0d, a1, a1d;
    int size;
};

inline FitRec make_fit_rec(const ModelDev &md)
{
    FitRec r{};
    int off = 0, wmax = 0;
    for (int k = 0; k < md.n_fit; ++k) {
        const int win = md.fit.win[k], wout = md.fit.wout[k];
        wmax = wmax > wout ? wmax : wout;
        if (k > 0) {
            r.x[k] = off; off += win;
            r.xd[k] = off; off += win;
        }
        r.t[k] = off; off += wout;
        r.zd[k] = off; off += wout;
        r.zb[k] = off; off += wout;
        r.zdb[k] = off; off += wout;
    }
    const int wl = md.fit.wout[md.n_fit - 1];
    r.yl = off; off += wl;
    r.yld = off; off += wl;
    r.a0 = off; off += wmax;
    r.a0d = off; off += wmax;
    r.a1 = off; off += wmax;
    r.a1d = off; off += wmax;
    r.size = off;
    return r;
}

constexpr int kFgM = 32, kFgN = 64, kFgK = 16, kFgThreads = 128;

enum FitGemmMode { FG_FWD = 0, FG_REV = 1 };

struct FitGemmArgs {
    const void *A, *Ad;        // [position - row0][K] at row stride lda (Real); Ad unused without TAN
    int64_t lda;
    const void *B;             // [K][N] row-major (Real)
    const void *bias;          // FG_FWD: [N]
    int M, N, K;
    int k;                     // layer
    int64_t pos_begin, row0;
    int yb, ydb, xb, xdb;      // FG_REV: adjoint buffer offsets in rec
};

__device__ __forceinline__ double fg_tanh(double x) { return tanh_f64(x); }
__device__ __forceinline__ float fg_tanh(float x) { return tanhf(x); }

template <typename Real, int MODE, bool TAN>
__global__ void __launch_bounds__(kFgThreads) k_fit_gemm(ModelDev md, FitRec fr, FitGemmArgs g,
                                                         Real *__restrict__ rec, Real *__restrict__ Db,
                                                         Real *__restrict__ Ddb)
{
    __shared__ __align__(16) Real sA[kFgK][kFgM], sAd[TAN ? kFgK : 1][kFgM], sB[kFgK][kFgN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // 16 column groups x 8 row groups
    const int m0 = blockIdx.x * kFgM, n0 = blockIdx.y * kFgN;
    const Real *A = reinterpret_cast<const Real *>(g.A), *Ad = reinterpret_cast<const Real *>(g.Ad);
    const Real *B = reinterpret_cast<const Real *>(g.B);
    const int64_t r0 = g.pos_begin - g.row0;   // row of the first atom in the per-atom buffers
    Real acc[4][4], accd[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = accd[r][c] = Real(0);
    // the next K step's operands are loaded into registers while the current one is multiplied
    constexpr int LA = kFgM * kFgK / kFgThreads, LB = kFgK * kFgN / kFgThreads;
    Real ra[LA], rad[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * kFgThreads, a = e / kFgK, kk = e - a * kFgK;
            const bool ok = m0 + a < g.M && k0 + kk < g.K;
            const int64_t off = (r0 + m0 + a) * g.lda + k0 + kk;
            ra[q] = ok ? A[off] : Real(0);
            if (TAN) rad[q] = ok ? Ad[off] : Real(0);
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * kFgThreads, kk = e / kFgN, c = e - kk * kFgN;
            rb[q] = (k0 + kk < g.K && n0 + c < g.N) ? B[(int64_t)(k0 + kk) * g.N + n0 + c] : Real(0);
        }
    };
    load(0);
    for (int k0 = 0; k0 < g.K; k0 += kFgK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * kFgThreads, a = e / kFgK, kk = e - a * kFgK;
            sA[kk][a] = ra[q];
            if (TAN) sAd[TAN ? kk : 0][a] = rad[q];
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * kFgThreads, kk = e / kFgN, c = e - kk * kFgN;
            sB[kk][c] = rb[q];
        }
        __syncthreads();
        if (k0 + kFgK < g.K) load(k0 + kFgK);
#pragma unroll
        for (int kk = 0; kk < kFgK; ++kk) {
            Real a[4], ad[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = sA[kk][4 * ty + r];
                ad[r] = TAN ? sAd[TAN ? kk : 0][4 * ty + r] : Real(0);
                b[r] = sB[kk][4 * tx + r];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c] = fma(a[r], b[c], acc[r][c]);
                    if (TAN) accd[r][c] = fma(ad[r], b[c], accd[r][c]);
                }
        }
    }
    const int k = g.k, win = md.fit.win[k], wout = md.fit.wout[k], nd = md.desc_dim;
    const bool skip1 = wout == win, skip2 = wout == 2 * win;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int a = m0 + 4 * ty + r;
        if (a >= g.M) continue;
        const int64_t ra = r0 + a;
        Real *R = rec + ra * fr.size;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = n0 + 4 * tx + c;
            if (j >= g.N) continue;
            if (MODE == FG_FWD) {
                const Real t = fg_tanh(acc[r][c] + reinterpret_cast<const Real *>(g.bias)[j]);
                Real sx = Real(0), sxd = Real(0);
                if (skip1 || skip2) {
                    const int oi = j % win;
                    sx = A[ra * g.lda + oi];
                    if (TAN) sxd = Ad[ra * g.lda + oi];
                }
                R[fr.t[k] + j] = t;
                const Real y = sx + t;
                if (TAN) R[fr.zd[k] + j] = accd[r][c];
                const Real yd = TAN ? sxd + (Real(1) - t * t) * accd[r][c] : Real(0);
                if (k + 1 < md.n_fit) {
                    R[fr.x[k + 1] + j] = y;
                    if (TAN) R[fr.xd[k + 1] + j] = yd;
                } else {
                    R[fr.yl + j] = y;
                    if (TAN) R[fr.yld + j] = yd;
                }
            } else {
                Real s1 = acc[r][c], s2 = accd[r][c];
                if (skip1) {
                    s1 += R[g.yb + j];
                    if (TAN) s2 += R[g.ydb + j];
                } else if (skip2) {
                    s1 += R[g.yb + j] + R[g.yb + j + win];
                    if (TAN) s2 += R[g.ydb + j] + R[g.ydb + j + win];
                }
                if (k == 0) {
                    Db[ra * nd + j] = s1;
                    if (TAN) Ddb[ra * nd + j] = s2;
                } else {
                    R[g.xb + j] = s1;
                    if (TAN) R[g.xdb + j] = s2;
                }
            }
        }
    }
}

// Output layer (one warp per atom): E_i = y . w + b (Edot_i = y' . w), and the output adjoints of the
// last hidden layer, alpha w (beta w), into rec's first adjoint buffer.  ab = [beta, alpha of frame
// 0, 1, ...] (the gradient's loss weights), or null: alpha = 1 (an evaluation's dE/dy).
template <typename Real, bool TAN>
__global__ void __launch_bounds__(256) k_fit_out(ModelDev md, FitRec fr, int ti, const int32_t *__restrict__ order,
                                                int64_t pos_begin, int64_t row0, int64_t count,
                                                const double *__restrict__ ab, int64_t frame_n,
                                                Real *__restrict__ rec, double *__restrict__ E_atom,
                                                double *__restrict__ Ed_atom)
{
    const int lane = threadIdx.x & 31;
    const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (a >= count) return;
    const Real *net = (sizeof(Real) == sizeof(double) ? reinterpret_cast<const Real *>(md.p)
                                                      : reinterpret_cast<const Real *>(md.p32)) +
                      md.fit_base + (int64_t)ti * md.fit.size;
    const int wl = md.fit.wout[md.n_fit - 1];
    const Real *Wout = net + md.fit.W[md.n_fit];
    const int64_t pa = pos_begin + a;
    Real *R = rec + (pa - row0) * fr.size;
    const Real alpha = ab ? (Real)ab[1 + order[pa] / frame_n] : Real(1);
    const Real beta = TAN ? (Real)ab[0] : Real(0);
    Real e = Real(0), ed = Real(0);
    for (int o = lane; o < wl; o += 32) {
        const Real w = Wout[o];
        e += R[fr.yl + o] * w;
        R[fr.a0 + o] = alpha * w;
        if (TAN) {
            ed += R[fr.yld + o] * w;
            R[fr.a0d + o] = beta * w;
        }
    }
    for (int s = 16; s > 0; s >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, s);
        if (TAN) ed += __shfl_xor_sync(0xffffffffu, ed, s);
    }
    if (lane == 0) {
        E_atom[order[pa]] = (double)(e + net[md.fit.b[md.n_fit]]);
        if (TAN) Ed_atom[order[pa]] = (double)ed;
    }
}

// z_bar = (y_bar + y'_bar z' (-2 t)) (1 - t^2), z'_bar = y'_bar (1 - t^2) of layer k for every atom
// (without TAN: z_bar = y_bar (1 - t^2)).
template <typename Real, bool TAN>
__global__ void k_fit_zbar(ModelDev md, FitRec fr, int k, int yb, int ydb, int64_t pos_begin, int64_t row0,
                           int64_t count, Real *__restrict__ rec)
{
    const int wout = md.fit.wout[k];
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count * wout) return;
    const int64_t a = q / wout;
    const int o = (int)(q - a * wout);
    Real *R = rec + (pos_begin - row0 + a) * fr.size;
    const Real t = R[fr.t[k] + o], g1 = Real(1) - t * t;
    if (TAN) {
        R[fr.zb[k] + o] = (R[yb + o] + R[ydb + o] * R[fr.zd[k] + o] * (Real(-2) * t)) * g1;
        R[fr.zdb[k] + o] = R[ydb + o] * g1;
    } else {
        R[fr.zb[k] + o] = R[yb + o] * g1;
    }
}

// Host side: the device parameters (flat order, or with every W transposed) in the precision Real.
template <typename Real>
const Real *fit_params(const ModelDev &md, bool transposed)
{
    if constexpr (sizeof(Real) == sizeof(double)) return transposed ? md.pT : md.p;
    else return transposed ? md.pT32 : md.p32;
}

// The fitting net of center type ti over `count` atoms at positions pos_begin.. of the type-sorted
// order: D (D') rows, rec and D_bar (D'_bar) indexed by position - row0; E_i (Edot_i) by atom index.
// Launches 2 n_fit + 1 + n_fit kernels on st.
template <typename Real, bool TAN>
void fit_net_run(const ModelDev &md, const FitRec &fr, int ti, const int32_t *order, int64_t pos_begin, int64_t row0,
                 int64_t count, const double *ab, int64_t frame_n, const Real *D, const Real *Dd, Real *rec,
                 double *E_atom, double *Ed_atom, Real *Db, Real *Ddb, cudaStream_t st)
{
    const Real *fnet = fit_params<Real>(md, false) + md.fit_base + (int64_t)ti * md.fit.size;
    const Real *fnetT = fit_params<Real>(md, true) + md.fit_base + (int64_t)ti * md.fit.size;
    const unsigned mt = (unsigned)((count + kFgM - 1) / kFgM);
    for (int k = 0; k < md.n_fit; ++k) {
        FitGemmArgs g{};
        g.A = k == 0 ? (const void *)D : (const void *)(rec + fr.x[k]);
        g.Ad = k == 0 ? (const void *)Dd : (const void *)(rec + fr.xd[k]);
        g.lda = k == 0 ? md.desc_dim : fr.size;
        g.B = fnet + md.fit.W[k];
        g.bias = fnet + md.fit.b[k];
        g.M = (int)count;
        g.N = md.fit.wout[k];
        g.K = md.fit.win[k];
        g.k = k;
        g.pos_begin = pos_begin;
        g.row0 = row0;
        k_fit_gemm<Real, FG_FWD, TAN><<<dim3(mt, (unsigned)((g.N + kFgN - 1) / kFgN)), kFgThreads, 0, st>>>(
            md, fr, g, rec, Db, Ddb);
    }
    k_fit_out<Real, TAN><<<(unsigned)((count * 32 + 255) / 256), 256, 0, st>>>(md, fr, ti, order, pos_begin, row0,
                                                                              count, ab, frame_n, rec, E_atom,
                                                                              Ed_atom);
    int cur = 0;   // adjoint buffer holding the current layer's output adjoints
    for (int k = md.n_fit - 1; k >= 0; --k) {
        FitGemmArgs g{};
        g.yb = cur ? fr.a1 : fr.a0;
        g.ydb = cur ? fr.a1d : fr.a0d;
        g.xb = cur ? fr.a0 : fr.a1;
        g.xdb = cur ? fr.a0d : fr.a1d;
        const int64_t nz = count * md.fit.wout[k];
        k_fit_zbar<Real, TAN><<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(md, fr, k, g.yb, g.ydb, pos_begin, row0,
                                                                           count, rec);
        g.A = rec + fr.zb[k];
        g.Ad = rec + fr.zdb[k];
        g.lda = fr.size;
        g.B = fnetT + md.fit.W[k];   // W^T: [wout][win]
        g.M = (int)count;
        g.N = md.fit.win[k];
        g.K = md.fit.wout[k];
        g.k = k;
        g.pos_begin = pos_begin;
        g.row0 = row0;
        k_fit_gemm<Real, FG_REV, TAN><<<dim3(mt, (unsigned)((g.N + kFgN - 1) / kFgN)), kFgThreads, 0, st>>>(
            md, fr, g, rec, Db, Ddb);
        cur ^= 1;
    }
}

}  // namespace fitg
}  // namespace dp

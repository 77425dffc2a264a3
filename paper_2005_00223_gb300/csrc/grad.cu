// Parameter gradient of alpha E + beta Edot, Edot = sum_k v_k . dE/dr_k, the
// primitive of force-matching training (the loss
// L = p_e (dE/N)^2 + p_f/(3N) sum |F - F_ref|^2 has
// dL/dtheta = 2 p_e dE/N^2 dE/dtheta - 2 p_f/(3N) dEdot/dtheta with
// v = F - F_ref held fixed, since F = -grad_r E).
//
// Edot is the forward-mode tangent of E along v: for atom i the tangent of
// the environment row is J (v_j - v_i), and every layer carries (x, x') with
// z' = x' W, t' = (1 - t^2) z', y' = skip(x') + t'.  The gradient over the
// parameters is reverse mode through the primal and tangent programs; per
// layer with output adjoints (y_bar, y'_bar):
//   z'_bar = y'_bar (1 - t^2),  t_bar = y_bar - 2 t z' z'_bar / (1 - t^2) * (1 - t^2)
//          = y_bar + y'_bar z' (-2 t),  z_bar = t_bar (1 - t^2),
//   W_bar += x^T z_bar + x'^T z'_bar,  b_bar += z_bar,
//   x_bar = z_bar W^T + skip^T(y_bar),  x'_bar = z'_bar W^T + skip^T(y'_bar).
// Embedding activations are recomputed in the reverse pass, not stored.
//
// Kernels per evaluation (SIMT, Real = double or float; geometry FP64):
//   k_jvp_fwd     CTA per atom: env rows and tangents, embedding primal +
//                 tangent, T, T', D, D'.
//   k_fit_gemm    per fitting layer, tiled GEMMs over the atoms of a type:
//                 primal + tangent forward (with tanh and skips), then with
//                 k_fit_out (E_i, Edot_i) and k_fit_zbar the reverse with
//                 (alpha, beta) -> D_bar, D'_bar; keeps layer inputs and
//                 pre-activation adjoints for k_fit_wgrad.
//   k_fit_wgrad   the fitting net's weight gradient as tiled GEMMs over the atoms of
//                 a type (split over chunks of atoms), k_fit_wgrad_reduce the chunks.
//   k_jvp_bwd     persistent CTAs over atoms: T_bar, T'_bar, then per chunk
//                 recompute the embedding primal + tangent and run it in
//                 reverse, accumulating the embedding gradient in a private
//                 slice per CTA.
//   k_grad_reduce the private slices, summed in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "dp_internal.cuh"
#include "fit_gemm.cuh"
#include "geom.cuh"
#include "tanh64.cuh"

namespace dp {
namespace {

// Atoms per CTA of the fitting tangent kernel: 4, or 1 when 4 would leave SMs idle.

__device__ __forceinline__ double g_tanh(double x) { return tanh_f64(x); }
__device__ __forceinline__ float g_tanh(float x) { return tanhf(x); }

template <typename Real>
__device__ __forceinline__ const Real *P_of(const ModelDev &md);
template <>
__device__ __forceinline__ const double *P_of<double>(const ModelDev &md) { return md.p; }
template <>
__device__ __forceinline__ const float *P_of<float>(const ModelDev &md) { return md.p32; }

template <int G_, int E0_, int E1_, int E2_>
struct GShape {
    static constexpr int G = G_, E0 = E0_, E1 = E1_, E2 = E2_, NT = 32 * G_, LD = 33;
    static constexpr int WMAX = E2_ > E1_ ? E2_ : E1_;
    static_assert(E0_ % G_ == 0 && E1_ % G_ == 0 && E2_ % G_ == 0, "channels split evenly over warps");
};

using GWater = GShape<5, 25, 50, 100>;
using GStudent = GShape<4, 8, 16, 32>;
using GPaper = GShape<4, 32, 64, 128>;

// Environment rows and tangents of one chunk (warp 0, lane = neighbor).
template <typename Real>
__device__ __forceinline__ void env_tangent(const ModelDev &md, const BoxDev &bx, const Pos4 *pos,
                                            const int32_t *nlist, const double *v, int i, const Pos4 &pi, int tj,
                                            int c0, int cnt, int n, Real *sR, Real *sRd)
{
    double R[4] = {0, 0, 0, 0}, Rd[4] = {0, 0, 0, 0};
    const int j = c0 + n < cnt ? nlist[(int64_t)i * md.nsel + md.sel_off[tj] + c0 + n] : -1;
    if (c0 + n < cnt && DP_IDX_OK(j, md.n_list, BS_NLIST_J)) {
        double d[3], J[12];
        const double r = min_image_r(pi, pos[j], bx, d);
        env_row(d, r, md.rcs, md.rcut, md.inv_sw, R, J);
        double dd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) dd[k] = v[3 * (int64_t)j + k] - v[3 * (int64_t)i + k];
#pragma unroll
        for (int c = 0; c < 4; ++c) Rd[c] = J[3 * c] * dd[0] + J[3 * c + 1] * dd[1] + J[3 * c + 2] * dd[2];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        sR[n * 4 + c] = (Real)R[c];
        sRd[n * 4 + c] = (Real)Rd[c];
    }
}

// Primal + tangent of one hidden layer for the chunk; thread owns outputs
// o = g + G u.  Inputs X/Xd [WIN][LD], outputs Y/Yd [WOUT][LD]; t and z'
// of the owned outputs are returned in registers.
template <class S, int WIN, int WOUT, typename Real>
__device__ __forceinline__ void layer_ft(const Real *W, const Real *b, const Real *X, const Real *Xd, Real *Y,
                                         Real *Yd, Real (&t)[WOUT / S::G], Real (&zd)[WOUT / S::G], int g, int n)
{
    constexpr int NO = WOUT / S::G;
    Real z[NO];
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        z[u] = b[g + S::G * u];
        zd[u] = Real(0);
    }
    for (int k = 0; k < WIN; ++k) {
        const Real x = X[k * S::LD + n], xd = Xd[k * S::LD + n];
        const Real *Wr = W + k * WOUT + g;
#pragma unroll
        for (int u = 0; u < NO; ++u) {
            const Real w = Wr[S::G * u];
            z[u] += x * w;
            zd[u] += xd * w;
        }
    }
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        const int o = g + S::G * u;
        t[u] = g_tanh(z[u]);
        Real sx = Real(0), sxd = Real(0);
        if (WOUT == WIN) { sx = X[o * S::LD + n]; sxd = Xd[o * S::LD + n]; }
        else if (WOUT == 2 * WIN) { sx = X[(o % WIN) * S::LD + n]; sxd = Xd[(o % WIN) * S::LD + n]; }
        Y[o * S::LD + n] = sx + t[u];
        Yd[o * S::LD + n] = sxd + (Real(1) - t[u] * t[u]) * zd[u];
    }
}

// Layer 0 (input width 1: s and s').
template <class S, typename Real>
__device__ __forceinline__ void layer0_ft(const Real *W, const Real *b, Real s, Real sd, Real *Y, Real *Yd,
                                          Real (&t)[S::E0 / S::G], Real (&zd)[S::E0 / S::G], int g, int n)
{
    constexpr int NO = S::E0 / S::G;
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        const int o = g + S::G * u;
        const Real z = b[o] + s * W[o];
        zd[u] = sd * W[o];
        t[u] = g_tanh(z);
        Real sx = Real(0), sxd = Real(0);
        if (S::E0 == 1 || S::E0 == 2) { sx = s; sxd = sd; }
        Y[o * S::LD + n] = sx + t[u];
        Yd[o * S::LD + n] = sxd + (Real(1) - t[u] * t[u]) * zd[u];
    }
}

template <class S, typename Real>
__global__ void __launch_bounds__(S::NT) k_jvp_fwd(ModelDev md, BoxDev bx, const int32_t *__restrict__ order,
                                                  const Pos4 *__restrict__ pos, const int32_t *__restrict__ nlist,
                                                  const int32_t *__restrict__ nnei, const double *__restrict__ v,
                                                  Real *__restrict__ Tp, Real *__restrict__ Tdp, Real *__restrict__ Dp,
                                                  Real *__restrict__ Ddp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    constexpr int G = S::G, NT = S::NT, LD = S::LD;
    const int tid = threadIdx.x, n = tid & 31, g = tid >> 5;
    Real *sW = sm;
    Real *X1 = sW + md.emb.size, *X1d = X1 + S::E0 * LD;
    Real *X2 = X1d + S::E0 * LD, *X2d = X2 + S::E1 * LD;
    Real *X3 = X2d + S::E1 * LD, *X3d = X3 + S::E2 * LD;
    Real *sR = X3d + S::E2 * LD, *sRd = sR + 128;
    Real *sT = sRd + 128, *sTd = sT + 4 * S::E2;
    const int64_t p = blockIdx.x;
    const int i = order[p];
    const Pos4 pi = pos[i];
    const int ti = (int)pi.w;
    const Real *P = P_of<Real>(md);
    constexpr int KT = (4 * S::E2 + NT - 1) / NT;
    Real ta[KT], tda[KT];
#pragma unroll
    for (int u = 0; u < KT; ++u) ta[u] = tda[u] = Real(0);
    for (int tj = 0; tj < md.ntypes; ++tj) {
        const int cnt = nnei[(int64_t)i * md.ntypes + tj];
        if (cnt == 0) continue;
        __syncthreads();
        const Real *net = P + md.emb_base + (int64_t)(ti * md.ntypes + tj) * md.emb.size;
        for (int q = tid; q < md.emb.size; q += NT) sW[q] = net[q];
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            if (g == 0) env_tangent<Real>(md, bx, pos, nlist, v, i, pi, tj, c0, cnt, n, sR, sRd);
            __syncthreads();
            Real t0[S::E0 / G], z0[S::E0 / G], t1[S::E1 / G], z1[S::E1 / G], t2[S::E2 / G], z2[S::E2 / G];
            layer0_ft<S, Real>(sW + md.emb.W[0], sW + md.emb.b[0], sR[n * 4], sRd[n * 4], X1, X1d, t0, z0, g, n);
            __syncthreads();
            layer_ft<S, S::E0, S::E1, Real>(sW + md.emb.W[1], sW + md.emb.b[1], X1, X1d, X2, X2d, t1, z1, g, n);
            __syncthreads();
            layer_ft<S, S::E1, S::E2, Real>(sW + md.emb.W[2], sW + md.emb.b[2], X2, X2d, X3, X3d, t2, z2, g, n);
            __syncthreads();
#pragma unroll
            for (int u = 0; u < KT; ++u) {
                const int q = tid + u * NT;
                if (q < 4 * S::E2) {
                    const int m = q >> 2, c = q & 3;
                    Real a = Real(0), ad = Real(0);
                    for (int nn = 0; nn < 32; ++nn) {
                        const Real G_ = X3[m * LD + nn], Gd = X3d[m * LD + nn];
                        a += G_ * sR[nn * 4 + c];
                        ad += Gd * sR[nn * 4 + c] + G_ * sRd[nn * 4 + c];
                    }
                    ta[u] += a;
                    tda[u] += ad;
                }
            }
            __syncthreads();
        }
    }
    const Real inv = (Real)md.inv_nsel;
#pragma unroll
    for (int u = 0; u < KT; ++u) {
        const int q = tid + u * NT;
        if (q < 4 * S::E2) {
            sT[q] = ta[u] * inv;
            sTd[q] = tda[u] * inv;
            Tp[p * 4 * S::E2 + q] = sT[q];
            Tdp[p * 4 * S::E2 + q] = sTd[q];
        }
    }
    __syncthreads();
    const int nd = S::E2 * md.m2;
    for (int q = tid; q < nd; q += NT) {
        const int a = q / md.m2, b = q - a * md.m2;
        Real dv = Real(0), ddv = Real(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            dv += sT[4 * a + c] * sT[4 * b + c];
            ddv += sTd[4 * a + c] * sT[4 * b + c] + sT[4 * a + c] * sTd[4 * b + c];
        }
        Dp[p * nd + q] = dv;
        Ddp[p * nd + q] = ddv;
    }
}

using fitg::FitRec;
using fitg::make_fit_rec;

// Weight gradient of the fitting net of type ti as GEMMs over the atoms.  For each layer k,
// with the bias as one more input row of constant 1:
//   W_bar[i][o] = sum_a x[a][i] z_bar[a][o] + x'[a][i] z'_bar[a][o],  b_bar[o] = sum_a z_bar[a][o],
// and for the linear output layer x = y, z_bar = alpha_frame(a), x' = y', z'_bar = beta.
// Work: 64 x 64 tiles of (inputs + 1) x outputs of every layer (WgPlan) times chunks of the
// atoms; each thread holds a 4 x 4 block of the tile, stages 16 atoms of x, x', z_bar, z'_bar in
// shared memory at a time and accumulates in Real over its chunk; the chunk's partial sums go to
// part[chunk][parameter] (FP64) and k_fit_wgrad_reduce adds the chunks in a fixed order.
constexpr int kWgTile = 64, kWgAtoms = 16, kWgThreads = 256;

struct WgPlan {
    int nlayers;                  // hidden layers + the output layer
    int tiles_in[kMaxFit + 1];    // tiles over win + 1 (the bias row)
    int tiles_out[kMaxFit + 1];
    int start[kMaxFit + 2];       // first tile of each layer
    int chunk;                    // atoms per chunk
};

WgPlan make_wg_plan(const ModelDev &md)
{
    WgPlan p{};
    p.nlayers = md.n_fit + 1;
    p.start[0] = 0;
    for (int k = 0; k < p.nlayers; ++k) {
        p.tiles_in[k] = (md.fit.win[k] + 1 + kWgTile - 1) / kWgTile;
        p.tiles_out[k] = (md.fit.wout[k] + kWgTile - 1) / kWgTile;
        p.start[k + 1] = p.start[k] + p.tiles_in[k] * p.tiles_out[k];
    }
    return p;
}

template <typename Real>
__global__ void __launch_bounds__(kWgThreads) k_fit_wgrad(ModelDev md, FitRec fr, WgPlan pl,
                                                          const int32_t *__restrict__ order, int64_t pos_begin,
                                                          int64_t count, const double *__restrict__ ab,
                                                          int64_t frame_n, const Real *__restrict__ D,
                                                          const Real *__restrict__ Dd, const Real *__restrict__ rec,
                                                          double *__restrict__ part)
{
    __shared__ __align__(16) Real sX[kWgAtoms][kWgTile], sXd[kWgAtoms][kWgTile];
    __shared__ __align__(16) Real sZ[kWgAtoms][kWgTile], sZd[kWgAtoms][kWgTile];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int k = 0;
    while (k + 1 < pl.nlayers && (int)blockIdx.x >= pl.start[k + 1]) ++k;
    const int tt = (int)blockIdx.x - pl.start[k];
    const int in0 = (tt / pl.tiles_out[k]) * kWgTile, o0 = (tt % pl.tiles_out[k]) * kWgTile;
    const int win = md.fit.win[k], wout = md.fit.wout[k], nd = md.desc_dim;
    const bool last = k == md.n_fit;
    const int64_t a_begin = (int64_t)blockIdx.y * pl.chunk;
    const int64_t a_end = a_begin + pl.chunk < count ? a_begin + pl.chunk : count;
    Real acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = Real(0);
    for (int64_t a0 = a_begin; a0 < a_end; a0 += kWgAtoms) {
        __syncthreads();
        // stage x, x' (inputs in0 ..) and z_bar, z'_bar (outputs o0 ..) of kWgAtoms atoms
        for (int e = tid; e < 4 * kWgAtoms * kWgTile; e += kWgThreads) {
            const int arr = e / (kWgAtoms * kWgTile), rem = e - arr * (kWgAtoms * kWgTile);
            const int aa = rem / kWgTile, col = rem - aa * kWgTile;
            const int64_t pa = pos_begin + a0 + aa;
            Real v = Real(0);
            if (a0 + aa < a_end) {
                const Real *R = rec + pa * fr.size;
                if (arr < 2) {   // x or x' at input in0 + col; the row win is the bias input
                    const int i = in0 + col;
                    if (i < win) {
                        if (last) v = R[(arr == 0 ? fr.yl : fr.yld) + i];
                        else if (k == 0) v = (arr == 0 ? D : Dd)[pa * nd + i];
                        else v = R[(arr == 0 ? fr.x[k] : fr.xd[k]) + i];
                    } else if (i == win && arr == 0) {
                        v = Real(1);
                    }
                } else {         // z_bar or z'_bar at output o0 + col
                    const int o = o0 + col;
                    if (o < wout) {
                        if (last) v = arr == 2 ? (Real)ab[1 + order[pa] / frame_n] : (Real)ab[0];
                        else v = R[(arr == 2 ? fr.zb[k] : fr.zdb[k]) + o];
                    }
                }
            }
            Real *dst = arr == 0 ? &sX[0][0] : arr == 1 ? &sXd[0][0] : arr == 2 ? &sZ[0][0] : &sZd[0][0];
            dst[rem] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int aa = 0; aa < kWgAtoms; ++aa) {
            Real x[4], xd[4], z[4], zd[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                x[r] = sX[aa][4 * ty + r];
                xd[r] = sXd[aa][4 * ty + r];
                z[r] = sZ[aa][4 * tx + r];
                zd[r] = sZd[aa][4 * tx + r];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(x[r], z[c], fma(xd[r], zd[c], acc[r][c]));
        }
    }
    double *pc = part + (int64_t)blockIdx.y * md.fit.size;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = in0 + 4 * ty + r;
        if (i > win) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int o = o0 + 4 * tx + c;
            if (o >= wout) continue;
            const int64_t q = i < win ? md.fit.W[k] + (int64_t)i * wout + o : md.fit.b[k] + o;
            pc[q] = (double)acc[r][c];
        }
    }
}

// grad[fitting net ti] += the chunks' partial sums, added in chunk order.
__global__ void k_fit_wgrad_reduce(ModelDev md, int ti, const double *__restrict__ part, int nchunks,
                                   double *__restrict__ grad)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= md.fit.size) return;
    double acc = 0.0;
    for (int c = 0; c < nchunks; ++c) acc += part[(int64_t)c * md.fit.size + q];
    grad[md.fit_base + (int64_t)ti * md.fit.size + q] += acc;
}

// formula(Xb, Y)[a][c] = sum_b Xb[a][b] Y[b][c] + [a < M2] sum_a' Xb[a'][a] Y[a'][c]
template <typename Real>
__device__ __forceinline__ Real desc_adj(const Real *Xb, const Real *Y, int m1, int m2, int a, int c)
{
    Real acc = Real(0);
    for (int b = 0; b < m2; ++b) acc += Xb[a * m2 + b] * Y[4 * b + c];
    if (a < m2)
        for (int a2 = 0; a2 < m1; ++a2) acc += Xb[a2 * m2 + a] * Y[4 * a2 + c];
    return acc;
}

// Reverse of one hidden layer for a chunk.  dy, dyd: owned output adjoints
// (registers, with the skip terms of the layer above already added); t, zd:
// owned t and z'.  Writes z_bar, z'_bar to Zb/Zdb [WOUT][LD]; after a sync
// accumulates W_bar and b_bar into gW (private slice); returns the input
// adjoints (owned inputs) without this layer's skip terms added.
template <class S, int WIN, int WOUT, typename Real>
__device__ __forceinline__ void layer_rev(const Real *W, const Real *X, const Real *Xd, Real *Zb, Real *Zdb,
                                          const Real (&dy)[WOUT / S::G], const Real (&dyd)[WOUT / S::G],
                                          const Real (&t)[WOUT / S::G], const Real (&zd)[WOUT / S::G], Real *gW,
                                          Real *gb, Real (&xb)[WIN / S::G], Real (&xdb)[WIN / S::G], int tid, int g,
                                          int n)
{
    constexpr int NO = WOUT / S::G, NI = WIN / S::G, LD = S::LD, NT = S::NT;
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        const int o = g + S::G * u;
        const Real g1 = Real(1) - t[u] * t[u];
        const Real zdb = dyd[u] * g1;
        const Real tb = dy[u] + dyd[u] * zd[u] * (Real(-2) * t[u]);
        Zb[o * LD + n] = tb * g1;
        Zdb[o * LD + n] = zdb;
    }
    __syncthreads();
    // FP32: W_bar in 4 x 4 blocks of (input k, output o) where there are enough blocks for every
    // thread: each row's 4 + 4 inputs and 4 + 4 adjoints feed 32 multiply-adds (one shared-memory load
    // per two multiply-adds instead of two per one).  Smaller layers, and FP64, whose DFMA-bound loop
    // gains nothing from fewer loads and would lose to the blocks' uneven split over the threads, keep
    // one entry per thread.
    constexpr int KB = (WIN + 3) / 4, OB = (WOUT + 3) / 4;
    if (KB * OB < NT || sizeof(Real) == sizeof(double)) {
        for (int e = tid; e < WIN * WOUT; e += NT) {
            const int k = e / WOUT, o = e - k * WOUT;
            Real acc = Real(0);
#pragma unroll 8
            for (int nn = 0; nn < 32; ++nn) acc += X[k * LD + nn] * Zb[o * LD + nn] + Xd[k * LD + nn] * Zdb[o * LD + nn];
            gW[e] += acc;
        }
    } else {
        for (int blk = tid; blk < KB * OB; blk += NT) {
            const int k0 = (blk / OB) * 4, q0 = (blk % OB) * 4;
            Real acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = Real(0);
#pragma unroll 2
            for (int nn = 0; nn < 32; ++nn) {
                Real x[4], xd[4], zb[4], zdb[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k = k0 + r < WIN ? k0 + r : WIN - 1;
                    const int o = q0 + r < WOUT ? q0 + r : WOUT - 1;
                    x[r] = X[k * LD + nn];
                    xd[r] = Xd[k * LD + nn];
                    zb[r] = Zb[o * LD + nn];
                    zdb[r] = Zdb[o * LD + nn];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += x[r] * zb[c] + xd[r] * zdb[c];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (k0 + r < WIN && q0 + c < WOUT) gW[(k0 + r) * WOUT + q0 + c] += acc[r][c];
        }
    }
    for (int o = tid; o < WOUT; o += NT) {
        Real acc = Real(0);
        for (int nn = 0; nn < 32; ++nn) acc += Zb[o * LD + nn];
        gb[o] += acc;
    }
#pragma unroll
    for (int u = 0; u < NI; ++u) { xb[u] = Real(0); xdb[u] = Real(0); }
    for (int o = 0; o < WOUT; ++o) {
        const Real zb = Zb[o * LD + n], zdb = Zdb[o * LD + n];
        const Real *Wc = W + g * WOUT + o;
#pragma unroll
        for (int u = 0; u < NI; ++u) {
            const Real w = Wc[S::G * u * WOUT];
            xb[u] += zb * w;
            xdb[u] += zdb * w;
        }
    }
}

template <class S, typename Real>
__global__ void __launch_bounds__(S::NT) k_jvp_bwd(ModelDev md, BoxDev bx, const int32_t *__restrict__ order, int64_t n_atoms,
                                                  const Pos4 *__restrict__ pos, const int32_t *__restrict__ nlist,
                                                  const int32_t *__restrict__ nnei, const double *__restrict__ v,
                                                  const Real *__restrict__ Tp, const Real *__restrict__ Tdp,
                                                  const Real *__restrict__ Dbp, const Real *__restrict__ Ddbp,
                                                  Real *__restrict__ gpriv)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    constexpr int G = S::G, NT = S::NT, LD = S::LD;
    const int tid = threadIdx.x, n = tid & 31, g = tid >> 5;
    const int nq = 4 * S::E2, nd = S::E2 * md.m2;
    Real *sW = sm;
    Real *X1 = sW + md.emb.size, *X1d = X1 + S::E0 * LD;
    Real *X2 = X1d + S::E0 * LD, *X2d = X2 + S::E1 * LD;
    Real *Zb = X2d + S::E1 * LD, *Zdb = Zb + S::WMAX * LD;       // reused by each layer
    Real *sR = Zdb + S::WMAX * LD, *sRd = sR + 128;
    Real *sT = sRd + 128, *sTd = sT + nq, *sTb = sTd + nq, *sTdb = sTb + nq;
    Real *stage = Zb;                                             // D_bar / D'_bar staging at atom start
    Real *X3 = Zb, *X3d = Zdb;                                    // layer-3 forward outputs (only t, z' kept)
    Real *gpb = gpriv + (int64_t)blockIdx.x * md.ntypes * md.ntypes * md.emb.size;
    const Real *P = P_of<Real>(md);
    for (int64_t p = blockIdx.x; p < n_atoms; p += gridDim.x) {
        const int i = order[p];
        const Pos4 pi = pos[i];
        const int ti = (int)pi.w;
        __syncthreads();
        for (int q = tid; q < nq; q += NT) {
            sT[q] = Tp[p * nq + q];
            sTd[q] = Tdp[p * nq + q];
        }
        for (int q = tid; q < nd; q += NT) {
            stage[q] = Dbp[p * nd + q];
            stage[nd + q] = Ddbp[p * nd + q];
        }
        __syncthreads();
        // T_bar = f(D_bar, T) + f(D'_bar, T'),  T'_bar = f(D'_bar, T), both times 1/sum(sel)
        const Real inv = (Real)md.inv_nsel;
        for (int q = tid; q < nq; q += NT) {
            const int a = q >> 2, c = q & 3;
            sTb[q] = (desc_adj<Real>(stage, sT, S::E2, md.m2, a, c) + desc_adj<Real>(stage + nd, sTd, S::E2, md.m2, a, c)) * inv;
            sTdb[q] = desc_adj<Real>(stage + nd, sT, S::E2, md.m2, a, c) * inv;
        }
        for (int tj = 0; tj < md.ntypes; ++tj) {
            const int cnt = nnei[(int64_t)i * md.ntypes + tj];
            if (cnt == 0) continue;
            __syncthreads();
            const int net_id = ti * md.ntypes + tj;
            const Real *net = P + md.emb_base + (int64_t)net_id * md.emb.size;
            for (int q = tid; q < md.emb.size; q += NT) sW[q] = net[q];
            Real *gnet = gpb + (int64_t)net_id * md.emb.size;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                if (g == 0) env_tangent<Real>(md, bx, pos, nlist, v, i, pi, tj, c0, cnt, n, sR, sRd);
                __syncthreads();
                Real t0[S::E0 / G], z0[S::E0 / G], t1[S::E1 / G], z1[S::E1 / G], t2[S::E2 / G], z2[S::E2 / G];
                const Real s = sR[n * 4], sd = sRd[n * 4];
                layer0_ft<S, Real>(sW + md.emb.W[0], sW + md.emb.b[0], s, sd, X1, X1d, t0, z0, g, n);
                __syncthreads();
                layer_ft<S, S::E0, S::E1, Real>(sW + md.emb.W[1], sW + md.emb.b[1], X1, X1d, X2, X2d, t1, z1, g, n);
                __syncthreads();
                layer_ft<S, S::E1, S::E2, Real>(sW + md.emb.W[2], sW + md.emb.b[2], X2, X2d, X3, X3d, t2, z2, g, n);
                // G_bar = (T_bar R + T'_bar R') for the owned channels, G'_bar = T'_bar R
                Real gb2[S::E2 / G], gdb2[S::E2 / G];
                const Real R0 = sR[n * 4], R1 = sR[n * 4 + 1], R2 = sR[n * 4 + 2], R3 = sR[n * 4 + 3];
                const Real Q0 = sRd[n * 4], Q1 = sRd[n * 4 + 1], Q2 = sRd[n * 4 + 2], Q3 = sRd[n * 4 + 3];
#pragma unroll
                for (int u = 0; u < S::E2 / G; ++u) {
                    const int m = g + G * u;
                    const Real *tb = sTb + 4 * m, *tdb = sTdb + 4 * m;
                    gb2[u] = tb[0] * R0 + tb[1] * R1 + tb[2] * R2 + tb[3] * R3 + tdb[0] * Q0 + tdb[1] * Q1 +
                             tdb[2] * Q2 + tdb[3] * Q3;
                    gdb2[u] = tdb[0] * R0 + tdb[1] * R1 + tdb[2] * R2 + tdb[3] * R3;
                }
                __syncthreads();   // X3/X3d (aliasing Zb/Zdb) are no longer read
                Real xb1[S::E1 / G], xdb1[S::E1 / G];
                layer_rev<S, S::E1, S::E2, Real>(sW + md.emb.W[2], X2, X2d, Zb, Zdb, gb2, gdb2, t2, z2,
                                                 gnet + md.emb.W[2], gnet + md.emb.b[2], xb1, xdb1, tid, g, n);
                // skip of layer 3 into y2: owned k and k + E1 belong to the same thread
#pragma unroll
                for (int u = 0; u < S::E1 / G; ++u) {
                    if (S::E2 == S::E1) { xb1[u] += gb2[u]; xdb1[u] += gdb2[u]; }
                    else if (S::E2 == 2 * S::E1) {
                        xb1[u] += gb2[u] + gb2[u + S::E1 / G];
                        xdb1[u] += gdb2[u] + gdb2[u + S::E1 / G];
                    }
                }
                __syncthreads();
                Real xb0[S::E0 / G], xdb0[S::E0 / G];
                layer_rev<S, S::E0, S::E1, Real>(sW + md.emb.W[1], X1, X1d, Zb, Zdb, xb1, xdb1, t1, z1,
                                                 gnet + md.emb.W[1], gnet + md.emb.b[1], xb0, xdb0, tid, g, n);
#pragma unroll
                for (int u = 0; u < S::E0 / G; ++u) {
                    if (S::E1 == S::E0) { xb0[u] += xb1[u]; xdb0[u] += xdb1[u]; }
                    else if (S::E1 == 2 * S::E0) {
                        xb0[u] += xb1[u] + xb1[u + S::E0 / G];
                        xdb0[u] += xdb1[u] + xdb1[u + S::E0 / G];
                    }
                }
                __syncthreads();
                // layer 0: input (s, s'); W_bar[0][k] += s z_bar + s' z'_bar, b_bar += z_bar
#pragma unroll
                for (int u = 0; u < S::E0 / G; ++u) {
                    const int o = g + G * u;
                    const Real g1 = Real(1) - t0[u] * t0[u];
                    const Real zdb = xdb0[u] * g1;
                    const Real tb = xb0[u] + xdb0[u] * z0[u] * (Real(-2) * t0[u]);
                    Zb[o * LD + n] = tb * g1;
                    Zdb[o * LD + n] = zdb;
                }
                __syncthreads();
                for (int o = tid; o < S::E0; o += NT) {
                    Real aw = Real(0), abb = Real(0);
                    for (int nn = 0; nn < 32; ++nn) {
                        aw += sR[nn * 4] * Zb[o * LD + nn] + sRd[nn * 4] * Zdb[o * LD + nn];
                        abb += Zb[o * LD + nn];
                    }
                    gnet[md.emb.W[0] + o] += aw;
                    gnet[md.emb.b[0] + o] += abb;
                }
                __syncthreads();
            }
        }
    }
}

// grad[emb part] += sum over the private slices, in slice order.
template <typename Real>
__global__ void __launch_bounds__(256) k_grad_reduce(const Real *__restrict__ gpriv, int nslices, int64_t len,
                                                     double *__restrict__ grad)
{
    // 32 entries per block, the slices split over 8 groups (group g sums slices g, g + 8, ...); the
    // group sums are added in group order, so the result does not depend on the scheduling
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int64_t q = blockIdx.x * (int64_t)32 + lane;
    double acc = 0.0;
    if (q < len)
        for (int s = grp; s < nslices; s += 8) acc += (double)gpriv[(int64_t)s * len + q];
    part[grp][lane] = acc;
    __syncthreads();
    if (grp == 0 && q < len) {
        double sum = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) sum += part[g][lane];
        grad[q] += sum;
    }
}

// Per frame (one block each, fixed-order sums): v = F - F_ref, the frame's
// energy E_f = sum of its E_i, the loss weight alpha_f = 2 p_e (E_f - E_ref,f) / n_f^2
// of dE_f/dtheta, and the frame's loss p_e (dE_f / n_f)^2 + p_f / (3 n_f) sum |F - F_ref|^2;
// beta = -2 p_f / (3 n_f) weighs dEdot/dtheta (Edot along v, since F = -grad E).
__global__ void __launch_bounds__(256) k_loss_frames(int64_t frame_n, const double *__restrict__ F,
                                                    const double *__restrict__ F_ref, const double *__restrict__ Ei,
                                                    const double *__restrict__ E_ref, double p_e, double p_f,
                                                    double *__restrict__ v, double *__restrict__ ab,
                                                    double *__restrict__ lf)
{
    __shared__ double s[2][256];
    const int t = threadIdx.x, f = blockIdx.x;
    const int64_t a0 = (int64_t)f * frame_n;
    double acc = 0.0, e = 0.0;
    for (int64_t q = t; q < 3 * frame_n; q += 256) {
        const double d = F[3 * a0 + q] - F_ref[3 * a0 + q];
        v[3 * a0 + q] = d;
        acc += d * d;
    }
    for (int64_t i = t; i < frame_n; i += 256) e += Ei[a0 + i];
    s[0][t] = acc;
    s[1][t] = e;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) {
            s[0][t] += s[0][t + h];
            s[1][t] += s[1][t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double nn = (double)frame_n, dE = s[1][0] - E_ref[f];
        ab[1 + f] = 2.0 * p_e * dE / (nn * nn);
        lf[f] = p_e * (dE / nn) * (dE / nn) + p_f * s[0][0] / (3.0 * nn);
        if (f == 0) ab[0] = -2.0 * p_f / (3.0 * nn);
    }
}

__global__ void __launch_bounds__(256) k_loss_sum(int nframes, const double *__restrict__ lf, double *__restrict__ loss)
{
    __shared__ double s[256];
    const int t = threadIdx.x;
    double acc = 0.0;
    for (int f = t; f < nframes; f += 256) acc += lf[f];
    s[t] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) s[t] += s[t + h];
        __syncthreads();
    }
    if (t == 0) loss[0] += s[0];
}

template <class S, typename Real>
size_t fwd_smem(const ModelDev &md)
{
    return sizeof(Real) * ((size_t)md.emb.size + 2 * (S::E0 + S::E1 + S::E2) * S::LD + 256 + 8 * S::E2);
}

template <class S, typename Real>
size_t bwd_smem(const ModelDev &md)
{
    size_t zb = (size_t)2 * S::WMAX * S::LD;
    size_t stage = (size_t)2 * S::E2 * md.m2;
    return sizeof(Real) * ((size_t)md.emb.size + 2 * (S::E0 + S::E1) * S::LD + (zb > stage ? zb : stage) + 256 +
                           16 * S::E2);
}

template <class S, typename Real>
dp_status run_grad(dp_model *m, dp_nlist *nl, const double *d_v, const double *d_ab, double *d_E_atom,
                   double *d_Ed_atom, double *d_grad, cudaStream_t st)
{
    m->dev.n_list = nl->n;
    const ModelDev &md = m->dev;
    const int64_t n = nl->n;
    const FitRec fr = make_fit_rec(md);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    // the embedding reverse runs as many persistent CTAs as fit on the SMs at once (each with its own
    // gradient slice): one CTA of a few warps per SM leaves its chains of small products and barriers
    // exposed
    const size_t sf = fwd_smem<S, Real>(md), sb = bwd_smem<S, Real>(md);
    DP_CUDA(cudaFuncSetAttribute(k_jvp_fwd<S, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
    DP_CUDA(cudaFuncSetAttribute(k_jvp_bwd<S, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    int per_sm = 1;
    DP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jvp_bwd<S, Real>, S::NT, sb));
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    const int64_t bwd_atoms = n > 0 ? n : 1;
    const int nslices = (int)std::min<int64_t>((int64_t)nsm * per_sm, bwd_atoms);
    const int64_t emb_len = (int64_t)md.ntypes * md.ntypes * md.emb.size;
    size_t need = 0;
    auto sz = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    sz(sizeof(Real) * 4 * md.m1 * n * 2);
    sz(sizeof(Real) * md.desc_dim * n * 4);
    sz(sizeof(Real) * (size_t)fr.size * n);
    sz(sizeof(Real) * emb_len * nslices);
    // fitting weight gradient: chunks of atoms so that the tiles x chunks fill the GPU
    const WgPlan plan0 = make_wg_plan(md);
    const int wg_tiles = plan0.start[plan0.nlayers];
    auto wg_chunks = [&](int64_t cnt) {
        const int64_t want = (4 * (int64_t)nsm + wg_tiles - 1) / wg_tiles;
        const int64_t most = (cnt + kWgAtoms - 1) / kWgAtoms;
        return want < 1 ? 1 : (want > most ? (most < 1 ? 1 : most) : want);
    };
    sz(sizeof(double) * (size_t)wg_chunks(n) * md.fit.size);
    DP_TRY(ensure_workspace(m, need));
    char *w = m->ws;
    auto carve = [&](size_t bytes) {
        char *p = w;
        w += (bytes + 255) & ~(size_t)255;
        return p;
    };
    Real *T = (Real *)carve(sizeof(Real) * 4 * md.m1 * n * 2), *Td = T + 4 * md.m1 * n;
    Real *D = (Real *)carve(sizeof(Real) * md.desc_dim * n * 4);
    Real *Dd = D + md.desc_dim * n, *Db = Dd + md.desc_dim * n, *Ddb = Db + md.desc_dim * n;
    Real *rec = (Real *)carve(sizeof(Real) * (size_t)fr.size * n);
    Real *gpriv = (Real *)carve(sizeof(Real) * emb_len * nslices);
    double *wg_part = (double *)carve(sizeof(double) * (size_t)wg_chunks(n) * md.fit.size);
    DP_CUDA(cudaMemsetAsync(gpriv, 0, sizeof(Real) * emb_len * nslices, st));
    BoxDev bx = make_box(nl);
    const Pos4 *pos = (const Pos4 *)nl->d_pos;
    {
        ProfScope ps(m->prof, PG_GRAD, 1, st);
        k_jvp_fwd<S, Real><<<(unsigned)n, S::NT, sf, st>>>(md, bx, nl->d_order, pos, nl->d_nlist, nl->d_nnei, d_v, T,
                                                          Td, D, Dd);
    }
    DP_CUDA(cudaGetLastError());
    for (int t = 0; t < md.ntypes; ++t) {
        const int64_t b = nl->type_off[t], cnt = nl->type_count[t];
        if (cnt <= 0) continue;
        ProfScope ps(m->prof, PG_GRAD, 2, st);
        const int64_t fn = nl->frame_n > 0 ? nl->frame_n : n;
        // fitting net: primal + tangent forward, output layer, reverse, as tiled GEMMs over the atoms
        fitg::fit_net_run<Real, true>(md, fr, t, nl->d_order, b, 0, cnt, d_ab, fn, D, Dd, rec, d_E_atom, d_Ed_atom,
                                      Db, Ddb, st);
        WgPlan plan = plan0;
        int64_t nch = wg_chunks(cnt);
        const int64_t per = ((cnt + nch - 1) / nch + kWgAtoms - 1) / kWgAtoms * kWgAtoms;
        nch = (cnt + per - 1) / per;
        plan.chunk = (int)per;
        k_fit_wgrad<Real><<<dim3((unsigned)wg_tiles, (unsigned)nch), kWgThreads, 0, st>>>(
            md, fr, plan, nl->d_order, b, cnt, d_ab, fn, D, Dd, rec, wg_part);
        k_fit_wgrad_reduce<<<(unsigned)((md.fit.size + 255) / 256), 256, 0, st>>>(md, t, wg_part, (int)nch, d_grad);
        DP_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(m->prof, PG_GRAD, 2, st);
        k_jvp_bwd<S, Real><<<(unsigned)nslices, S::NT, sb, st>>>(md, bx, nl->d_order, n, pos, nl->d_nlist,
                                                                 nl->d_nnei, d_v, T, Td, Db, Ddb, gpriv);
        k_grad_reduce<Real><<<(unsigned)((emb_len + 31) / 32), 256, 0, st>>>(gpriv, nslices, emb_len,
                                                                               d_grad + md.emb_base);
    }
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace

DP_BOUNDS_ACCESSOR(bounds_read_grad)

dp_status param_grad_device(dp_model *m, dp_nlist *nl, const double *d_v, const double *d_ab, dp_precision prec,
                            double *d_E_atom, double *d_Ed_atom, double *d_grad, cudaStream_t st)
{
    const int *e = m->dev.emb.wout;
    const bool f64 = prec == DP_FP64;
    if (e[0] == 25)
        return f64 ? run_grad<GWater, double>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st)
                   : run_grad<GWater, float>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st);
    if (e[0] == 8)
        return f64 ? run_grad<GStudent, double>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st)
                   : run_grad<GStudent, float>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st);
    return f64 ? run_grad<GPaper, double>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st)
               : run_grad<GPaper, float>(m, nl, d_v, d_ab, d_E_atom, d_Ed_atom, d_grad, st);
}

dp_status loss_terms_device(int64_t n, int64_t frame_n, const double *d_F, const double *d_F_ref,
                            const double *d_Ei, const double *d_E_ref, double p_e, double p_f, double *d_v,
                            double *d_ab, double *d_lf, double *d_loss, cudaStream_t st)
{
    const int nframes = (int)(n / frame_n);
    k_loss_frames<<<nframes, 256, 0, st>>>(frame_n, d_F, d_F_ref, d_Ei, d_E_ref, p_e, p_f, d_v, d_ab, d_lf);
    k_loss_sum<<<1, 256, 0, st>>>(nframes, d_lf, d_loss);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace dp

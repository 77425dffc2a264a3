// CUDA-core (SIMT) evaluation of the DeepPot-SE energy, forces and virial
// (Sec. 2, Fig. 1) in two of the precision schemes of Sec. 4.1.3:
//   Real = double: the "double" scheme, every step in FP64;
//   Real = float:  MIX-32, nets (embedding, contraction, descriptor,
//                  fitting and their gradients) in FP32 with FP32 weights,
//                  while coordinates, the environment matrix and its
//                  Jacobian, the chain to dE/dd_ij, the force / virial
//                  accumulation and the energy sum stay FP64.
//
// Three kernels per batch of atoms (atoms in type-sorted order so that
// neighboring CTAs share nets):
//   k_embed_fwd  one CTA per atom: environment rows, the embedding net on
//                32-neighbor chunks (one neighbor per lane, output channels
//                split over the CTA's G warps), the contraction
//                T = (1/sum sel) sum_j G_j^T R_j and D = T T<^T.  The tanh
//                values of every layer and the last embedding output are
//                stored for the backward pass (recomputing tanh costs more
//                than the HBM round trip here).
//   k_fit        A atoms per CTA: fitting net forward (E_i) and its input
//                gradient dE/dD, weights read through L2.
//   k_embed_bwd  one CTA per atom: dE/dT, then per chunk dE/dG_j and dE/dR_j,
//                back through the embedding net to dE/ds_j, the chain
//                through the environment row to g_ij = dE_i/dd_ij, and the
//                scatter F_i += g_ij, F_j -= g_ij (FP64 atomics) with the
//                per-atom virial -sum_j d_ij (x) g_ij.
// The MATMUL+SUM and CONCAT+SUM fusions of Sec. 4.2 are the bias and skip
// terms added in registers; TANH and TANHGrad (Sec. 4.2.3) share the stored
// tanh value.
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "fit_gemm.cuh"
#include "geom.cuh"
#include "tanh64.cuh"

namespace dp {
namespace {


__device__ __forceinline__ double act_tanh(double x) { return tanh_f64(x); }
__device__ __forceinline__ float act_tanh(float x) { return tanhf(x); }

template <typename Real>
__device__ __forceinline__ const Real *params_of(const ModelDev &md);
template <>
__device__ __forceinline__ const double *params_of<double>(const ModelDev &md) { return md.p; }
template <>
__device__ __forceinline__ const float *params_of<float>(const ModelDev &md) { return md.p32; }
template <typename Real>
__device__ __forceinline__ const Real *paramsT_of(const ModelDev &md);
template <>
__device__ __forceinline__ const double *paramsT_of<double>(const ModelDev &md) { return md.pT; }
template <>
__device__ __forceinline__ const float *paramsT_of<float>(const ModelDev &md) { return md.pT32; }

// Compile-time embedding shape: three layers of widths E0, E1, E2 (= M1),
// split over G warps (channel o belongs to warp o % G).
template <int G_, int E0_, int E1_, int E2_>
struct EmbShape {
    static constexpr int G = G_, E0 = E0_, E1 = E1_, E2 = E2_;
    static constexpr int WMAX = E2_ > E1_ ? (E2_ > E0_ ? E2_ : E0_) : (E1_ > E0_ ? E1_ : E0_);
    static constexpr int NT = 32 * G_;
    static constexpr int KT = (4 * E2_ + NT - 1) / NT;   // T entries per thread
    static constexpr int ACT = E0_ + E1_ + E2_ + E2_;    // stored per neighbor: t of each layer, then G_j
};

template <typename Real>
__device__ __forceinline__ Real skip_term(int wout, int win, const Real *x, int o, int n)
{
    if (wout == win) return x[o * 32 + n];
    if (wout == 2 * win) return x[(o % win) * 32 + n];
    return Real(0);
}

// One hidden embedding layer for the 32 neighbors of a chunk: y = skip + tanh(x W + b).
template <int G, int WIN, int WOUT, typename Real>
__device__ __forceinline__ void emb_layer_fwd(const Real *__restrict__ sWl, const Real *__restrict__ sbl,
                                              const Real *__restrict__ xin, Real *__restrict__ yout,
                                              Real *__restrict__ act_t, Real *__restrict__ act_y, int g, int n)
{
    constexpr int NO = (WOUT + G - 1) / G;
    Real acc[NO];
#pragma unroll
    for (int u = 0; u < NO; ++u) acc[u] = (g + G * u < WOUT) ? sbl[g + G * u] : Real(0);
#pragma unroll 5
    for (int kk = 0; kk < WIN; ++kk) {
        const Real xv = xin[kk * 32 + n];
        const Real *Wr = sWl + kk * WOUT + g;
#pragma unroll
        for (int u = 0; u < NO; ++u)
            if (WOUT % G == 0 || g + G * u < WOUT) acc[u] += xv * Wr[G * u];
    }
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        const int o = g + G * u;
        if (WOUT % G == 0 || o < WOUT) {
            const Real t = act_tanh(acc[u]);
            const Real y = skip_term(WOUT, WIN, xin, o, n) + t;
            yout[o * 32 + n] = y;
            act_t[o * 32 + n] = t;
            if (act_y) act_y[o * 32 + n] = y;
        }
    }
}

template <class S, typename Real>
__global__ void __launch_bounds__(S::NT) k_embed_fwd(ModelDev md, BoxDev bx, const int32_t *__restrict__ order,
                                                    int64_t p0, const Pos4 *__restrict__ pos,
                                                    const int32_t *__restrict__ nlist, const int32_t *__restrict__ nnei,
                                                    Real *__restrict__ T_out, Real *__restrict__ D_out,
                                                    Real *__restrict__ act)
{
    constexpr int G = S::G, NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *smem = reinterpret_cast<Real *>(smem_raw);
    const int tid = threadIdx.x, n = tid & 31, g = tid >> 5;
    Real *sW = smem;
    Real *sA = sW + md.emb.size;
    Real *sB = sA + S::WMAX * 32;
    Real *sR = sB + S::WMAX * 32;         // [32][4]
    Real *sT = sR + 32 * 4;               // [M1][4]
    const int64_t p = p0 + blockIdx.x;
    const int i = order[p];
    const Pos4 pi = pos[i];
    const int ti = (int)pi.w;
    Real tacc[S::KT];
#pragma unroll
    for (int u = 0; u < S::KT; ++u) tacc[u] = Real(0);
    constexpr int act_chunk = S::ACT * 32;
    Real *act_atom = act + (int64_t)blockIdx.x * md.chunks_per_atom * act_chunk;
    const Real *P = params_of<Real>(md);

    for (int tj = 0; tj < md.ntypes; ++tj) {
        const int cnt = nnei[(int64_t)i * md.ntypes + tj];
        if (cnt == 0) continue;
        __syncthreads();
        const Real *net = P + md.emb_base + (int64_t)(ti * md.ntypes + tj) * md.emb.size;
        for (int q = tid; q < md.emb.size; q += NT) sW[q] = net[q];
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            if (g == 0) {
                double R[4] = {0.0, 0.0, 0.0, 0.0};
                if (c0 + n < cnt) {
                    int j = nlist[(int64_t)i * md.nsel + md.sel_off[tj] + c0 + n];
                    if (DP_IDX_OK(j, md.n_list, BS_NLIST_J)) {
                        double d[3], J[12];
                        double r = min_image_r(pi, pos[j], bx, d);
                        env_row(d, r, md.rcs, md.rcut, md.inv_sw, R, J);
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) sR[n * 4 + c] = (Real)R[c];
            }
            __syncthreads();
            Real *ca = act_atom + (int64_t)(md.chunk_off[tj] + c0 / 32) * act_chunk;
            // layer 0: the input is the scalar s = R[0]
            {
                constexpr int NO = (S::E0 + G - 1) / G;
                const Real s = sR[n * 4];
                const Real *W0 = sW + md.emb.W[0], *b0 = sW + md.emb.b[0];
#pragma unroll
                for (int u = 0; u < NO; ++u) {
                    const int o = g + G * u;
                    if (S::E0 % G == 0 || o < S::E0) {
                        const Real t = act_tanh(b0[o] + s * W0[o]);
                        const Real y = ((S::E0 == 1 || S::E0 == 2) ? s : Real(0)) + t;
                        sA[o * 32 + n] = y;
                        ca[o * 32 + n] = t;
                    }
                }
            }
            __syncthreads();
            emb_layer_fwd<G, S::E0, S::E1, Real>(sW + md.emb.W[1], sW + md.emb.b[1], sA, sB, ca + S::E0 * 32,
                                                 nullptr, g, n);
            __syncthreads();
            emb_layer_fwd<G, S::E1, S::E2, Real>(sW + md.emb.W[2], sW + md.emb.b[2], sB, sA,
                                                 ca + (S::E0 + S::E1) * 32, ca + (S::E0 + S::E1 + S::E2) * 32, g, n);
            __syncthreads();
            // T[m][c] += sum_n G[m][n] R[n][c]
#pragma unroll
            for (int u = 0; u < S::KT; ++u) {
                const int q = tid + u * NT;
                if (q < 4 * S::E2) {
                    const int m = q >> 2, c = q & 3;
                    Real a = Real(0);
#pragma unroll 8
                    for (int nn = 0; nn < 32; ++nn) a += sA[m * 32 + nn] * sR[nn * 4 + c];
                    tacc[u] += a;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < S::KT; ++u) {
        const int q = tid + u * NT;
        if (q < 4 * S::E2) {
            const Real t = tacc[u] * (Real)md.inv_nsel;
            sT[q] = t;
            T_out[(int64_t)blockIdx.x * 4 * S::E2 + q] = t;
        }
    }
    __syncthreads();
    const int nd = S::E2 * md.m2;
    for (int q = tid; q < nd; q += NT) {
        const int a = q / md.m2, b = q - a * md.m2;
        Real v = sT[4 * a] * sT[4 * b] + sT[4 * a + 1] * sT[4 * b + 1];
        v += sT[4 * a + 2] * sT[4 * b + 2] + sT[4 * a + 3] * sT[4 * b + 3];
        D_out[(int64_t)blockIdx.x * nd + q] = v;
    }
}

// Fitting net of center type ti on A atoms (positions pos_begin + A*blockIdx.x
// of the type-sorted order): E_i forward, dE/dD backward.
// OZ: the first layer's products are done elsewhere (FP64 on the tensor
// cores): its pre-activations z1 [count][f0] (bias included) are read, and
// its pre-activation adjoints are written to dz1 [count][f0] instead of
// forming dE/dD here.
template <typename Real, int A, bool OZ>
__global__ void __launch_bounds__(256) k_fit(ModelDev md, int ti, const int32_t *__restrict__ order, int64_t p0,
                                            int64_t pos_begin, int64_t count, const Real *__restrict__ D,
                                            Real *__restrict__ dD, double *__restrict__ E_atom,
                                            const double *__restrict__ z1, double *__restrict__ dz1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *smem = reinterpret_cast<Real *>(smem_raw);
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int nd = md.desc_dim;
    int wmax = 0;
    for (int k = 0; k < md.n_fit; ++k) wmax = max(wmax, md.fit.wout[k]);
    int fsum = 0;
    for (int k = 0; k < md.n_fit; ++k) fsum += md.fit.wout[k];
    Real *sX = smem;                                     // [A][nd] (not with OZ), later dy/dz buffers
    Real *sT = sX + max(OZ ? 0 : A * nd, 3 * A * wmax);  // [A][fsum] tanh values
    Real *sY = sT + A * fsum;                            // [A][fsum] layer outputs
    const int64_t first = pos_begin + (int64_t)blockIdx.x * A;
    const int na = (int)min((int64_t)A, pos_begin + count - first);
    const Real *net = params_of<Real>(md) + md.fit_base + (int64_t)ti * md.fit.size;
    const Real *netT = paramsT_of<Real>(md) + md.fit_base + (int64_t)ti * md.fit.size;

    if (!OZ)
        for (int q = tid; q < A * nd; q += nthreads) {
            int a = q / nd;
            sX[q] = a < na ? D[(first + a - p0) * nd + (q - a * nd)] : Real(0);
        }
    __syncthreads();
    // forward
    const Real *xin = sX;
    int win = nd, off = 0;
    for (int k = 0; k < md.n_fit; ++k) {
        const int wout = md.fit.wout[k];
        const Real *W = net + md.fit.W[k];
        const Real *b = net + md.fit.b[k];
        for (int o = tid; o < wout; o += nthreads) {
            Real acc[A];
            if (OZ && k == 0) {
#pragma unroll
                for (int a = 0; a < A; ++a) acc[a] = a < na ? (Real)z1[(first + a - pos_begin) * wout + o] : Real(0);
            } else {
                const Real bo = __ldg(b + o);
#pragma unroll
                for (int a = 0; a < A; ++a) acc[a] = bo;
#pragma unroll 4
                for (int kk = 0; kk < win; ++kk) {
                    const Real w = __ldg(W + (int64_t)kk * wout + o);
#pragma unroll
                    for (int a = 0; a < A; ++a) acc[a] += xin[a * win + kk] * w;
                }
            }
#pragma unroll
            for (int a = 0; a < A; ++a) {
                Real t = act_tanh(acc[a]);
                Real res = Real(0);
                if (wout == win) res = xin[a * win + o];
                else if (wout == 2 * win) res = xin[a * win + (o % win)];
                sT[a * fsum + off + o] = t;
                sY[a * fsum + off + o] = res + t;
            }
        }
        __syncthreads();
        // the next layer reads dense [A][wout] rows of this layer's outputs
        Real *dense = sX + (k & 1) * A * wmax;
        for (int q = tid; q < A * wout; q += nthreads) {
            int a = q / wout;
            dense[q] = sY[a * fsum + off + (q - a * wout)];
        }
        __syncthreads();
        xin = dense;
        win = wout;
        off += wout;
    }
    // output layer: E = y . w_out + b_out (warp a handles atom a); E_i in FP64
    const Real *Wout = net + md.fit.W[md.n_fit];
    const Real bout = net[md.fit.b[md.n_fit]];
    {
        const int warp = tid >> 5, lane = tid & 31;
        for (int a = warp; a < A; a += nthreads / 32) {
            Real e = Real(0);
            for (int o = lane; o < win; o += 32) e += xin[a * win + o] * __ldg(Wout + o);
            for (int s = 16; s > 0; s >>= 1) e += __shfl_xor_sync(0xffffffffu, e, s);
            if (lane == 0 && a < na) E_atom[order[first + a]] = (double)(e + bout);
        }
    }
    __syncthreads();
    // backward: dy = w_out for the last hidden layer
    Real *dy = sX, *dz = sX + A * wmax, *dyn = sX + 2 * A * wmax;
    for (int q = tid; q < A * win; q += nthreads) dy[q] = __ldg(Wout + (q % win));
    __syncthreads();
    for (int k = md.n_fit - 1; k >= 0; --k) {
        const int wout = md.fit.wout[k];
        const int kin = k == 0 ? nd : md.fit.wout[k - 1];
        off -= wout;
        for (int q = tid; q < A * wout; q += nthreads) {
            int a = q / wout, o = q - a * wout;
            Real t = sT[a * fsum + off + o];
            dz[q] = dy[q] * (Real(1) - t * t);
        }
        __syncthreads();
        if (OZ && k == 0) {
            for (int q = tid; q < A * wout; q += nthreads) {
                const int a = q / wout, o = q - a * wout;
                if (a < na) dz1[(first + a - pos_begin) * wout + o] = (double)dz[q];
            }
            break;
        }
        const Real *WT = netT + md.fit.W[k];             // [wout][kin]
        for (int kk = tid; kk < kin; kk += nthreads) {
            Real acc[A];
#pragma unroll
            for (int a = 0; a < A; ++a) acc[a] = Real(0);
#pragma unroll 4
            for (int o = 0; o < wout; ++o) {
                const Real w = __ldg(WT + (int64_t)o * kin + kk);
#pragma unroll
                for (int a = 0; a < A; ++a) acc[a] += dz[a * wout + o] * w;
            }
#pragma unroll
            for (int a = 0; a < A; ++a) {
                Real v = acc[a];
                if (wout == kin) v += dy[a * wout + kk];
                else if (wout == 2 * kin) v += dy[a * wout + kk] + dy[a * wout + kk + kin];
                if (k == 0) {
                    if (a < na) dD[(first + a - p0) * nd + kk] = v;
                } else {
                    dyn[a * kin + kk] = v;
                }
            }
        }
        __syncthreads();
        Real *tmp = dy; dy = dyn; dyn = tmp;
    }
}

// Input gradient of one hidden embedding layer for a chunk: given dy of the
// layer outputs (registers, channel o = g + G u) and the stored tanh values,
// returns dx of the layer inputs in the same ownership pattern.
template <int G, int WIN, int WOUT, typename Real>
__device__ __forceinline__ void emb_layer_bwd(const Real *__restrict__ sWl, const Real *__restrict__ act_t,
                                              Real *__restrict__ sdz, const Real (&dy)[(WOUT + G - 1) / G],
                                              Real (&dx)[(WIN + G - 1) / G], int g, int n)
{
    constexpr int NO = (WOUT + G - 1) / G, NI = (WIN + G - 1) / G;
    // the skip sources of input kk (outputs kk and kk + WIN) belong to this
    // thread too, since channel o is owned by warp o % G and G divides WIN
    static_assert(WIN % G == 0 || (WOUT != WIN && WOUT != 2 * WIN), "skip sources on another warp");
#pragma unroll
    for (int u = 0; u < NO; ++u) {
        const int o = g + G * u;
        if (WOUT % G == 0 || o < WOUT) {
            const Real t = act_t[o * 32 + n];
            sdz[o * 32 + n] = dy[u] * (Real(1) - t * t);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NI; ++u) dx[u] = Real(0);
#pragma unroll 5
    for (int o = 0; o < WOUT; ++o) {
        const Real z = sdz[o * 32 + n];
        const Real *Wc = sWl + g * WOUT + o;
#pragma unroll
        for (int u = 0; u < NI; ++u)
            if (WIN % G == 0 || g + G * u < WIN) dx[u] += z * Wc[G * u * WOUT];
    }
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        if (WOUT == WIN) dx[u] += dy[u];
        else if (WOUT == 2 * WIN) dx[u] += dy[u] + dy[u + WIN / G];
    }
    __syncthreads();
}

template <class S, typename Real>
__global__ void __launch_bounds__(S::NT) k_embed_bwd(ModelDev md, BoxDev bx, const int32_t *__restrict__ order,
                                                    int64_t p0, const Pos4 *__restrict__ pos,
                                                    const int32_t *__restrict__ nlist, const int32_t *__restrict__ nnei,
                                                    const Real *__restrict__ T_in, const Real *__restrict__ dD_in,
                                                    const Real *__restrict__ act, double *__restrict__ force,
                                                    double *__restrict__ atom_virial)
{
    constexpr int G = S::G, NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, n = tid & 31, g = tid >> 5;
    const int nq = 4 * S::E2, nd = S::E2 * md.m2;
    // FP64 geometry first (8-byte aligned), then the Real buffers
    double *sJ = reinterpret_cast<double *>(smem_raw);   // [32][12]
    double *sd = sJ + 32 * 12;                           // [32][3]
    Real *sW = reinterpret_cast<Real *>(sd + 32 * 3);
    Real *sdz = sW + md.emb.size;          // [WMAX][32] pre-activation adjoints of one layer
    Real *sdy = sdz + S::WMAX * 32;        // [2][32] layer-1 skip adjoints (first layer of width 1 or 2)
    Real *sR = sdy + 2 * 32;               // [32][4]
    Real *sdR = sR + 32 * 4;               // [G][32][4]
    Real *sT = sdR + G * 32 * 4;           // [M1][4]
    Real *sdT = sT + nq;                   // [M1][4]
    const Real *gdD = dD_in + (int64_t)blockIdx.x * nd;   // dE/dD of this atom (read through L1)
    const int64_t p = p0 + blockIdx.x;
    const int i = order[p];
    const Pos4 pi = pos[i];
    const int ti = (int)pi.w;
    const Real *P = params_of<Real>(md);

    for (int q = tid; q < nq; q += NT) sT[q] = T_in[(int64_t)blockIdx.x * nq + q];
    __syncthreads();
    // dE/dT[m][c] = sum_b dD[m][b] T[b][c] + [m < M2] sum_a dD[a][m] T[a][c], times 1/sum(sel)
    for (int q = tid; q < nq; q += NT) {
        const int m = q >> 2, c = q & 3;
        Real acc = Real(0);
        for (int b = 0; b < md.m2; ++b) acc += __ldg(gdD + m * md.m2 + b) * sT[b * 4 + c];
        if (m < md.m2)
            for (int a = 0; a < S::E2; ++a) acc += __ldg(gdD + a * md.m2 + m) * sT[a * 4 + c];
        sdT[q] = acc * (Real)md.inv_nsel;
    }
    constexpr int act_chunk = S::ACT * 32;
    const Real *act_atom = act + (int64_t)blockIdx.x * md.chunks_per_atom * act_chunk;
    double fi[3] = {0.0, 0.0, 0.0};
    double vir[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) vir[q] = 0.0;

    for (int tj = 0; tj < md.ntypes; ++tj) {
        const int cnt = nnei[(int64_t)i * md.ntypes + tj];
        if (cnt == 0) continue;
        __syncthreads();
        const Real *net = P + md.emb_base + (int64_t)(ti * md.ntypes + tj) * md.emb.size;
        for (int q = tid; q < md.emb.size; q += NT) sW[q] = net[q];
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            int j = -1;
            if (g == 0) {
                double R[4] = {0, 0, 0, 0}, J[12], d[3] = {0, 0, 0};
#pragma unroll
                for (int q = 0; q < 12; ++q) J[q] = 0.0;
                if (c0 + n < cnt) {
                    j = nlist[(int64_t)i * md.nsel + md.sel_off[tj] + c0 + n];
                    if (DP_IDX_OK(j, md.n_list, BS_NLIST_J)) {
                        double r = min_image_r(pi, pos[j], bx, d);
                        env_row(d, r, md.rcs, md.rcut, md.inv_sw, R, J);
                    } else {
                        j = -1;
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) sR[n * 4 + c] = (Real)R[c];
#pragma unroll
                for (int q = 0; q < 12; ++q) sJ[n * 12 + q] = J[q];
#pragma unroll
                for (int q = 0; q < 3; ++q) sd[n * 3 + q] = d[q];
            }
            __syncthreads();
            const Real *ca = act_atom + (int64_t)(md.chunk_off[tj] + c0 / 32) * act_chunk;
            // dE/dG_j for the owned channels and the partial dE/dR_j
            constexpr int N2 = (S::E2 + G - 1) / G, N1 = (S::E1 + G - 1) / G, N0 = (S::E0 + G - 1) / G;
            Real dy2[N2];
            Real dRp[4] = {Real(0), Real(0), Real(0), Real(0)};
            const Real R0 = sR[n * 4], R1 = sR[n * 4 + 1], R2 = sR[n * 4 + 2], R3 = sR[n * 4 + 3];
            const Real *cy = ca + (S::E0 + S::E1 + S::E2) * 32;
#pragma unroll
            for (int u = 0; u < N2; ++u) {
                const int m = g + G * u;
                if (S::E2 % G == 0 || m < S::E2) {
                    const Real *dt = sdT + 4 * m;
                    dy2[u] = dt[0] * R0 + dt[1] * R1 + dt[2] * R2 + dt[3] * R3;
                    const Real y = cy[m * 32 + n];
                    dRp[0] += dt[0] * y;
                    dRp[1] += dt[1] * y;
                    dRp[2] += dt[2] * y;
                    dRp[3] += dt[3] * y;
                } else {
                    dy2[u] = Real(0);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) sdR[(g * 32 + n) * 4 + c] = dRp[c];
            Real dy1[N1], dy0[N0];
            emb_layer_bwd<G, S::E1, S::E2, Real>(sW + md.emb.W[2], ca + (S::E0 + S::E1) * 32, sdz, dy2, dy1, g, n);
            emb_layer_bwd<G, S::E0, S::E1, Real>(sW + md.emb.W[1], ca + S::E0 * 32, sdz, dy1, dy0, g, n);
            // layer 0 (input width 1): ds = sum_o dz_o W0[o] (+ skip when E0 is 1 or 2)
#pragma unroll
            for (int u = 0; u < N0; ++u) {
                const int o = g + G * u;
                if (S::E0 % G == 0 || o < S::E0) {
                    const Real t = ca[o * 32 + n];
                    sdz[o * 32 + n] = dy0[u] * (Real(1) - t * t);
                    if (S::E0 <= 2) sdy[o * 32 + n] = dy0[u];
                }
            }
            __syncthreads();
            if (g == 0 && c0 + n < cnt) {
                const Real *W0 = sW + md.emb.W[0];
                Real ds = Real(0);
                for (int o = 0; o < S::E0; ++o) ds += sdz[o * 32 + n] * W0[o];
                if (S::E0 == 1) ds += sdy[n];
                else if (S::E0 == 2) ds += sdy[n] + sdy[32 + n];
                // from here on FP64: dE/dR_j, the Jacobian chain, forces and virial
                double dR[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    Real a = Real(0);
#pragma unroll
                    for (int gg = 0; gg < G; ++gg) a += sdR[(gg * 32 + n) * 4 + c];
                    dR[c] = (double)a;
                }
                dR[0] += (double)ds;
                const double *J = sJ + n * 12;
                double gv[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) gv[k] = dR[0] * J[k] + dR[1] * J[3 + k] + dR[2] * J[6 + k] + dR[3] * J[9 + k];
                const double *dv = sd + n * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    fi[k] += gv[k];
                    if (j >= 0) acc_add(md.fx, force, 3 * (int64_t)j + k, -gv[k]);
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) vir[3 * a + b] -= dv[a] * gv[b];
            }
            __syncthreads();
        }
    }
    if (g == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            for (int s = 16; s > 0; s >>= 1) fi[k] += __shfl_xor_sync(0xffffffffu, fi[k], s);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            for (int s = 16; s > 0; s >>= 1) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], s);
        if (n == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) acc_add(md.fx, force, 3 * (int64_t)i + k, fi[k]);
        }
        if (n < 9 && atom_virial) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < 9; ++q) v = (q == n) ? vir[q] : v;
            atom_virial[9 * (int64_t)i + n] = v;
        }
    }
}

template <class S, typename Real>
size_t embed_fwd_smem(const ModelDev &md)
{
    return sizeof(Real) * ((size_t)md.emb.size + 2 * S::WMAX * 32 + 32 * 4 + 4 * S::E2);
}

template <class S, typename Real>
size_t embed_bwd_smem(const ModelDev &md)
{
    return sizeof(double) * 32 * (12 + 3) +
           sizeof(Real) * ((size_t)md.emb.size + S::WMAX * 32 + 2 * 32 + 32 * 4 + S::G * 32 * 4 + 8 * S::E2);
}

template <typename Real>
size_t fit_smem(const ModelDev &md, int A, bool oz = false)
{
    int wmax = 0, fsum = 0;
    for (int k = 0; k < md.n_fit; ++k) {
        wmax = wmax > md.fit.wout[k] ? wmax : md.fit.wout[k];
        fsum += md.fit.wout[k];
    }
    size_t a = oz ? 0 : (size_t)A * md.desc_dim, b = (size_t)3 * A * wmax;
    return sizeof(Real) * ((a > b ? a : b) + 2 * (size_t)A * fsum);
}

template <typename Real, int A, bool OZ>
dp_status launch_fit_a(dp_model *m, const int32_t *order, int t, int64_t p0, int64_t b, int64_t count,
                       const Real *D, Real *dD, double *E_atom, const double *z1, double *dz1, cudaStream_t st)
{
    const size_t sfit = fit_smem<Real>(m->dev, A, OZ);
    const unsigned tiles = (unsigned)((count + A - 1) / A);
    DP_CUDA(cudaFuncSetAttribute(k_fit<Real, A, OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sfit));
    k_fit<Real, A, OZ><<<tiles, 256, sfit, st>>>(m->dev, t, order, p0, b, count, D, dD, E_atom, z1, dz1);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// Launches the fitting net of type t over `count` type-sorted positions from
// `b`.  Atoms per CTA A: when 6 per CTA would leave SMs idle, each CTA gets
// an SM of its own and the time goes with A, so A in {1, 2, 4, 6} minimises
// ceil(ceil(count / A) / SMs) * A (ties to the larger A, whose weight loads
// serve more atoms).  Otherwise A in 6..9 minimises (waves x A) with the
// CTAs that fit on an SM at once, since the kernel is arithmetic bound and a
// partly filled last wave idles SMs.
template <typename Real, bool OZ>
dp_status launch_fit_oz(dp_model *m, const int32_t *order, int t, int64_t p0, int64_t b, int64_t count,
                        const Real *D, Real *dD, double *E_atom, const double *z1, double *dz1, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    int bestA = 0;
    long best = -1;
    if (count < 6L * nsm) {
        for (int A : {1, 2, 4, 6}) {
            if (fit_smem<Real>(md, A, OZ) > 227 * 1024) continue;
            const long tiles = (long)((count + A - 1) / A);
            const long cost = ((tiles + nsm - 1) / nsm) * A;
            if (best < 0 || cost <= best) { best = cost; bestA = A; }
        }
    } else {
        for (int A = 6; A <= 9; ++A) {
            const size_t sm = fit_smem<Real>(md, A, OZ);
            if (sm > 227 * 1024) continue;
            const long fit = (long)((228 * 1024) / (sm + 1024));
            const long per_sm = fit < 1 ? 1 : (fit > 8 ? 8 : fit);
            const long tiles = (long)((count + A - 1) / A);
            const long slots = (long)nsm * per_sm;
            const long cost = ((tiles + slots - 1) / slots) * A;
            if (best < 0 || cost < best) { best = cost; bestA = A; }
        }
    }
    if (bestA == 0) {
        set_error("fitting net too wide for the shared-memory tile");
        return DP_ERR_UNSUPPORTED;
    }
    switch (bestA) {
    case 1: return launch_fit_a<Real, 1, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    case 2: return launch_fit_a<Real, 2, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    case 4: return launch_fit_a<Real, 4, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    case 6: return launch_fit_a<Real, 6, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    case 7: return launch_fit_a<Real, 7, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    case 8: return launch_fit_a<Real, 8, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    default: return launch_fit_a<Real, 9, OZ>(m, order, t, p0, b, count, D, dD, E_atom, z1, dz1, st);
    }
}

// Launches the fitting net of type t over `count` type-sorted positions from
// `b`.  Atoms per CTA A: when 6 per CTA would leave SMs idle, each CTA gets
// an SM of its own and the time goes with A, so A in {1, 2, 4, 6} minimises
// ceil(ceil(count / A) / SMs) * A (ties to the larger A, whose weight loads
// serve more atoms).  Otherwise A in 6..9 minimises (waves x A) with the
// CTAs that fit on an SM at once, since the kernel is arithmetic bound and a
// partly filled last wave idles SMs.
//
// MIX-32 (frec given): the layers as tiled GEMMs over the type's atoms instead (fit_gemm.cuh), with
// the per-atom record frec [batch][FitRec size] holding each layer's inputs, t and adjoints.
template <typename Real>
dp_status launch_fit(dp_model *m, const int32_t *order, int t, int64_t p0, int64_t b, int64_t count, const Real *D, Real *dD,
                     double *E_atom, Real *frec, cudaStream_t st)
{
    if (frec) {
        const ModelDev &md = m->dev;
        ProfScope ps(m->prof, PG_FIT, 3 * md.n_fit + 1, st);
        fitg::fit_net_run<Real, false>(md, fitg::make_fit_rec(md), t, order, b, p0, count, nullptr, 1, D, nullptr,
                                       frec, E_atom, nullptr, dD, nullptr, st);
        DP_CUDA(cudaGetLastError());
        return DP_OK;
    }
    ProfScope ps(m->prof, PG_FIT, 1, st);
    return launch_fit_oz<Real, false>(m, order, t, p0, b, count, D, dD, E_atom, nullptr, nullptr, st);
}

// The first fitting layer of the FP64 scheme as FP64 products on the tensor
// cores (ozaki.cu): digits of W1 (6-bit, rows of W1^T, for z1 = D W1) and of
// W1^T (7-bit, rows of W1, for dE/dD = dz1 W1^T) per center type.
constexpr int kOzSF = 9, kOzBF = 6, kOzSB = 8, kOzBB = 7;
// Below this many atoms (of a type, for the fitting net; in all, for the
// embedding net) the split products cannot fill the GPU and the CUDA-core
// kernels are faster (1024; DP_OZ_MIN_ATOMS overrides it, e.g. for tests of
// the split route on small systems).
int64_t oz_min_atoms()
{
    const char *v = getenv("DP_OZ_MIN_ATOMS");
    return v ? atoll(v) : 1024;
}

// z1 = D W1 over K = nd is taken in kp ranges of kh columns (the last one
// shorter), each at most 1808 long so that its FP32 digit sums stay exact
// (9 digits of 6 bits: 9 K 2^10 <= 2^24), and summed in FP64.
int oz_kparts(int nd, int *kh)
{
    const int kp = (nd + 1807) / 1808;
    *kh = ((nd + kp - 1) / kp + 15) / 16 * 16;
    return kp;
}

bool oz_fit_ok(const ModelDev &md)
{
    const int f0 = md.fit.wout[0], nd = md.desc_dim;
    return f0 % 48 == 0 && f0 <= 256 && nd % 64 == 0 && getenv("DP_NO_OZAKI") == nullptr;
}

size_t oz_weight_halves(const ModelDev &md)
{
    return (size_t)(kOzSF + kOzSB) * md.fit.wout[0] * md.desc_dim;
}

dp_status oz_refresh_weights(dp_model *m, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int f0 = md.fit.wout[0], nd = md.desc_dim;
    int kh;
    const int kp = oz_kparts(nd, &kh);
    if (!m->d_ozw) {
        DP_CUDA(cudaMalloc(&m->d_ozw, sizeof(__half) * oz_weight_halves(md) * md.ntypes));
        DP_CUDA(cudaMalloc((void **)&m->d_oze, sizeof(int) * (size_t)(kp * f0 + nd) * md.ntypes));
        ++m->epoch;
        m->oz_stale = true;
    }
    if (!m->oz_stale) return DP_OK;
    for (int t = 0; t < md.ntypes; ++t) {
        __half *wf = (__half *)m->d_ozw + oz_weight_halves(md) * t, *wb = wf + (size_t)kOzSF * f0 * nd;
        int *ef = m->d_oze + (size_t)(kp * f0 + nd) * t, *eb = ef + kp * f0;
        const int64_t W0 = md.fit_base + (int64_t)t * md.fit.size + md.fit.W[0];
        for (int q = 0, k0 = 0; q < kp; ++q, k0 += kh) {   // rows of W1^T, per K range
            const int kq = nd - k0 < kh ? nd - k0 : kh;
            DP_TRY((oz_split<kOzSF, kOzBF>(md.pT + W0 + k0, nd, f0, f0, kq, kq, 48, 16, wf + (size_t)kOzSF * f0 * k0,
                                           ef + q * f0, st)));
        }
        DP_TRY((oz_split<kOzSB, kOzBB>(md.p + W0, f0, nd, nd, f0, f0, 64, 16, wb, eb, st)));    // rows of W1
    }
    m->oz_stale = false;
    return DP_OK;
}

// Scratch of the split-product fitting net for nb atoms (rows padded per type).
size_t oz_bytes(const ModelDev &md, int64_t nb)
{
    const int64_t rows = nb + 128 * md.ntypes;
    const int f0 = md.fit.wout[0], nd = md.desc_dim;
    return sizeof(__half) * rows * (size_t)(kOzSF * nd + kOzSB * f0) + sizeof(int) * rows * 2 +
           sizeof(double) * rows * 2 * f0 + 6 * 256 + (oz_fit_chain_ok(md) ? oz_fit_chain_bytes(md, rows) : 0);
}

dp_status fit_fp64_oz(dp_model *m, dp_nlist *nl, int t, int64_t p0, int64_t b, int64_t count, const double *D,
                      double *dD, double *E_atom, char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int f0 = md.fit.wout[0], nd = md.desc_dim;
    const int64_t rows_pad = (count + 127) / 128 * 128;
    auto carve = [&](size_t bytes) {
        char *p = scratch;
        scratch += (bytes + 255) & ~(size_t)255;
        return p;
    };
    int kh;
    const int kp = oz_kparts(nd, &kh);
    __half *da = (__half *)carve(sizeof(__half) * rows_pad * kOzSF * kh);
    __half *db = (__half *)carve(sizeof(__half) * rows_pad * kOzSB * f0);
    int *ea = (int *)carve(sizeof(int) * rows_pad), *eb = (int *)carve(sizeof(int) * rows_pad);
    double *z1 = (double *)carve(sizeof(double) * count * f0), *dz1 = (double *)carve(sizeof(double) * count * f0);
    const __half *wf = (const __half *)m->d_ozw + oz_weight_halves(md) * t, *wb = wf + (size_t)kOzSF * f0 * nd;
    const int *ef = m->d_oze + (size_t)(kp * f0 + nd) * t, *eb2 = ef + kp * f0;
    const double *b1 = md.p + md.fit_base + (int64_t)t * md.fit.size + md.fit.b[0];
    const bool chain = oz_fit_chain_ok(md);
    ProfScope ps(m->prof, PG_FIT, (chain ? 13 : 5) + 2 * (kp - 1), st);
    for (int q = 0, k0 = 0; q < kp; ++q, k0 += kh) {   // z1 = sum over the K ranges, the bias with the first
        const int kq = nd - k0 < kh ? nd - k0 : kh;
        DP_TRY((oz_split<kOzSF, kOzBF>(D + (b - p0) * nd + k0, nd, count, rows_pad, kq, kq, 128, 16, da, ea, st)));
        DP_TRY((oz_gemm<kOzSF, kOzBF, 48, 16>(m, count, f0, kq, da, ea, rows_pad, wf + (size_t)kOzSF * f0 * k0,
                                              ef + q * f0, b1, z1, f0, st, q > 0)));
    }
    if (chain)   // the hidden layers after the first as split products too
        DP_TRY(oz_fit_chain(m, t, nl->d_order, b, count, z1, dz1, E_atom, scratch, st));
    else
        DP_TRY((launch_fit_oz<double, true>(m, nl->d_order, t, p0, b, count, D, dD, E_atom, z1, dz1, st)));
    DP_TRY((oz_split<kOzSB, kOzBB>(dz1, f0, count, rows_pad, f0, f0, 128, 16, db, eb, st)));
    return oz_gemm<kOzSB, kOzBB, 64, 16>(m, count, nd, f0, db, eb, rows_pad, wb, eb2, nullptr, dD + (b - p0) * nd, nd,
                                        st);
}

template <class S, typename Real>
dp_status launch_batch(dp_model *m, dp_nlist *nl, BoxDev bx, int64_t p0, int64_t nb, Real *T, Real *D, Real *dD,
                       Real *act, double *E_atom, double *force, double *atom_virial, char *oz_scratch,
                       char *ozemb_scratch, Real *frec, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    size_t sf = embed_fwd_smem<S, Real>(md), sb = embed_bwd_smem<S, Real>(md);
    DP_CUDA(cudaFuncSetAttribute(k_embed_fwd<S, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
    DP_CUDA(cudaFuncSetAttribute(k_embed_bwd<S, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    const Pos4 *pos = (const Pos4 *)nl->d_pos;
    if (ozemb_scratch) {
        DP_TRY(oz_emb_fwd(m, nl, bx, p0, nb, (double *)T, (double *)D, (double *)act, ozemb_scratch, st));
    } else {
        ProfScope ps(m->prof, PG_EMBED_FWD, 1, st);
        k_embed_fwd<S, Real><<<(unsigned)nb, S::NT, sf, st>>>(md, bx, nl->d_order, p0, pos, nl->d_nlist, nl->d_nnei,
                                                              T, D, act);
    }
    DP_CUDA(cudaGetLastError());
    for (int t = 0; t < md.ntypes; ++t) {
        int64_t b = nl->type_off[t] > p0 ? nl->type_off[t] : p0;
        int64_t e = nl->type_off[t] + nl->type_count[t];
        if (e > p0 + nb) e = p0 + nb;
        if (e <= b) continue;
        if (oz_scratch && e - b >= oz_min_atoms())
            DP_TRY(fit_fp64_oz(m, nl, t, p0, b, e - b, (const double *)D, (double *)dD, E_atom, oz_scratch, st));
        else
            DP_TRY(launch_fit<Real>(m, nl->d_order, t, p0, b, e - b, D, dD, E_atom, frec, st));
    }
    if (ozemb_scratch) {
        DP_TRY(oz_emb_bwd(m, nl, bx, nb, (const double *)T, (const double *)dD, (const double *)act, force,
                          atom_virial, ozemb_scratch, st));
    } else {
        ProfScope ps(m->prof, PG_EMBED_BWD, 1, st);
        k_embed_bwd<S, Real><<<(unsigned)nb, S::NT, sb, st>>>(md, bx, nl->d_order, p0, pos, nl->d_nlist, nl->d_nnei,
                                                              T, dD, act, force, atom_virial);
    }
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

using ShapeWater = EmbShape<5, 25, 50, 100>;   // also copper: the (25, 50, 100) nets
using ShapeStudent = EmbShape<4, 8, 16, 32>;
using ShapePaper = EmbShape<4, 32, 64, 128>;   // the nets of the paper's production models (Sec. 5.1)

template <typename Real>
size_t bytes_per_atom(const ModelDev &md)
{
    return sizeof(Real) * ((size_t)4 * md.m1 + 2 * (size_t)md.desc_dim +
                           (size_t)md.chunks_per_atom * md.act_stride * 32);
}

template <typename Real>
dp_status compute_simt(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                       double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int64_t n = nl->n;
    const size_t per_atom = bytes_per_atom<Real>(md);
    int64_t B = m->batch_atoms > 0 ? m->batch_atoms : n;
    if (B > n) B = n;
    if (B < 1) B = 1;
    B = (n + (n + B - 1) / B - 1) / ((n + B - 1) / B);   // equal batches: no small tail batch
    const bool oz = sizeof(Real) == sizeof(double) && oz_fit_ok(md);
    // the split-product embedding pays off once the tiles fill the GPU; small systems keep the
    // one-CTA-per-atom kernels
    const bool ozemb = sizeof(Real) == sizeof(double) && oz_emb_ok(md) && n >= oz_min_atoms();
    if (oz) DP_TRY(oz_refresh_weights(m, st));
    if (oz && oz_fit_chain_ok(md)) DP_TRY(oz_fit_chain_refresh(m, st));
    if (ozemb) DP_TRY(oz_emb_refresh(m, st));
    // MIX-32: the fitting net runs as GEMMs over the atoms with a per-atom record (fit_gemm.cuh)
    const size_t frec_bytes = sizeof(Real) == sizeof(float) ? sizeof(Real) * (size_t)fitg::make_fit_rec(md).size * B : 0;
    DP_TRY(ensure_workspace(m, per_atom * (size_t)B + 256 * 6 + (oz ? oz_bytes(md, B) : 0) +
                                   (ozemb ? oz_emb_bytes(md, B) : 0) + frec_bytes));
    char *w = m->ws;
    auto carve = [&](size_t bytes) {
        char *p = w;
        w += (bytes + 255) & ~(size_t)255;
        return p;
    };
    Real *T = (Real *)carve(sizeof(Real) * 4 * md.m1 * B);
    Real *D = (Real *)carve(sizeof(Real) * md.desc_dim * B);
    Real *dD = (Real *)carve(sizeof(Real) * md.desc_dim * B);
    Real *act = (Real *)carve(sizeof(Real) * (size_t)md.chunks_per_atom * md.act_stride * 32 * B);
    char *ozs = oz ? carve(oz_bytes(md, B)) : nullptr;
    char *ozes = ozemb ? carve(oz_emb_bytes(md, B)) : nullptr;
    Real *frec = frec_bytes ? (Real *)carve(frec_bytes) : nullptr;
    DP_CUDA(cudaMemsetAsync(d_force, 0, sizeof(double) * 3 * n, st));
    if (ozemb) DP_CUDA(cudaMemsetAsync(d_atom_virial, 0, sizeof(double) * 9 * n, st));   // accumulated per chunk
    // deterministic mode: the scatters go to fixed-point limbs (F, and W_i where it is accumulated
    // per chunk), converted to FP64 after the last batch
    struct LimbScope {
        ModelDev &d;
        ~LimbScope() { d.fx = d.fxv = nullptr; }
    } limb_scope{m->dev};
    if (m->deterministic) {
        const size_t need = (size_t)36 * (size_t)n;
        if (nl->fx_cap < need) {
            cudaFree(nl->d_fx);
            nl->d_fx = nullptr;
            nl->fx_cap = 0;
            DP_CUDA(cudaMalloc((void **)&nl->d_fx, need * sizeof(unsigned long long)));
            nl->fx_cap = need;
        }
        DP_CUDA(cudaMemsetAsync(nl->d_fx, 0, need * sizeof(unsigned long long), st));
        m->dev.fx = nl->d_fx;
        m->dev.fxv = ozemb ? nl->d_fx + (size_t)9 * n : nullptr;
    }
    BoxDev bx = make_box(nl);
    const int *e = md.emb.wout;
    for (int64_t p0 = 0; p0 < n; p0 += B) {
        int64_t nb = n - p0 < B ? n - p0 : B;
        dp_status s;
        if (e[0] == 25)
            s = launch_batch<ShapeWater, Real>(m, nl, bx, p0, nb, T, D, dD, act, d_atom_energy, d_force, d_atom_virial, ozs, ozes, frec, st);
        else if (e[0] == 8)
            s = launch_batch<ShapeStudent, Real>(m, nl, bx, p0, nb, T, D, dD, act, d_atom_energy, d_force, d_atom_virial, ozs, ozes, frec, st);
        else
            s = launch_batch<ShapePaper, Real>(m, nl, bx, p0, nb, T, D, dD, act, d_atom_energy, d_force, d_atom_virial, ozs, ozes, frec, st);
        if (s != DP_OK) return s;
    }
    if (m->dev.fx) {
        DP_TRY(fx_finish(3 * n, m->dev.fx, d_force, st));
        if (m->dev.fxv) DP_TRY(fx_finish(9 * n, m->dev.fxv, d_atom_virial, st));
    }
    ProfScope ps(m->prof, PG_REDUCE, 1, st);
    return reduce_energy_virial(d_atom_energy, d_atom_virial, centers_of(nl), d_energy, d_virial, m->d_red, st);
}

}  // namespace

DP_BOUNDS_ACCESSOR(bounds_read_simt)

// Embedding shapes compiled into the SIMT and tensor-core kernels.
bool embed_shape_supported(int n_embed, const int *e)
{
    if (n_embed != 3) return false;
    return (e[0] == 25 && e[1] == 50 && e[2] == 100) || (e[0] == 8 && e[1] == 16 && e[2] == 32) ||
           (e[0] == 32 && e[1] == 64 && e[2] == 128) || embed_is_wide(n_embed, e);
}

size_t fp64_bytes_per_atom(const ModelDev &md)
{
    // plus the first fitting layer's digits and pre-activations on the tensor-core route
    size_t oz = oz_fit_ok(md) ? sizeof(__half) * (size_t)(kOzSF * md.desc_dim + kOzSB * md.fit.wout[0]) +
                                    2 * sizeof(int) + 2 * sizeof(double) * md.fit.wout[0]
                              : 0;
    if (oz && oz_fit_chain_ok(md)) oz += (oz_fit_chain_bytes(md, 2048) - oz_fit_chain_bytes(md, 1024)) / 1024 + 1;
    // and the split-product embedding's buffers (affine in the batch size)
    const size_t ozemb = oz_emb_ok(md) ? (oz_emb_bytes(md, 2048) - oz_emb_bytes(md, 1024)) / 1024 + 1 : 0;
    return bytes_per_atom<double>(md) + oz + ozemb;
}

dp_status fit_f32(dp_model *m, dp_nlist *nl, const float *D, float *dD, double *d_atom_energy, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    for (int t = 0; t < md.ntypes; ++t) {
        const int64_t b = nl->type_off[t], cnt = nl->type_count[t];
        if (cnt <= 0) continue;
        DP_TRY(launch_fit<float>(m, nl->d_order, t, 0, b, cnt, D, dD, d_atom_energy, nullptr, st));
    }
    return DP_OK;
}

dp_status compute_fp64(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                       double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    return compute_simt<double>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
}

dp_status compute_mix32(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                        double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    return compute_simt<float>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
}

}  // namespace dp

namespace dp {
namespace {

__global__ void k_tanh_f64(int64_t n, const double *__restrict__ x, double *__restrict__ y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = tanh_f64(x[i]);
}

}  // namespace
}  // namespace dp

extern "C" dp_status dp_tanh_f64_dev(int64_t n, const double *d_x, double *d_y, void *stream)
{
    if (n < 0 || (n > 0 && (!d_x || !d_y))) {
        dp::set_error("dp_tanh_f64_dev: bad argument");
        return DP_ERR_ARG;
    }
    if (n == 0) return DP_OK;
    dp::k_tanh_f64<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, d_x, d_y);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dp::set_error("dp_tanh_f64_dev: %s", cudaGetErrorString(e));
        return DP_ERR_CUDA;
    }
    return DP_OK;
}

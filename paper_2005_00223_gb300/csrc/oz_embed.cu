// Embedding net forward of the double-precision scheme (Sec. 2, Fig. 1(c,e,f))
// with its widest layer (E1 -> E2 channels, the bulk of the multiply-adds)
// as FP64 products on the tensor cores by error-free splitting (ozaki.cuh).
//
// Per batch of atoms (type-sorted positions [p0, p0 + nb)), over a work list
// of 32-neighbor chunks grouped into tiles of 128 rows (one neighbor per
// row) that never mix nets:
//   k_ozf_front  one thread per row: environment row R (FP64), layer 0 and
//                layer 1 (E0 -> E1, FP64 with the library's tanh), the tanh
//                values stored for the backward pass, x2 (the layer-1
//                output), R, and the fp16 digits of x2 with their row scale;
//   oz::k_gemm   z3 = x2 W2 from the digits of x2 and of W2^T (per net), and
//                in its epilogue (8 warps, two per row quarter, alternate
//                groups of 8 channels) t3 = tanh(z3 + b2), the
//                embedding output G = skip(x2) + t3, both stored for the
//                backward pass, and the chunk's part of the contraction
//                sum_j G_j^T R_j (a 32-row sum per chunk, in row order);
//   k_ozf_T      per atom: T = (1/sum sel) sum over its chunks (type, then
//                chunk order) and D = T T<^T.
// Results agree with the FP64 SIMT kernel to the rounding of the split
// product (about K 2^-52 of |x2|_max |W2|_max per entry).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "geom.cuh"
#include "ozaki.cuh"
#include "tanh64.cuh"

namespace dp {
namespace {

template <int E0_, int E1_, int E2_>
struct OzEmb {
    static constexpr int E0 = E0_, E1 = E1_, E2 = E2_;
    static constexpr int S = 8, BETA = 7, NC = 64, KC = 16;
    static constexpr int KP = (E1 + 15) / 16 * 16;   // padded K of z3 = x2 W2
    static constexpr int NN = (E2 + NC - 1) / NC;    // units of 64 output channels
    static constexpr int ACT = E0 + E1 + E2 + E2;    // stored per neighbor: t of each layer, then G
    static constexpr int WSM = 2 * E0 + E0 * E1 + E1;
    static constexpr int EPI = 26624;                // epilogue: G [8][8][33] and R [8][4][33] doubles
    using Sh = oz::Shape<S, BETA, NC, KC, EPI>;
    static_assert(8 * (8 + 4) * 33 * 8 <= EPI, "epilogue shared memory");
    // backward: dE/dx2 = dz3 W2^T, K = E2 padded, one unit of 64 >= E1 channels
    static constexpr int KP2 = (E2 + 15) / 16 * 16;
    static constexpr int WSM2 = E0 + E0 * E1;        // W0, W1 of the backward epilogue
    static constexpr int EPI2 = ((WSM2 + 4 * E0 * 32) * 8 + 16 + 1023) / 1024 * 1024;
    using Sh2 = oz::Shape<S, BETA, NC, KC, EPI2>;
    static_assert(E1 <= NC, "one unit of dE/dx2 channels");
    static_assert((long long)S * KP2 * (1LL << (2 * BETA - 2)) <= (1LL << 24), "exact FP32 digit sums");
    static_assert((long long)S * KP * (1LL << (2 * BETA - 2)) <= (1LL << 24), "exact FP32 digit sums");
};

template <class O>
__global__ void __launch_bounds__(128, 2) k_ozf_front(ModelDev md, BoxDev bx, const Pos4 *__restrict__ pos,
                                                      const int32_t *__restrict__ nlist,
                                                      const int32_t *__restrict__ nnei,
                                                      const int4 *__restrict__ chunks, const int *__restrict__ ntiles_dev,
                                                      double *__restrict__ act, __half *__restrict__ dig,
                                                      int *__restrict__ eA, double *__restrict__ x2buf,
                                                      double *__restrict__ Rbuf)
{
    constexpr int E0 = O::E0, E1 = O::E1;
    __shared__ double sW[O::WSM];   // W0 [E0], b0 [E0], W1 [E0][E1], b1 [E1]
    const double *W0 = sW, *b0 = sW + E0, *W1 = sW + 2 * E0, *b1 = sW + 2 * E0 + E0 * E1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = *ntiles_dev;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int net = chunks[(int64_t)t * 4].w;
        if (net != cur) {   // uniform over the CTA: the 4 chunks of a tile share the net
            __syncthreads();
            const double *P = md.p + md.emb_base + (int64_t)net * md.emb.size;
            for (int q = tid; q < E0; q += 128) {
                sW[q] = P[md.emb.W[0] + q];
                sW[E0 + q] = P[md.emb.b[0] + q];
            }
            for (int q = tid; q < E0 * E1; q += 128) sW[2 * E0 + q] = P[md.emb.W[1] + q];
            for (int q = tid; q < E1; q += 128) sW[2 * E0 + E0 * E1 + q] = P[md.emb.b[1] + q];
            __syncthreads();
            cur = net;
        }
        const int4 c4 = chunks[(int64_t)t * 4 + warp];
        const int a = c4.x, tj = net % md.ntypes;
        const int cnt = a >= 0 ? nnei[(int64_t)a * md.ntypes + tj] : 0;
        const bool valid = c4.z + lane < cnt;
        double R[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid) {
            const int j = nlist[(int64_t)a * md.nsel + md.sel_off[tj] + c4.z + lane];
            double d[3], J[12];
            const double r = min_image_r(pos[a], pos[j], bx, d);
            env_row(d, r, md.rcs, md.rcut, R, J);
        }
        const int64_t row = (int64_t)t * 128 + tid;
#pragma unroll
        for (int c = 0; c < 4; ++c) Rbuf[((int64_t)t * 4 + c) * 128 + tid] = R[c];
        double *ca = a >= 0 ? act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) *
                                        (O::ACT * 32)
                            : nullptr;
        // layer 0: the input is the scalar s = R[0]
        double x1[E0];
#pragma unroll
        for (int o = 0; o < E0; ++o) {
            const double t1 = tanh_f64(b0[o] + R[0] * W0[o]);
            x1[o] = ((E0 == 1 || E0 == 2) ? R[0] : 0.0) + t1;
            if (ca) ca[o * 32 + lane] = t1;
        }
        // layer 1
        double *x2t = x2buf + (int64_t)t * E1 * 128 + tid;   // x2 of this row, channel stride 128
        double mx = 0.0;
        // channels o = h OW + o0: the skip source x1[o0] has a compile-time index
        constexpr int NH = (E1 == 2 * E0) ? 2 : 1, OW = E1 / NH;
#pragma unroll 1
        for (int h = 0; h < NH; ++h) {
#pragma unroll
            for (int o0 = 0; o0 < OW; ++o0) {
                const int o = h * OW + o0;
                double z = b1[o];
#pragma unroll
                for (int k = 0; k < E0; ++k) z += x1[k] * W1[k * E1 + o];
                const double t2 = tanh_f64(z);
                const double x2 = ((E1 == E0 || E1 == 2 * E0) ? x1[o0] : 0.0) + t2;
                if (ca) ca[(E0 + o) * 32 + lane] = t2;
                x2t[o * 128] = x2;
                mx = fmax(mx, fabs(x2));
            }
        }
        // digits of x2 (zero for rows without a neighbor), x2 read back by the thread that wrote it
        const int e = valid ? oz::row_exp(mx) : 0;
        eA[row] = e;
#pragma unroll 1
        for (int k0 = 0; k0 < O::KP; k0 += 8) {
            int d[8][O::S];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                oz::digits<O::S, O::BETA>((valid && k0 + c < E1) ? x2t[(k0 + c) * 128] : 0.0, e, d[c]);
#pragma unroll
            for (int i = 0; i < O::S; ++i) {
                int v[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) v[c] = d[c][i];
                *reinterpret_cast<uint4 *>(dig + oz::tiled(row, k0, i, O::S, 128, O::KC, O::KP)) = oz::pack8(v);
            }
        }
    }
}

template <class O>
struct FwdEpi {
    using Sh = typename O::Sh;
    ModelDev md;
    const int4 *chunks;
    const __half *wdig;   // digits of W2^T per net: [net][NN][KP / 16][S][64 x 16]
    const int *weB;       // their row scales [net][NN * 64]
    const int *eA;
    const double *x2buf, *Rbuf;
    double *act, *Tpart;
    __device__ const __half *b_unit(int64_t tile, int nchunk) const
    {
        const int net = chunks[tile * 4].w;
        return wdig + ((int64_t)net * O::NN + nchunk) * (O::KP / O::KC) * O::S * O::NC * O::KC;
    }
    // 8 warps: the two warps of a row quarter (one chunk) take alternate groups of 8 output channels
    __device__ void operator()(int64_t tile, int nchunk, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0, E1 = O::E1, E2 = O::E2;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, half = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        if (c4.x < 0) return;   // a padding chunk: both warps of the quarter skip
        double *sG = reinterpret_cast<double *>(esm) + warp * 8 * 33;              // [8][33]
        double *sR = reinterpret_cast<double *>(esm) + 8 * 8 * 33 + warp * 4 * 33;   // [4][33]
        const int net = c4.w, tj = net % md.ntypes;
        const int rt = quarter * 32 + lane;   // row in the tile
        const int64_t row = tile * 128 + rt;
#pragma unroll
        for (int c = 0; c < 4; ++c) sR[c * 33 + lane] = Rbuf[(tile * 4 + c) * 128 + rt];
        const int er = eA[row];
        const double *b2 = md.p + md.emb_base + (int64_t)net * md.emb.size + md.emb.b[2];
        const int *eB = weB + (int64_t)net * O::NN * O::NC;
        double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        double *Tp = Tpart + (tile * 4 + quarter) * 4 * E2;
        __syncwarp();
#pragma unroll 1
        for (int c0 = 8 * half; c0 < O::NC; c0 += 16) {
            const int m0 = nchunk * O::NC + c0;
            if (m0 >= E2) break;
            double xs[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int m = m0 + c;
                xs[c] = 0.0;
                if (m < E2) {
                    if (E2 == E1) xs[c] = x2buf[(tile * E1 + m) * 128 + rt];
                    else if (E2 == 2 * E1) xs[c] = x2buf[(tile * E1 + m % E1) * 128 + rt];
                }
            }
            long long H[8], L[8];
            oz::acc_load8<Sh>(trow, c0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int m = m0 + c;
                double g = 0.0;
                if (m < E2) {
                    const double z = oz::acc_value<Sh>(H[c], L[c], er + eB[m]) + b2[m];
                    const double t3 = tanh_f64(z);
                    g = xs[c] + t3;
                    ca[(E0 + E1 + m) * 32 + lane] = t3;
                    ca[(E0 + E1 + E2 + m) * 32 + lane] = g;
                }
                sG[c * 33 + lane] = g;
            }
            __syncwarp();
            // the chunk's part of sum_j G_j[m] R_j[c] for m in m0 .. m0+7: 32 sums, one per lane
            const int mi = lane >> 2, cc = lane & 3;
            if (m0 + mi < E2) {
                double acc = 0.0;
#pragma unroll 8
                for (int nn = 0; nn < 32; ++nn) acc += sG[mi * 33 + nn] * sR[cc * 33 + nn];
                Tp[(m0 + mi) * 4 + cc] = acc;
            }
            __syncwarp();
        }
    }
};

template <class O>
__global__ void __launch_bounds__(128) k_ozf_T(ModelDev md, const int32_t *__restrict__ order, int64_t p0,
                                               const int32_t *__restrict__ nnei, const int *__restrict__ firstc,
                                               const double *__restrict__ Tpart, double *__restrict__ T_out,
                                               double *__restrict__ D_out)
{
    constexpr int NQ = 4 * O::E2;
    __shared__ double sT[NQ];
    const int q = blockIdx.x;
    const int a = order[p0 + q];
    for (int idx = threadIdx.x; idx < NQ; idx += blockDim.x) {
        double acc = 0.0;
        for (int tj = 0; tj < md.ntypes; ++tj) {
            const int nch = (nnei[(int64_t)a * md.ntypes + tj] + 31) >> 5;
            const int64_t f = firstc[(int64_t)q * md.ntypes + tj];
            for (int k = 0; k < nch; ++k) acc += Tpart[(f + k) * NQ + idx];
        }
        const double t = acc * md.inv_nsel;
        sT[idx] = t;
        T_out[(int64_t)q * NQ + idx] = t;
    }
    __syncthreads();
    const int nd = O::E2 * md.m2;
    for (int r = threadIdx.x; r < nd; r += blockDim.x) {
        const int i = r / md.m2, b = r - i * md.m2;
        double v = sT[4 * i] * sT[4 * b] + sT[4 * i + 1] * sT[4 * b + 1];
        v += sT[4 * i + 2] * sT[4 * b + 2] + sT[4 * i + 3] * sT[4 * b + 3];
        D_out[(int64_t)q * nd + r] = v;
    }
}

// dE/dT [m][c] = (sum_b dD[m][b] T[b][c] + [m < M2] sum_a dD[a][m] T[a][c]) / sum(sel), per atom.
template <class O>
__global__ void __launch_bounds__(128) k_ozb_dT(ModelDev md, const double *__restrict__ T,
                                                const double *__restrict__ dD, double *__restrict__ dTbuf)
{
    constexpr int NQ = 4 * O::E2;
    __shared__ double sT[NQ];
    const int64_t q = blockIdx.x;
    const int m2 = md.m2;
    const double *gdD = dD + q * (int64_t)O::E2 * m2;
    for (int idx = threadIdx.x; idx < NQ; idx += blockDim.x) sT[idx] = T[q * NQ + idx];
    __syncthreads();
    for (int idx = threadIdx.x; idx < NQ; idx += blockDim.x) {
        const int m = idx >> 2, c = idx & 3;
        double acc = 0.0;
        for (int b = 0; b < m2; ++b) acc += gdD[m * m2 + b] * sT[b * 4 + c];
        if (m < m2)
            for (int i = 0; i < O::E2; ++i) acc += gdD[i * m2 + m] * sT[i * 4 + c];
        dTbuf[q * NQ + idx] = acc * md.inv_nsel;
    }
}

// One thread per row: dE/dG_j = dT R_j, the direct part dE/dR_j = sum_m G_j[m] dT[m],
// dz3 = dE/dG_j (1 - t3^2) and its digits (the A operand of dx2 = dz3 W2^T),
// and the skip part of dE/dx2.
template <class O>
__global__ void __launch_bounds__(128) k_ozb_front(ModelDev md, const int4 *__restrict__ chunks,
                                                   const int *__restrict__ ntiles_dev, const double *__restrict__ act,
                                                   const double *__restrict__ Rbuf, const double *__restrict__ dTbuf,
                                                   __half *__restrict__ dig, int *__restrict__ eA,
                                                   double *__restrict__ dskip, double *__restrict__ dRbuf,
                                                   double *__restrict__ dzbuf)
{
    constexpr int E0 = O::E0, E1 = O::E1, E2 = O::E2, KP = O::KP2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = *ntiles_dev;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // dz3 staged per tile [KP][128] (L2-resident) until the row maximum is known; the skip part of
        // dE/dx2 accumulated in place [E1][128]
        double *sdz = dzbuf + (int64_t)t * KP * 128;
        double *sdk = dskip + (int64_t)t * E1 * 128;
        const int4 c4 = chunks[(int64_t)t * 4 + warp];
        const int64_t row = (int64_t)t * 128 + tid;
        double R[4], dR[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int c = 0; c < 4; ++c) R[c] = Rbuf[((int64_t)t * 4 + c) * 128 + tid];
        double mx = 0.0;
        if (c4.x >= 0) {
            const int tj = c4.w % md.ntypes;
            const double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
            const double *dT = dTbuf + (int64_t)c4.y * 4 * E2;
#pragma unroll 4
            for (int m = 0; m < E2; ++m) {
                const double4 dt = *reinterpret_cast<const double4 *>(dT + 4 * m);
                const double dg = dt.x * R[0] + dt.y * R[1] + dt.z * R[2] + dt.w * R[3];
                const double y = ca[(E0 + E1 + E2 + m) * 32 + lane];
                dR[0] += dt.x * y;
                dR[1] += dt.y * y;
                dR[2] += dt.z * y;
                dR[3] += dt.w * y;
                const double t3 = ca[(E0 + E1 + m) * 32 + lane];
                const double dz = dg * (1.0 - t3 * t3);
                sdz[m * 128 + tid] = dz;
                mx = fmax(mx, fabs(dz));
                if (E2 == E1) sdk[m * 128 + tid] = dg;
                else if (E2 == 2 * E1) {
                    if (m < E1) sdk[m * 128 + tid] = dg;
                    else sdk[(m - E1) * 128 + tid] += dg;
                }
            }
        } else {
            for (int m = 0; m < E2; ++m) sdz[m * 128 + tid] = 0.0;
            for (int k = 0; k < E1; ++k) sdk[k * 128 + tid] = 0.0;
        }
        if (E2 != E1 && E2 != 2 * E1)
            for (int k = 0; k < E1; ++k) sdk[k * 128 + tid] = 0.0;
        for (int m = E2; m < KP; ++m) sdz[m * 128 + tid] = 0.0;
        const int e = oz::row_exp(mx);
        eA[row] = e;
#pragma unroll 1
        for (int k0 = 0; k0 < KP; k0 += 8) {
            int d[8][O::S];
#pragma unroll
            for (int c = 0; c < 8; ++c) oz::digits<O::S, O::BETA>(sdz[(k0 + c) * 128 + tid], e, d[c]);
#pragma unroll
            for (int i = 0; i < O::S; ++i) {
                int v[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) v[c] = d[c][i];
                *reinterpret_cast<uint4 *>(dig + oz::tiled(row, k0, i, O::S, 128, O::KC, KP)) = oz::pack8(v);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) dRbuf[((int64_t)t * 4 + c) * 128 + tid] = dR[c];
    }
}

__device__ __forceinline__ void bar_pair(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Epilogue of dx2 = dz3 W2^T (8 warps; the two warps of a row quarter take
// alternate groups of 8 of the E1 channels): dE/dx2 = dx2 + skip, dz2, the
// layer-1 input gradient (partial sums of the two warps combined through
// shared memory), then one warp per quarter: layer 0, dE/ds, the chain
// through the environment row's Jacobian to g_ij, the force scatter
// F_i += g_ij, F_j -= g_ij and the virial -d_ij (x) g_ij (both reduced over
// the chunk's 32 rows and added to the center atom).
template <class O>
struct BwdEpi {
    using Sh = typename O::Sh2;
    ModelDev md;
    BoxDev bx;
    const Pos4 *pos;
    const int32_t *nlist, *nnei;
    const int4 *chunks;
    const __half *wdig;   // digits of W2 (rows k, K = E2) per net: [net][KP2 / 16][S][64 x 16]
    const int *weB;       // their row scales [net][64]
    const int *eA;
    const double *act, *dskip, *dRbuf;
    double *force, *atom_virial;
    __device__ const __half *b_unit(int64_t tile, int) const
    {
        const int net = chunks[tile * 4].w;
        return wdig + (int64_t)net * (O::KP2 / O::KC) * O::S * O::NC * O::KC;
    }
    // dE/dx2 for the channel groups k0 = 8 HF + 16 i, dz2, and their part of dE/dx1 (with the skip)
    template <int HF>
    __device__ __forceinline__ void layer1(int64_t tile, uint32_t trow, int rt, int lane, int er, const int *eB,
                                           const double *ca, const double *W1, double (&dx1)[O::E0]) const
    {
        constexpr int E0 = O::E0, E1 = O::E1;
#pragma unroll
        for (int k0 = 8 * HF; k0 < E1; k0 += 16) {
            double ds8[8], t2v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int k = k0 + c;
                ds8[c] = k < E1 ? dskip[(tile * E1 + k) * 128 + rt] : 0.0;
                t2v[c] = k < E1 ? ca[(E0 + k) * 32 + lane] : 0.0;
            }
            long long H[8], L[8];
            oz::acc_load8<Sh>(trow, k0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int k = k0 + c;
                if (k < E1) {
                    const double dy = oz::acc_value<Sh>(H[c], L[c], er + eB[k]) + ds8[c];   // dE/dx2[k]
                    const double dz = dy * (1.0 - t2v[c] * t2v[c]);
#pragma unroll
                    for (int j = 0; j < E0; ++j) dx1[j] += dz * W1[j * E1 + k];
                    if (E1 == E0 || E1 == 2 * E0) dx1[k % E0] += dy;
                }
            }
        }
    }
    __device__ void operator()(int64_t tile, int, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0, E1 = O::E1;
        int *s_net = reinterpret_cast<int *>(esm);                // net + 1 of the weights held (0: none yet)
        double *sW = reinterpret_cast<double *>(esm + 16);        // W0 [E0], W1 [E0][E1]
        double *sx = sW + O::WSM2;                                // [4][E0][32] partial dE/dx1
        const int net = chunks[tile * 4].w;
        if (*s_net != net + 1) {   // uniform over the CTA
            __syncthreads();
            const double *P = md.p + md.emb_base + (int64_t)net * md.emb.size;
            for (int q = tid; q < E0; q += 256) sW[q] = P[md.emb.W[0] + q];
            for (int q = tid; q < E0 * E1; q += 256) sW[E0 + q] = P[md.emb.W[1] + q];
            __syncthreads();
            if (tid == 0) *s_net = net + 1;
        }
        const double *W0 = sW, *W1 = sW + E0;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, half = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        if (c4.x < 0) return;   // a padding chunk: both warps of the quarter skip
        const int a = c4.x, tj = net % md.ntypes;
        const int rt = quarter * 32 + lane;
        const int64_t row = tile * 128 + rt;
        const int er = eA[row];
        const int *eB = weB + (int64_t)net * O::NC;
        const double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        double dx1[E0];
#pragma unroll
        for (int j = 0; j < E0; ++j) dx1[j] = 0.0;
        if (half == 0) layer1<0>(tile, trow, rt, lane, er, eB, ca, W1, dx1);
        else layer1<1>(tile, trow, rt, lane, er, eB, ca, W1, dx1);
        double *sxq = sx + quarter * E0 * 32;
        if (half == 1) {
#pragma unroll
            for (int j = 0; j < E0; ++j) sxq[j * 32 + lane] = dx1[j];
        }
        bar_pair(1 + quarter);
        if (half == 1) return;
#pragma unroll
        for (int j = 0; j < E0; ++j) dx1[j] += sxq[j * 32 + lane];
        const int cnt = nnei[(int64_t)a * md.ntypes + tj];
        const bool valid = c4.z + lane < cnt;
        double fi[3] = {0.0, 0.0, 0.0}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.0;
        if (valid) {
            // layer 0 (input width 1): ds = sum_o dz_o W0[o] (+ the skip when E0 is 1 or 2)
            double ds = 0.0;
#pragma unroll
            for (int j = 0; j < E0; ++j) {
                const double t1 = ca[j * 32 + lane];
                ds += dx1[j] * (1.0 - t1 * t1) * W0[j];
                if (E0 <= 2) ds += dx1[j];
            }
            double dR[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) dR[c] = dRbuf[(tile * 4 + c) * 128 + rt];
            dR[0] += ds;
            const int j = nlist[(int64_t)a * md.nsel + md.sel_off[tj] + c4.z + lane];
            double d[3], Rr[4], J[12];
            const double r = min_image_r(pos[a], pos[j], bx, d);
            env_row(d, r, md.rcs, md.rcut, Rr, J);
            double gv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) gv[k] = dR[0] * J[k] + dR[1] * J[3 + k] + dR[2] * J[6 + k] + dR[3] * J[9 + k];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fi[k] = gv[k];
                atomicAdd(&force[3 * (int64_t)j + k], -gv[k]);
            }
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) vir[3 * x + y] = -d[x] * gv[y];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
            for (int o = 16; o > 0; o >>= 1) fi[k] += __shfl_xor_sync(0xffffffffu, fi[k], o);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            for (int o = 16; o > 0; o >>= 1) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) atomicAdd(&force[3 * (int64_t)a + k], fi[k]);
#pragma unroll
            for (int q = 0; q < 9; ++q) atomicAdd(&atom_virial[9 * (int64_t)a + q], vir[q]);
        }
    }
};

// Scratch of one batch: the work list, the digit and activation buffers of
// both passes (the backward reuses the forward's digit, scale and x2
// buffers), per-chunk contraction parts, dE/dT and the direct dE/dR.
struct Bufs {
    int4 *chunks;
    int *firstc, *ntiles, *eA;
    __half *dig;
    double *x2buf, *Rbuf, *Tpart, *dTbuf, *dRbuf, *dzbuf;
    char *cbs;
    size_t bytes;
};

int64_t max_tiles_of(const ModelDev &md, int64_t nb)
{
    return (nb * md.chunks_per_atom + 3 * md.ntypes * md.ntypes) / 4 + 1;
}

template <class O>
Bufs layout(const ModelDev &md, int64_t nb, char *base)
{
    const int64_t tiles = max_tiles_of(md, nb), rows = tiles * 128;
    const int kmax = O::KP > O::KP2 ? O::KP : O::KP2;
    Bufs b;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    b.chunks = (int4 *)carve(sizeof(int4) * tiles * 4);
    b.firstc = (int *)carve(sizeof(int) * (size_t)nb * md.ntypes);
    b.ntiles = (int *)carve(sizeof(int) * 4);
    b.dig = (__half *)carve(sizeof(__half) * rows * O::S * kmax);
    b.eA = (int *)carve(sizeof(int) * rows);
    b.x2buf = (double *)carve(sizeof(double) * rows * O::E1);
    b.Rbuf = (double *)carve(sizeof(double) * rows * 4);
    b.Tpart = (double *)carve(sizeof(double) * tiles * 4 * 4 * O::E2);
    b.dTbuf = (double *)carve(sizeof(double) * (size_t)nb * 4 * O::E2);
    b.dRbuf = (double *)carve(sizeof(double) * rows * 4);
    b.dzbuf = (double *)carve(sizeof(double) * rows * O::KP2);
    b.cbs = carve(chunks_batch_scratch(md, nb));
    b.bytes = off;
    return b;
}

template <class O>
size_t scratch_bytes(const ModelDev &md, int64_t nb)
{
    return layout<O>(md, nb, nullptr).bytes;
}

template <class O>
dp_status refresh(dp_model *m, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int nnet = md.ntypes * md.ntypes;
    const size_t per = (size_t)O::NN * O::NC * O::S * O::KP, per2 = (size_t)O::NC * O::S * O::KP2;
    const size_t eper = (size_t)O::NN * O::NC + O::NC;
    if (!m->d_ozw_emb) {
        DP_CUDA(cudaMalloc(&m->d_ozw_emb, sizeof(__half) * (per + per2) * nnet));
        DP_CUDA(cudaMalloc((void **)&m->d_oze_emb, sizeof(int) * eper * nnet));
        m->oz_emb_stale = true;
    }
    if (!m->oz_emb_stale) return DP_OK;
    __half *wf = (__half *)m->d_ozw_emb, *wb = wf + per * nnet;
    int *ef = m->d_oze_emb, *eb = ef + (size_t)O::NN * O::NC * nnet;
    for (int net = 0; net < nnet; ++net) {
        // rows of W2^T (output channel m, input k) from the transposed parameter copy, for z3 = x2 W2
        const double *W2T = md.pT + md.emb_base + (int64_t)net * md.emb.size + md.emb.W[2];
        DP_TRY((oz_split<O::S, O::BETA>(W2T, O::E1, O::E2, (int64_t)O::NN * O::NC, O::E1, O::KP, O::NC, O::KC,
                                        wf + per * net, ef + (size_t)O::NN * O::NC * net, st)));
        // rows of W2 (input k, output channel m), for dE/dx2 = dz3 W2^T
        const double *W2 = md.p + md.emb_base + (int64_t)net * md.emb.size + md.emb.W[2];
        DP_TRY((oz_split<O::S, O::BETA>(W2, O::E2, O::E1, (int64_t)O::NC, O::E2, O::KP2, O::NC, O::KC,
                                        wb + per2 * net, eb + (size_t)O::NC * net, st)));
    }
    m->oz_emb_stale = false;
    return DP_OK;
}

template <class O>
dp_status fwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t p0, int64_t nb, double *T, double *D, double *act,
              char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    using Sh = typename O::Sh;
    const int64_t tiles = max_tiles_of(md, nb), rows = tiles * 128;
    const Bufs b = layout<O>(md, nb, scratch);
    DP_TRY(build_chunks_batch(m, nl, p0, nb, b.chunks, b.firstc, b.ntiles, b.cbs, st));
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    const Pos4 *pos = (const Pos4 *)nl->d_pos;
    {
        const int64_t g = tiles < 4 * (int64_t)nsm ? tiles : 4 * (int64_t)nsm;
        k_ozf_front<O><<<(unsigned)g, 128, 0, st>>>(md, bx, pos, nl->d_nlist, nl->d_nnei, b.chunks, b.ntiles, act,
                                                    b.dig, b.eA, b.x2buf, b.Rbuf);
        DP_CUDA(cudaGetLastError());
    }
    {
        FwdEpi<O> epi{md, b.chunks, (const __half *)m->d_ozw_emb, m->d_oze_emb, b.eA, b.x2buf, b.Rbuf, act, b.Tpart};
        auto kern = oz::k_gemm<Sh, FwdEpi<O>, 256>;
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
        const int64_t units = tiles * O::NN;
        const unsigned g = (unsigned)(units < nsm ? units : nsm);
        kern<<<g, 256, Sh::SMEM, st>>>(rows, b.ntiles, O::NN * O::NC, O::KP, b.dig, epi, m->d_err);
        DP_CUDA(cudaGetLastError());
    }
    k_ozf_T<O><<<(unsigned)nb, 128, 0, st>>>(md, nl->d_order, p0, nl->d_nnei, b.firstc, b.Tpart, T, D);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// The backward of the batch whose forward ran last on the same scratch.
template <class O>
dp_status bwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t nb, const double *T, const double *dD,
              const double *act, double *force, double *atom_virial, char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    using Sh = typename O::Sh2;
    const int64_t tiles = max_tiles_of(md, nb), rows = tiles * 128;
    const Bufs b = layout<O>(md, nb, scratch);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    k_ozb_dT<O><<<(unsigned)nb, 128, 0, st>>>(md, T, dD, b.dTbuf);
    DP_CUDA(cudaGetLastError());
    {
        const int64_t g = tiles < 8 * (int64_t)nsm ? tiles : 8 * (int64_t)nsm;
        k_ozb_front<O><<<(unsigned)g, 128, 0, st>>>(md, b.chunks, b.ntiles, act, b.Rbuf, b.dTbuf, b.dig, b.eA,
                                                    b.x2buf, b.dRbuf, b.dzbuf);
        DP_CUDA(cudaGetLastError());
    }
    {
        const __half *wb = (const __half *)m->d_ozw_emb + (size_t)O::NN * O::NC * O::S * O::KP * md.ntypes * md.ntypes;
        const int *eb = m->d_oze_emb + (size_t)O::NN * O::NC * md.ntypes * md.ntypes;
        BwdEpi<O> epi{md, bx, (const Pos4 *)nl->d_pos, nl->d_nlist, nl->d_nnei, b.chunks, wb, eb, b.eA, act,
                      b.x2buf, b.dRbuf, force, atom_virial};
        auto kern = oz::k_gemm<Sh, BwdEpi<O>, 256>;
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
        const unsigned g = (unsigned)(tiles < nsm ? tiles : nsm);
        kern<<<g, 256, Sh::SMEM, st>>>(rows, b.ntiles, O::NC, O::KP2, b.dig, epi, m->d_err);
        DP_CUDA(cudaGetLastError());
    }
    return DP_OK;
}

using OzWater = OzEmb<25, 50, 100>;     // also copper: the (25, 50, 100) nets
using OzStudent = OzEmb<8, 16, 32>;
using OzPaper = OzEmb<32, 64, 128>;

int shape_of(const ModelDev &md)
{
    const int *e = md.emb.wout;
    if (md.n_embed != 3) return 0;
    if (e[0] == 25 && e[1] == 50 && e[2] == 100) return 1;
    if (e[0] == 8 && e[1] == 16 && e[2] == 32) return 2;
    if (e[0] == 32 && e[1] == 64 && e[2] == 128) return 3;
    return 0;
}

}  // namespace

bool oz_emb_ok(const ModelDev &md) { return shape_of(md) != 0 && getenv("DP_NO_OZAKI") == nullptr; }

size_t oz_emb_bytes(const ModelDev &md, int64_t nb)
{
    switch (shape_of(md)) {
    case 1: return scratch_bytes<OzWater>(md, nb);
    case 2: return scratch_bytes<OzStudent>(md, nb);
    case 3: return scratch_bytes<OzPaper>(md, nb);
    default: return 0;
    }
}

dp_status oz_emb_refresh(dp_model *m, cudaStream_t st)
{
    switch (shape_of(m->dev)) {
    case 1: return refresh<OzWater>(m, st);
    case 2: return refresh<OzStudent>(m, st);
    case 3: return refresh<OzPaper>(m, st);
    default: set_error("no split-product embedding for this shape"); return DP_ERR_UNSUPPORTED;
    }
}

dp_status oz_emb_bwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t nb, const double *T, const double *dD,
                     const double *act, double *force, double *atom_virial, char *scratch, cudaStream_t st)
{
    switch (shape_of(m->dev)) {
    case 1: return bwd<OzWater>(m, nl, bx, nb, T, dD, act, force, atom_virial, scratch, st);
    case 2: return bwd<OzStudent>(m, nl, bx, nb, T, dD, act, force, atom_virial, scratch, st);
    case 3: return bwd<OzPaper>(m, nl, bx, nb, T, dD, act, force, atom_virial, scratch, st);
    default: set_error("no split-product embedding for this shape"); return DP_ERR_UNSUPPORTED;
    }
}

dp_status oz_emb_fwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t p0, int64_t nb, double *T, double *D, double *act,
                     char *scratch, cudaStream_t st)
{
    switch (shape_of(m->dev)) {
    case 1: return fwd<OzWater>(m, nl, bx, p0, nb, T, D, act, scratch, st);
    case 2: return fwd<OzStudent>(m, nl, bx, p0, nb, T, D, act, scratch, st);
    case 3: return fwd<OzPaper>(m, nl, bx, p0, nb, T, D, act, scratch, st);
    default: set_error("no split-product embedding for this shape"); return DP_ERR_UNSUPPORTED;
    }
}

}  // namespace dp

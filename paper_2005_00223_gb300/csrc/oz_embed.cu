// Embedding net of the double-precision scheme (Sec. 2, Fig. 1(c,e,f)),
// forward and backward, with the products of its two hidden layers as FP64
// products on the tensor cores by error-free splitting (ozaki.cuh); the
// tanh, skip, contraction and force arithmetic around them stays FP64 on
// the CUDA cores.
//
// Per batch of atoms (type-sorted positions [p0, p0 + nb)), over a work list
// of 32-neighbor chunks grouped into tiles of 128 rows (one neighbor per
// row, one chunk per row quarter) that never mix nets.  Forward:
//   k_ozf_front  one thread per row: environment row R, layer 0 (t1 stored
//                for the backward pass, x1) and the digits of x1;
//   GEMM 1       z2 = x1 W1; epilogue: t2 = tanh(z2 + b1) (stored),
//                x2 = skip(x1) + t2 and the digits of x2;
//   GEMM 2       z3 = x2 W2; epilogue: t3 = tanh(z3 + b2), the embedding
//                output G = skip(x2) + t3 (both stored) and the chunk's part
//                of the contraction sum_j G_j^T R_j (a 32-row sum in row
//                order);
//   k_ozf_T      per atom: T = (1/sum sel) sum over its chunks (type, then
//                chunk order) and D = T T<^T.
// Backward:
//   k_ozb_dT     per atom: dE/dT from dE/dD;
//   k_ozb_front  one thread per row: dE/dG_j = dE/dT R_j, the direct part
//                sum_m G_j[m] dE/dT[m] of dE/dR_j, dz3 = dE/dG_j (1 - t3^2)
//                and its digits, the skip part of dE/dx2;
//   GEMM 3       dE/dx2 = dz3 W2^T + skip; epilogue: dz2 = dE/dx2 (1 - t2^2)
//                and its digits;
//   GEMM 4       dE/dx1 = dz2 W1^T + skip; epilogue: layer 0, dE/ds, the
//                chain through the environment row's Jacobian to g_ij and
//                the scatter F_i += g_ij, F_j -= g_ij with the virial
//                -d_ij (x) g_ij (reduced over the chunk's rows, added to the
//                center atom).
// The GEMM epilogues run on 8 warps, the two warps of a row quarter taking
// alternate groups of 8 channels.  Results agree with the FP64 SIMT kernels
// to the rounding of the split products (about K 2^-52 of |x|_max |W|_max
// per entry).
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
    static constexpr int KP1 = (E0 + 15) / 16 * 16;  // E0 padded: channel groups of dE/dx1
    static constexpr int KA1 = (E0 + 16) / 16 * 16;  // padded K of z2 = [x1, 1] [W1; b1] (the bias as a column)
    static constexpr int KA2 = (E1 + 16) / 16 * 16;  // padded K of z3 = [x2, 1] [W2; b2]
    static constexpr int KP = (E1 + 15) / 16 * 16;   // padded K of z3 = x2 W2 and of dE/dx1 = dz2 W1^T
    static constexpr int KP2 = (E2 + 15) / 16 * 16;  // padded K of dE/dx2 = dz3 W2^T
    static constexpr int NN = (E2 + NC - 1) / NC;    // units of 64 output channels of GEMM 2
    static constexpr int ACT = E0 + E1 + E2 + E2;    // stored per neighbor: t of each layer, then G
    static constexpr int NT2 = 384;                  // GEMM 2 epilogue: 12 warps, three per row quarter
    static constexpr int EPI = 38912;                // its G [12][8][33] and R [12][4][33] doubles
    static constexpr int NT1 = 384;                  // the other epilogues: 12 warps too
    static constexpr int EPIX = 4096;                // their [4][3][32] doubles after a 16-byte header
    using Sh = oz::Shape<S, BETA, NC, KC, EPI, 3>;   // GEMM 2 (3 stages: L1 keeps the tanh table)
    using Sh1 = oz::Shape<S, BETA, NC, KC, EPIX>;    // GEMM 1, 3, 4
    // digits of the weights per net (halves): W1^T (GEMM 1), W2^T (GEMM 2), W2 (GEMM 3), W1 (GEMM 4)
    static constexpr int64_t WF1 = (int64_t)NC * S * KA1, WF2 = (int64_t)NN * NC * S * KA2, WB2 = (int64_t)NC * S * KP2,
                             WB1 = (int64_t)NC * S * KP, WNET = WF1 + WF2 + WB2 + WB1;
    static constexpr int ENET = 3 * NC + NN * NC;    // their row scales per net: f1, f2, b2, b1
    static_assert(NT2 / 32 * (8 + 4) * 33 * 8 <= EPI, "epilogue shared memory");
    static_assert(E1 <= NC && E0 <= NC, "one unit of 64 channels for GEMM 1, 3 and 4");
    static_assert((long long)S * KP2 * (1LL << (2 * BETA - 2)) <= (1LL << 24), "exact FP32 digit sums");
    static_assert((long long)S * KP * (1LL << (2 * BETA - 2)) <= (1LL << 24), "exact FP32 digit sums");
    // every accumulator below 2^22 in magnitude: read back without conversions
    static constexpr int KMAX = KP2 > KA2 ? KP2 : KA2;
    static constexpr bool SMALL = (long long)S * KMAX * (1LL << (2 * BETA - 2)) <= (1LL << 22);
    // the weights augmented with the bias column, FP64, per net: [W1^T | b1] and [W2^T | b2]
    static constexpr int64_t AUG = (int64_t)E1 * (E0 + 1) + (int64_t)E2 * (E1 + 1);
};

// Digits of 8 consecutive columns k0 .. k0+7 of a row for row scale e (one 16-byte store per plane).
template <class O, int KPAD>
__device__ __forceinline__ void put_digits8(__half *dig, int64_t row, int k0, const double (&x)[8], int e)
{
    int d[8][O::S];
#pragma unroll
    for (int c = 0; c < 8; ++c) oz::digits<O::S, O::BETA>(x[c], e, d[c]);
#pragma unroll
    for (int i = 0; i < O::S; ++i) {
        int v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = d[c][i];
        *reinterpret_cast<uint4 *>(dig + oz::tiled(row, k0, i, O::S, 128, O::KC, KPAD)) = oz::pack8(v);
    }
}

// Barrier of the NPART warps of a row quarter (named barrier 1 + quarter).
__device__ __forceinline__ void bar_quarter(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The largest of v over the NPART warps of the row's quarter.
template <int NPART>
__device__ __forceinline__ double quarter_max(double v, unsigned char *esm, int quarter, int part, int lane)
{
    double *sm = reinterpret_cast<double *>(esm + 16);   // [4][NPART][32]
    sm[(quarter * NPART + part) * 32 + lane] = v;
    bar_quarter(1 + quarter, 32 * NPART);
#pragma unroll
    for (int q = 0; q < NPART; ++q) v = oz::amax(v, sm[(quarter * NPART + q) * 32 + lane]);
    return v;
}

template <class O>
__global__ void __launch_bounds__(128) k_ozf_front(ModelDev md, BoxDev bx, const Pos4 *__restrict__ pos,
                                                   const int32_t *__restrict__ nlist, const int32_t *__restrict__ nnei,
                                                   const int4 *__restrict__ chunks, const int *__restrict__ ntiles_dev,
                                                   double *__restrict__ act, __half *__restrict__ dig1,
                                                   int *__restrict__ eA1, double *__restrict__ x1buf,
                                                   double *__restrict__ Rbuf)
{
    constexpr int E0 = O::E0;
    __shared__ double sW[2 * E0];   // W0 [E0], b0 [E0]
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
            __syncthreads();
            cur = net;
        }
        const int4 c4 = chunks[(int64_t)t * 4 + warp];
        int a = c4.x;
        if (a >= 0 && !DP_IDX_OK(a, md.n_list, BS_CHUNK_ATOM)) a = -1;
        const int tj = net % md.ntypes;
        const int cnt = a >= 0 ? nnei[(int64_t)a * md.ntypes + tj] : 0;
        const bool valid = c4.z + lane < cnt;
        double R[4] = {0.0, 0.0, 0.0, 0.0};
        const int j = valid ? nlist[(int64_t)a * md.nsel + md.sel_off[tj] + c4.z + lane] : -1;
        if (valid && DP_IDX_OK(j, md.n_list, BS_NLIST_J)) {
            double d[3], J[12];
            const double r = min_image_r(pos[a], pos[j], bx, d);
            env_row(d, r, md.rcs, md.rcut, md.inv_sw, R, J);
        }
        const int64_t row = (int64_t)t * 128 + tid;
#pragma unroll
        for (int c = 0; c < 4; ++c) Rbuf[((int64_t)t * 4 + c) * 128 + tid] = R[c];
        double *ca = a >= 0 ? act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) *
                                        (O::ACT * 32)
                            : nullptr;
        // layer 0: the input is the scalar s = R[0]
        double x1[O::KA1];
        double mx = 1.0;   // the constant input of the bias column
#pragma unroll
        for (int o = 0; o < O::KA1; ++o) {
            x1[o] = o == E0 ? 1.0 : 0.0;
            if (o < E0) {
                const double t1 = tanh_f64(sW[E0 + o] + R[0] * sW[o]);
                x1[o] = ((E0 == 1 || E0 == 2) ? R[0] : 0.0) + t1;
                if (ca) ca[o * 32 + lane] = t1;
                x1buf[((int64_t)t * E0 + o) * 128 + tid] = x1[o];
                mx = oz::amax(mx, x1[o]);
            }
        }
        const int e = oz::row_exp(mx);
        eA1[row] = e;
#pragma unroll
        for (int k0 = 0; k0 < O::KA1; k0 += 8) {
            double v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = x1[k0 + c];
            put_digits8<O, O::KA1>(dig1, row, k0, v, e);
        }
    }
}

// GEMM 1 epilogue: z2 = [x1, 1] [W1; b1], t2 = tanh(z2) stored, x2 = skip(x1) + t2 stored, the digits
// of [x2, 1].
template <class O>
struct Fwd1Epi {
    using Sh = typename O::Sh1;
    ModelDev md;
    const int4 *chunks;
    const __half *wdig;   // digits of W1^T of net 0; net n at + n WNET
    const int *weB;       // their row scales; net n at + n ENET
    const int *eA1;
    const double *x1buf;
    double *act, *x2buf;
    __half *dig2;
    int *eA2;
    __device__ const __half *b_unit(int64_t tile, int) const { return wdig + chunks[tile * 4].w * O::WNET; }
    // Column groups k0 = 8 part + 8 NPART i: values first (t2, x2 stored; the row maximum kept), then,
    // with the maximum over the quarter's warps, the digits of [x2, 1] read back from x2buf.
    __device__ void operator()(int64_t tile, int, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0, E1 = O::E1;
        constexpr int NPART = O::NT1 / 128;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, part = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        const int rt = quarter * 32 + lane;
        const int64_t row = tile * 128 + rt;
        double *x2t = x2buf + tile * E1 * 128 + rt;   // x2 of this row, channel stride 128
        if (c4.x < 0) {   // a padding chunk: zero digits
            const double z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k0 = 8 * part; k0 < O::KA2; k0 += 8 * NPART) put_digits8<O, O::KA2>(dig2, row, k0, z, 0);
            if (part == 0) eA2[row] = 0;
            return;
        }
        const int net = c4.w, tj = net % md.ntypes;
        const int er = eA1[row];
        const int *eB = weB + (int64_t)net * O::ENET;
        double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        double mx = 1.0;   // the constant input of the next product's bias column
#pragma unroll 1
        for (int k0 = 8 * part; k0 < O::KP; k0 += 8 * NPART) {
            double xs[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int o = k0 + c;
                xs[c] = 0.0;
                if (o < E1 && (E1 == E0 || E1 == 2 * E0)) xs[c] = x1buf[(tile * E0 + o % E0) * 128 + rt];
            }
            long long H[8], L[8];
            oz::acc_load8<Sh, O::SMALL>(trow, k0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int o = k0 + c;
                if (o < E1) {
                    const double t2 = tanh_f64(oz::acc_value<Sh>(H[c], L[c], er + eB[o]));   // the bias is in the product
                    const double x2 = xs[c] + t2;
                    ca[(E0 + o) * 32 + lane] = t2;
                    x2t[o * 128] = x2;
                    mx = oz::amax(mx, x2);
                }
            }
        }
        mx = quarter_max<NPART>(mx, esm, quarter, part, lane);
        const int e = oz::row_exp(mx);
        if (part == 0) eA2[row] = e;
#pragma unroll 1
        for (int k0 = 8 * part; k0 < O::KA2; k0 += 8 * NPART) {
            double v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = k0 + c < E1 ? x2t[(k0 + c) * 128] : (k0 + c == E1 ? 1.0 : 0.0);
            put_digits8<O, O::KA2>(dig2, row, k0, v, e);
        }
    }
};

template <class O>
struct FwdEpi {
    using Sh = typename O::Sh;
    ModelDev md;
    const int4 *chunks;
    const __half *wdig;   // digits of W2^T of net 0 ([NN][KP / 16][S][64 x 16]); net n at + n WNET
    const int *weB;       // their row scales; net n at + n ENET
    const int *eA;
    const double *x2buf, *Rbuf;
    double *act, *Tpart;
    __device__ const __half *b_unit(int64_t tile, int nchunk) const
    {
        const int net = chunks[tile * 4].w;
        return wdig + net * O::WNET + (int64_t)nchunk * (O::KA2 / O::KC) * O::S * O::NC * O::KC;
    }
    // NT2 / 32 warps: the warps of a row quarter (one chunk) take groups of 8 output channels in turn
    __device__ void operator()(int64_t tile, int nchunk, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0, E1 = O::E1, E2 = O::E2, NPART = O::NT2 / 128;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, part = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        if (c4.x < 0) return;   // a padding chunk: the quarter's warps skip
        double *sG = reinterpret_cast<double *>(esm) + warp * 8 * 33;                          // [8][33]
        double *sR = reinterpret_cast<double *>(esm) + (O::NT2 / 32) * 8 * 33 + warp * 4 * 33;   // [4][33]
        const int net = c4.w, tj = net % md.ntypes;
        const int rt = quarter * 32 + lane;   // row in the tile
        const int64_t row = tile * 128 + rt;
#pragma unroll
        for (int c = 0; c < 4; ++c) sR[c * 33 + lane] = Rbuf[(tile * 4 + c) * 128 + rt];
        const int er = eA[row];
        const int *eB = weB + (int64_t)net * O::ENET;
        double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        double *Tp = Tpart + (tile * 4 + quarter) * 4 * E2;
        __syncwarp();
#pragma unroll 1
        for (int c0 = 8 * part; c0 < O::NC; c0 += 8 * NPART) {
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
            oz::acc_load8<Sh, O::SMALL>(trow, c0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int m = m0 + c;
                double g = 0.0;
                if (m < E2) {
                    const double z = oz::acc_value<Sh>(H[c], L[c], er + eB[m]);   // the bias is in the product
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
                mx = oz::amax(mx, dz);
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

// GEMM 3 epilogue: dE/dx2 = dz3 W2^T + skip (stored), dz2 = dE/dx2 (1 - t2^2) and its digits.
template <class O>
struct Bwd3Epi {
    using Sh = typename O::Sh1;
    ModelDev md;
    const int4 *chunks;
    const __half *wdig;   // digits of W2 of net 0; net n at + n WNET
    const int *weB;
    const int *eA;
    const double *act;
    double *dskip, *dybuf;
    __half *dig1;
    int *eA1;
    __device__ const __half *b_unit(int64_t tile, int) const { return wdig + chunks[tile * 4].w * O::WNET; }
    // Values first (dE/dx2 to dybuf, dz2 in place of the skip part in dskip; the row maximum kept),
    // then the digits of dz2 read back.
    __device__ void operator()(int64_t tile, int, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0, E1 = O::E1;
        constexpr int NPART = O::NT1 / 128;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, part = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        const int rt = quarter * 32 + lane;
        const int64_t row = tile * 128 + rt;
        if (c4.x < 0) {
            const double z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int k0 = 8 * part; k0 < O::KP; k0 += 8 * NPART) put_digits8<O, O::KP>(dig1, row, k0, z, 0);
            if (part == 0) eA1[row] = 0;
            return;
        }
        const int net = c4.w, tj = net % md.ntypes;
        const int er = eA[row];
        const int *eB = weB + (int64_t)net * O::ENET + O::NC + O::NN * O::NC;
        const double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        double *dzt = dskip + tile * E1 * 128 + rt;   // the skip part of dE/dx2 in, dz2 out
        double *dyt = dybuf + tile * E1 * 128 + rt;
        double mx = 0.0;
#pragma unroll 1
        for (int k0 = 8 * part; k0 < O::KP; k0 += 8 * NPART) {
            double ds8[8], t2v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int k = k0 + c;
                ds8[c] = k < E1 ? dzt[k * 128] : 0.0;
                t2v[c] = k < E1 ? ca[(E0 + k) * 32 + lane] : 0.0;
            }
            long long H[8], L[8];
            oz::acc_load8<Sh, O::SMALL>(trow, k0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int k = k0 + c;
                if (k < E1) {
                    const double dy = oz::acc_value<Sh>(H[c], L[c], er + eB[k]) + ds8[c];   // dE/dx2[k]
                    const double dz = dy * (1.0 - t2v[c] * t2v[c]);
                    dyt[k * 128] = dy;
                    dzt[k * 128] = dz;
                    mx = oz::amax(mx, dz);
                }
            }
        }
        mx = quarter_max<NPART>(mx, esm, quarter, part, lane);
        const int e = oz::row_exp(mx);
        if (part == 0) eA1[row] = e;
#pragma unroll 1
        for (int k0 = 8 * part; k0 < O::KP; k0 += 8 * NPART) {
            double v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = k0 + c < E1 ? dzt[(k0 + c) * 128] : 0.0;
            put_digits8<O, O::KP>(dig1, row, k0, v, e);
        }
    }
};

// GEMM 4 epilogue: dE/dx1 = dz2 W1^T + skip(dE/dx2), layer 0 (dz1, dE/ds; the two halves' parts
// of dE/ds added through shared memory), then one warp per quarter: dE/dR_j, the Jacobian chain to
// g_ij, the force scatter and the virial, reduced over the chunk's rows for the center atom.
template <class O>
struct Bwd4Epi {
    using Sh = typename O::Sh1;
    ModelDev md;
    BoxDev bx;
    const Pos4 *pos;
    const int32_t *nlist, *nnei;
    const int4 *chunks;
    const __half *wdig;   // digits of W1 of net 0; net n at + n WNET
    const int *weB;
    const int *eA1;
    const double *act, *dybuf, *dRbuf;
    double *force, *atom_virial;
    __device__ const __half *b_unit(int64_t tile, int) const { return wdig + chunks[tile * 4].w * O::WNET; }
    // This warp's part of dE/ds: channel groups j0 = 8 part + 8 NPART i of layer 0.
    __device__ __forceinline__ double layer0(int64_t tile, uint32_t trow, int part, int rt, int lane, int er,
                                             const int *eB, const double *ca, const double *W0) const
    {
        constexpr int E0 = O::E0, E1 = O::E1;
        double ds = 0.0;
#pragma unroll 1
        for (int j0 = 8 * part; j0 < O::KP1; j0 += 8 * (O::NT1 / 128)) {
            double sk[8], t1v[8], w0[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + c;
                sk[c] = t1v[c] = w0[c] = 0.0;
                if (j < E0) {
                    if (E1 == E0) sk[c] = dybuf[(tile * E1 + j) * 128 + rt];
                    else if (E1 == 2 * E0)
                        sk[c] = dybuf[(tile * E1 + j) * 128 + rt] + dybuf[(tile * E1 + j + E0) * 128 + rt];
                    t1v[c] = ca[j * 32 + lane];
                    w0[c] = W0[j];
                }
            }
            long long H[8], L[8];
            oz::acc_load8<Sh, O::SMALL>(trow, j0, H, L);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + c;
                if (j < E0) {
                    const double dx1 = oz::acc_value<Sh>(H[c], L[c], er + eB[j]) + sk[c];   // dE/dx1[j]
                    ds += dx1 * (1.0 - t1v[c] * t1v[c]) * w0[c];
                    if (E0 <= 2) ds += dx1;   // the skip of a first layer of width 1 or 2
                }
            }
        }
        return ds;
    }
    __device__ void operator()(int64_t tile, int, uint32_t trow, int tid, unsigned char *esm) const
    {
        constexpr int E0 = O::E0;
        constexpr int NPART = O::NT1 / 128;
        const int warp = tid >> 5, lane = tid & 31, quarter = warp & 3, part = warp >> 2;
        const int4 c4 = chunks[tile * 4 + quarter];
        if (c4.x < 0) return;   // a padding chunk: the quarter's warps skip
        if (!DP_IDX_OK(c4.x, md.n_list, BS_CHUNK_ATOM)) return;
        const int a = c4.x, net = c4.w, tj = net % md.ntypes;
        const int rt = quarter * 32 + lane;
        const int64_t row = tile * 128 + rt;
        const int er = eA1[row];
        const int *eB = weB + (int64_t)net * O::ENET + 2 * O::NC + O::NN * O::NC;
        const double *ca = act + ((int64_t)c4.y * md.chunks_per_atom + md.chunk_off[tj] + c4.z / 32) * (O::ACT * 32);
        const double *W0 = md.p + md.emb_base + (int64_t)net * md.emb.size + md.emb.W[0];
        double ds = layer0(tile, trow, part, rt, lane, er, eB, ca, W0);
        double *sm = reinterpret_cast<double *>(esm + 16);   // [4][NPART][32]
        if (part > 0) sm[(quarter * NPART + part) * 32 + lane] = ds;
        bar_quarter(1 + quarter, 32 * NPART);
        if (part > 0) return;
#pragma unroll
        for (int q = 1; q < NPART; ++q) ds += sm[(quarter * NPART + q) * 32 + lane];
        const int cnt = nnei[(int64_t)a * md.ntypes + tj];
        const bool valid = c4.z + lane < cnt;
        double fi[3] = {0.0, 0.0, 0.0}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.0;
        const int j = valid ? nlist[(int64_t)a * md.nsel + md.sel_off[tj] + c4.z + lane] : -1;
        if (valid && DP_IDX_OK(j, md.n_list, BS_NLIST_J)) {
            double dR[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) dR[c] = dRbuf[(tile * 4 + c) * 128 + rt];
            dR[0] += ds;
            double d[3], Rr[4], J[12];
            const double r = min_image_r(pos[a], pos[j], bx, d);
            env_row(d, r, md.rcs, md.rcut, md.inv_sw, Rr, J);
            double gv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) gv[k] = dR[0] * J[k] + dR[1] * J[3 + k] + dR[2] * J[6 + k] + dR[3] * J[9 + k];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fi[k] = gv[k];
                acc_add(md.fx, force, 3 * (int64_t)j + k, -gv[k]);
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
            for (int k = 0; k < 3; ++k) acc_add(md.fx, force, 3 * (int64_t)a + k, fi[k]);
#pragma unroll
            for (int q = 0; q < 9; ++q) acc_add(md.fxv, atom_virial, 9 * (int64_t)a + q, vir[q]);
        }
        (void)E0;
    }
};

// Scratch of one batch: the work list, the digit and activation buffers of
// both passes (the backward reuses the forward's buffers where their
// contents are dead), per-chunk contraction parts, dE/dT and the direct
// dE/dR.
struct Bufs {
    int4 *chunks;
    int *firstc, *ntiles, *eA, *eA1;
    __half *dig, *dig1;
    double *x1buf, *x2buf, *Rbuf, *Tpart, *dTbuf, *dRbuf, *dzbuf;
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
    const int kmax = O::KA2 > O::KP2 ? O::KA2 : O::KP2, kmax1 = O::KP > O::KA1 ? O::KP : O::KA1;
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
    b.dig = (__half *)carve(sizeof(__half) * rows * O::S * kmax);     // x2 digits; then dz3
    b.dig1 = (__half *)carve(sizeof(__half) * rows * O::S * kmax1);   // x1 digits; then dz2
    b.eA = (int *)carve(sizeof(int) * rows);
    b.eA1 = (int *)carve(sizeof(int) * rows);
    b.x1buf = (double *)carve(sizeof(double) * rows * O::E0);
    b.x2buf = (double *)carve(sizeof(double) * rows * O::E1);          // x2; then the skip part of dE/dx2
    b.Rbuf = (double *)carve(sizeof(double) * rows * 4);
    b.Tpart = (double *)carve(sizeof(double) * tiles * 4 * 4 * O::E2);
    b.dTbuf = (double *)carve(sizeof(double) * (size_t)nb * 4 * O::E2);
    b.dRbuf = (double *)carve(sizeof(double) * rows * 4);
    b.dzbuf = (double *)carve(sizeof(double) * rows * O::KP2);        // dz3 staging; then dE/dx2
    b.cbs = carve(chunks_batch_scratch(md, nb));
    b.bytes = off;
    return b;
}

template <class O>
size_t scratch_bytes(const ModelDev &md, int64_t nb)
{
    return layout<O>(md, nb, nullptr).bytes;
}

// out [rows][cols + 1] = [WT | bias]: a weight matrix (rows = output channels) with its bias as the
// last column, the B operand of a product whose A rows end in a constant 1.
__global__ void k_aug_bias(const double *__restrict__ WT, const double *__restrict__ bias, int rows, int cols,
                           double *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= rows * (cols + 1)) return;
    const int r = q / (cols + 1), c = q - r * (cols + 1);
    out[q] = c < cols ? WT[(int64_t)r * cols + c] : bias[r];
}

template <class O>
dp_status refresh(dp_model *m, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int nnet = md.ntypes * md.ntypes;
    if (!m->d_ozw_emb) {
        // the digits, then (8-byte aligned) the FP64 augmented weights they are split from
        const size_t dig_bytes = (sizeof(__half) * O::WNET * nnet + 255) & ~(size_t)255;
        DP_CUDA(cudaMalloc(&m->d_ozw_emb, dig_bytes + sizeof(double) * O::AUG));
        DP_CUDA(cudaMalloc((void **)&m->d_oze_emb, sizeof(int) * O::ENET * nnet));
        ++m->epoch;
        m->oz_emb_stale = true;
    }
    if (!m->oz_emb_stale) return DP_OK;
    constexpr int S = O::S, B = O::BETA, NC = O::NC, KC = O::KC;
    double *aug1 = (double *)((char *)m->d_ozw_emb + ((sizeof(__half) * O::WNET * nnet + 255) & ~(size_t)255));
    double *aug2 = aug1 + (int64_t)O::E1 * (O::E0 + 1);
    for (int net = 0; net < nnet; ++net) {
        __half *w = (__half *)m->d_ozw_emb + net * O::WNET;
        int *e = m->d_oze_emb + (size_t)net * O::ENET;
        const int64_t base = md.emb_base + (int64_t)net * md.emb.size;
        // rows of [W1^T | b1] (channel o: input k, then the bias) and of [W2^T | b2] from the transposed
        // parameter copy, for z2 = [x1, 1] [W1; b1] and z3 = [x2, 1] [W2; b2]; rows of W2 (input k,
        // channel m) and of W1, for the input gradients
        k_aug_bias<<<(O::E1 * (O::E0 + 1) + 255) / 256, 256, 0, st>>>(md.pT + base + md.emb.W[1], md.p + base + md.emb.b[1],
                                                                    O::E1, O::E0, aug1);
        k_aug_bias<<<(O::E2 * (O::E1 + 1) + 255) / 256, 256, 0, st>>>(md.pT + base + md.emb.W[2], md.p + base + md.emb.b[2],
                                                                    O::E2, O::E1, aug2);
        DP_CUDA(cudaGetLastError());
        DP_TRY((oz_split<S, B>(aug1, O::E0 + 1, O::E1, NC, O::E0 + 1, O::KA1, NC, KC, w, e, st)));
        DP_TRY((oz_split<S, B>(aug2, O::E1 + 1, O::E2, (int64_t)O::NN * NC, O::E1 + 1, O::KA2, NC, KC, w + O::WF1,
                               e + NC, st)));
        DP_TRY((oz_split<S, B>(md.p + base + md.emb.W[2], O::E2, O::E1, NC, O::E2, O::KP2, NC, KC,
                               w + O::WF1 + O::WF2, e + NC + O::NN * NC, st)));
        DP_TRY((oz_split<S, B>(md.p + base + md.emb.W[1], O::E1, O::E0, NC, O::E1, O::KP, NC, KC,
                               w + O::WF1 + O::WF2 + O::WB2, e + 2 * NC + O::NN * NC, st)));
    }
    m->oz_emb_stale = false;
    return DP_OK;
}

template <class Sh, class Epi, int NT = 256>
dp_status run_gemm(dp_model *m, int64_t tiles, const int *ntiles, int nn, int K, const __half *dA, const Epi &epi,
                   cudaStream_t st)
{
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    auto kern = oz::k_gemm<Sh, Epi, NT>;
    static bool attrs_set = false;   // per instantiation: once per process
    if (!attrs_set) {
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
        // the smallest shared-memory carveout that holds the stages: the rest of the SM's 256 KB stays L1
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)((Sh::SMEM + 2048) * 100 / (228 * 1024)) + 1));
        attrs_set = true;
    }
    const int64_t units = tiles * nn;
    const unsigned g = (unsigned)(units < nsm ? units : nsm);
    kern<<<g, NT, Sh::SMEM, st>>>(tiles * 128, ntiles, nn * Sh::NC, K, dA, epi, m->d_err);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

template <class O>
dp_status fwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t p0, int64_t nb, double *T, double *D, double *act,
              char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int64_t tiles = max_tiles_of(md, nb);
    const Bufs b = layout<O>(md, nb, scratch);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    const Pos4 *pos = (const Pos4 *)nl->d_pos;
    const __half *w = (const __half *)m->d_ozw_emb;
    const int *e = m->d_oze_emb;
    {
        ProfScope ps(m->prof, PG_CHUNKS, 3, st);
        DP_TRY(build_chunks_batch(m, nl, p0, nb, b.chunks, b.firstc, b.ntiles, b.cbs, st));
    }
    {
        ProfScope ps(m->prof, PG_EMBED_FWD, 2, st);
        const int64_t g = tiles < 8 * (int64_t)nsm ? tiles : 8 * (int64_t)nsm;
        k_ozf_front<O><<<(unsigned)g, 128, 0, st>>>(md, bx, pos, nl->d_nlist, nl->d_nnei, b.chunks, b.ntiles, act,
                                                    b.dig1, b.eA1, b.x1buf, b.Rbuf);
        DP_CUDA(cudaGetLastError());
        Fwd1Epi<O> e1{md, b.chunks, w, e, b.eA1, b.x1buf, act, b.x2buf, b.dig, b.eA};
        DP_TRY((run_gemm<typename O::Sh1, Fwd1Epi<O>, O::NT1>(m, tiles, b.ntiles, 1, O::KA1, b.dig1, e1, st)));
    }
    {
        ProfScope ps(m->prof, PG_EMBED_FWD_L2, 1, st);
        FwdEpi<O> e2{md, b.chunks, w + O::WF1, e + O::NC, b.eA, b.x2buf, b.Rbuf, act, b.Tpart};
        DP_TRY((run_gemm<typename O::Sh, FwdEpi<O>, O::NT2>(m, tiles, b.ntiles, O::NN, O::KA2, b.dig, e2, st)));
    }
    ProfScope ps(m->prof, PG_DESC, 1, st);
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
    const int64_t tiles = max_tiles_of(md, nb);
    const Bufs b = layout<O>(md, nb, scratch);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    const __half *w = (const __half *)m->d_ozw_emb;
    const int *e = m->d_oze_emb;
    {
        ProfScope ps(m->prof, PG_DESC, 1, st);
        k_ozb_dT<O><<<(unsigned)nb, 128, 0, st>>>(md, T, dD, b.dTbuf);
        DP_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(m->prof, PG_EMBED_BWD, 1, st);
        const int64_t g = tiles < 8 * (int64_t)nsm ? tiles : 8 * (int64_t)nsm;
        k_ozb_front<O><<<(unsigned)g, 128, 0, st>>>(md, b.chunks, b.ntiles, act, b.Rbuf, b.dTbuf, b.dig, b.eA,
                                                    b.x2buf, b.dRbuf, b.dzbuf);
        DP_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(m->prof, PG_EMBED_BWD_L2, 1, st);
        Bwd3Epi<O> e3{md, b.chunks, w + O::WF1 + O::WF2, e, b.eA, act, b.x2buf, b.dzbuf, b.dig1, b.eA1};
        DP_TRY((run_gemm<typename O::Sh1, Bwd3Epi<O>, O::NT1>(m, tiles, b.ntiles, 1, O::KP2, b.dig, e3, st)));
    }
    ProfScope ps(m->prof, PG_EMBED_BWD, 1, st);
    Bwd4Epi<O> e4{md, bx, (const Pos4 *)nl->d_pos, nl->d_nlist, nl->d_nnei, b.chunks,
                  w + O::WF1 + O::WF2 + O::WB2, e, b.eA1, act, b.dzbuf, b.dRbuf, force, atom_virial};
    DP_TRY((run_gemm<typename O::Sh1, Bwd4Epi<O>, O::NT1>(m, tiles, b.ntiles, 1, O::KP, b.dig1, e4, st)));
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

DP_BOUNDS_ACCESSOR(bounds_read_oz_embed)

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

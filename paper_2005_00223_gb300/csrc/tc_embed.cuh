// Shared pieces of the tensor-core embedding kernels: the tile shapes and
// shared-memory layouts, operand packing, the skip rule, the per-row fetch
// of the neighbor geometry, layer 1 and the layer-2 epilogue of the MIX-16
// kernels, and the FP32 descriptor kernels between the embedding passes.
// Used by tc.cu (MIX-16, bf16 / fp16 operands) and tc_x3.cu (the same
// products as sums of three bf16 products, FP32 accuracy).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "tc_common.cuh"

namespace dp {

namespace {

constexpr long kWaitLimit = 1L << 25;   // mbarrier polls (~1 s) before a kernel gives up
constexpr int kTcThreads = 128;
constexpr int kTmemCols = 256;

template <int E0_, int E1_, int E2_>
struct TcShape {
    static constexpr int E0 = E0_, E1 = E1_, E2 = E2_;
    static constexpr int K2 = (E0 + 15) / 16 * 16;   // layer-2 K (E0 padded)
    static constexpr int N2 = (E1 + 15) / 16 * 16;   // layer-2 N, layer-3 K
    static constexpr int N3 = (E2 + 15) / 16 * 16;   // layer-3 N
    // packed weight image of one net (byte offsets; every part 16-byte aligned)
    static constexpr uint32_t B2_OFF = 0;                              // W2^T [N2][K2]
    static constexpr uint32_t B3_OFF = B2_OFF + N2 * K2 * 2;           // W3^T [N3][N2]
    static constexpr uint32_t B3B_OFF = B3_OFF + N3 * N2 * 2;          // W3   [N2][N3]
    static constexpr uint32_t B2B_OFF = B3B_OFF + N2 * N3 * 2;         // W2   [K2][N2]
    static constexpr uint32_t VEC_OFF = B2B_OFF + K2 * N2 * 2;         // W1[K2], b1[K2], b2[N2], b3[N3] (FP32)
    static constexpr uint32_t IMG = VEC_OFF + (2 * K2 + N2 + N3) * 4;
    static constexpr uint32_t BWD_SCRATCH = 4 * 4 * E2 * 4;             // backward: dE/dT per warp (FP32)
    // Forward kernel layout: only W2^T, W3^T and the vectors of the image, then one region that holds
    // A2 and A3 until the layer-3 MMA has read them and G^T afterwards (R^T after it); tensor memory
    // reused layer by layer (z2, then z3, then the four chunks' T, all from column 0).
    static constexpr uint32_t VEC_BYTES = (2 * K2 + N2 + N3) * 4;
    static constexpr uint32_t F_VEC_OFF = B3B_OFF;
    static constexpr uint32_t F_IMG = (F_VEC_OFF + VEC_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t F_A2_OFF = F_IMG, F_A3_OFF = F_A2_OFF + 128 * K2 * 2;
    static constexpr uint32_t F_GT_OFF = F_IMG, F_RT_OFF = F_GT_OFF + 128 * 128 * 2;
    static constexpr uint32_t F_ACT = 128 * K2 * 2 + 128 * N2 * 2;
    static constexpr uint32_t F_CON = 128 * 128 * 2 + 16 * 128 * 2;
    static constexpr uint32_t F_SMEM = F_IMG + (F_ACT > F_CON ? F_ACT : F_CON);
    static constexpr uint32_t F_MAXC = (N2 > N3 ? N2 : N3) > 64 ? (N2 > N3 ? N2 : N3) : 64;
    static constexpr uint32_t F_TCOLS = F_MAXC <= 32 ? 32 : F_MAXC <= 64 ? 64 : F_MAXC <= 128 ? 128 : 256;
    static constexpr int F_BY_SMEM = (int)((227 * 1024) / (F_SMEM + 1024 + 256));   // + reserved + static
    static constexpr int cmin(int a, int b) { return a < b ? a : b; }
    static constexpr int F_CTAS = cmin(cmin(F_BY_SMEM, (int)(512 / F_TCOLS)), 6);
    static_assert(F_RT_OFF + 16 * 128 * 2 <= F_SMEM && F_A3_OFF + 128 * N2 * 2 <= F_SMEM && F_CTAS >= 2,
                  "forward layout");
    // Backward kernel layout: the full image, then one region that holds A2 and A3 (the forward
    // recomputation) until the layer-3 MMA has read them, dz3 (AB1) from the layer-3 epilogue until
    // the dY2 MMA has read it, and dz2 in A3's place after that; then dE/dT per warp. Tensor memory
    // reused from column 0 by every product; the skip terms of dY2 and dY1 are stored into the
    // accumulator before their MMA, which adds onto them.
    static constexpr uint32_t B_IMG = (IMG + 127) / 128 * 128;
    static constexpr uint32_t B_A2_OFF = B_IMG, B_A3_OFF = B_A2_OFF + 128 * K2 * 2, B_AB1_OFF = B_IMG;
    static constexpr uint32_t B_ACT = F_ACT > 128 * N3 * 2 ? F_ACT : 128 * N3 * 2;
    static constexpr uint32_t B_X_OFF = B_IMG + B_ACT;
    static constexpr uint32_t B_SMEM = B_X_OFF + BWD_SCRATCH;
    static constexpr int B_BY_SMEM = (int)((227 * 1024) / (B_SMEM + 1024 + 256));
    static constexpr int B_CTAS = cmin(cmin(B_BY_SMEM, (int)(512 / F_TCOLS)), E2 <= 32 ? 4 : 3);
    static_assert(B_CTAS >= 2 && B_A3_OFF + 128 * N2 * 2 <= B_X_OFF, "backward layout");
    static_assert(N3 <= 128, "forward tile");
};

using TcWater = TcShape<25, 50, 100>;
using TcStudent = TcShape<8, 16, 32>;
using TcPaper = TcShape<32, 64, 128>;

template <int BF>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// Writes 8 consecutive K values of one row into a K-major core-matrix tile.
template <int BF>
__device__ __forceinline__ void st_row8(unsigned char *tile, int row, int k0, int K, const float *v)
{
    uint4 q;
    q.x = pack2<BF>(v[0], v[1]);
    q.y = pack2<BF>(v[2], v[3]);
    q.z = pack2<BF>(v[4], v[5]);
    q.w = pack2<BF>(v[6], v[7]);
    *reinterpret_cast<uint4 *>(tile + tc::kmaj_off(row, k0, K)) = q;
}

// Skip term of a hidden layer of widths win -> wout at output o (Fig. 1(e,f)).
template <int WIN, int WOUT>
__device__ __forceinline__ float skip_of(const float *x, int o)
{
    if (WOUT == WIN) return x[o];
    if (WOUT == 2 * WIN) return x[o % WIN];
    return 0.0f;
}

struct TileCtx {
    int atom, tj, c0, net;
};

// One thread's row of a tile as read from global memory: the chunk entry,
// the neighbor count of its (atom, type) block and the slot's neighbor
// geometry (s, u = d/r and, for the backward pass, ds/dr, r and j; all
// evaluated in FP64 by the formatting kernel).  Fetched one tile ahead: the
// slot loads do not wait for the count (they stay inside the type block's
// sel slots), and the row's validity is applied when it is used.
struct RowIn {
    TileCtx ch;
    int net, cnt, j;
    float4 a;
    float2 b;
};

template <bool BWD>
__device__ __forceinline__ RowIn fetch_row(const ModelDev &md, const int4 *__restrict__ chunks, int tile, int ntiles,
                                           int warp, int lane, const int32_t *__restrict__ nnei,
                                           const int32_t *__restrict__ nlist, const float4 *__restrict__ envA,
                                           const float2 *__restrict__ envB)
{
    RowIn r;
    r.ch = TileCtx{-1, 0, 0, 0};
    r.net = -1;
    r.cnt = 0;
    r.j = -1;
    r.a = make_float4(0.f, 0.f, 0.f, 0.f);
    r.b = make_float2(0.f, 0.f);
    if (tile >= ntiles) return r;
    const int4 c4 = chunks[(int64_t)tile * 4 + warp];
    r.net = chunks[(int64_t)tile * 4].w;
    r.ch = TileCtx{c4.x, c4.y, c4.z, c4.w};
    if (c4.x >= 0 && !(DP_IDX_OK(c4.x, md.n_list, BS_CHUNK_ATOM) && DP_IDX_OK(c4.y, md.ntypes, BS_TYPE)))
        r.ch.atom = -1;   // bounds-checked build: a bad chunk is treated as padding
    if (r.ch.atom >= 0) {
        const int k = c4.z + lane;
        r.cnt = nnei[(int64_t)c4.x * md.ntypes + c4.y];
        if (k < md.sel[c4.y]) {
            const int64_t slot = (int64_t)c4.x * md.nsel + md.sel_off[c4.y] + k;
            r.a = envA[slot];
            if (BWD) {
                r.b = envB[slot];
                r.j = nlist[slot];
                if (r.j >= 0 && !DP_IDX_OK(r.j, md.n_list, BS_NLIST_J)) r.j = -2;   // bounds-checked build
            }
        }
    }
    return r;
}

// The environment row Rf = (s, s u_x, s u_y, s u_z) of Eq. 4 and the
// geometry of this thread's row (zero on padded rows), plus layer 1 in
// FP32; writes the layer-1 output row into A2.
template <class S, int BF, bool BWD>
__device__ __forceinline__ void rows_layer1(const RowIn &in, int lane, int row, const float *vec, unsigned char *A2,
                                            float Rf[4], float t1[S::E0], float geo[6], int &j, bool &valid)
{
    // (j = -2 only in the bounds-checked build: a neighbor index outside the list, not used)
    valid = in.ch.atom >= 0 && in.ch.c0 + lane < in.cnt && in.j != -2;
    const float4 a = valid ? in.a : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 b = valid ? in.b : make_float2(0.f, 0.f);
    j = valid ? in.j : -1;
    Rf[0] = a.x;
    Rf[1] = a.x * a.y;
    Rf[2] = a.x * a.z;
    Rf[3] = a.x * a.w;
    geo[0] = a.y;                          // u
    geo[1] = a.z;
    geo[2] = a.w;
    geo[3] = b.x;                          // ds/dr
    geo[4] = b.y;                          // r
    geo[5] = (BWD && valid) ? a.x / b.y : 0.f;      // s/r
    const float *W1 = vec, *b1 = vec + S::K2;
    const float s = Rf[0];
    float buf[8];
#pragma unroll
    for (int k0 = 0; k0 < S::K2; k0 += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            float v = 0.0f;
            if (k < S::E0) {
                v = tc::tanh_fast(fmaf(s, W1[k], b1[k]));
                t1[k] = v;
                if (S::E0 == 1 || S::E0 == 2) v += s;
            }
            buf[u] = v;
        }
        st_row8<BF>(A2, row, k0, S::K2, buf);
    }
}

// Layer-2 epilogue: z2 from TMEM, y2 = skip(t1) + tanh(z2 + b2); writes A3.
template <class S, int BF>
__device__ __forceinline__ void epi_layer2(uint32_t taddr, const float *vec, const float t1[S::E0], float t2[S::E1],
                                           unsigned char *A3, int row)
{
    const float *b2 = vec + 2 * S::K2;
#pragma unroll
    for (int c0 = 0; c0 < S::N2; c0 += 16) {
        float z[16];
        tc::tmem_ld16(taddr + c0, z);
        tc::tmem_ld_wait();
        float buf[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int k = c0 + u;
            float v = 0.0f;
            if (k < S::E1) {
                const float t = tc::tanh_fast(z[u] + b2[k]);
                t2[k] = t;
                v = skip_of<S::E0, S::E1>(t1, k) + t;
            }
            buf[u] = v;
        }
        st_row8<BF>(A3, row, c0, S::N2, buf);
        st_row8<BF>(A3, row, c0 + 8, S::N2, buf + 8);
    }
}

__device__ __forceinline__ int4 load_chunk(const int4 *chunks, int64_t idx) { return chunks[idx]; }

// D[p] = T T<^T of atom order[p] (T scaled by 1/sum(sel)), flattened a*M2 + b.
__global__ void k_desc_f32(ModelDev md, const int32_t *__restrict__ order, int64_t n, const float *__restrict__ T,
                           float *__restrict__ D)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nd = md.desc_dim;
    if (q >= n * nd) return;
    const int64_t p = q / nd;
    const int r = (int)(q - p * nd), a = r / md.m2, b = r - a * md.m2;
    const float *Ta = T + (int64_t)order[p] * 4 * md.m1;
    const float s = (float)(md.inv_nsel * md.inv_nsel);
    const float4 x = *reinterpret_cast<const float4 *>(Ta + 4 * a);
    const float4 y = *reinterpret_cast<const float4 *>(Ta + 4 * b);
    D[q] = (x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w) * s;
}

// dE/dT (times 1/sum(sel)) of atom order[p] from dE/dD: one thread per (m, c).
__global__ void k_dT_f32(ModelDev md, const int32_t *__restrict__ order, int64_t n, const float *__restrict__ T,
                         const float *__restrict__ dD, float *__restrict__ dT)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nq = 4 * md.m1;
    if (q >= n * nq) return;
    const int64_t p = q / nq;
    const int r = (int)(q - p * nq), m = r >> 2, c = r & 3;
    const int a_id = order[p];
    const float *Ta = T + (int64_t)a_id * nq;
    const float *dDa = dD + p * md.desc_dim;
    const float inv = (float)md.inv_nsel;
    float acc = 0.f;
    for (int b = 0; b < md.m2; ++b) acc = fmaf(dDa[m * md.m2 + b], Ta[4 * b + c], acc);
    if (m < md.m2)
        for (int a = 0; a < md.m1; ++a) acc = fmaf(dDa[a * md.m2 + m], Ta[4 * a + c], acc);
    dT[(int64_t)a_id * nq + r] = acc * inv * inv;
}

// hi = bf16(x), lo = bf16(x - hi) of two values, packed as bf16 pairs.
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<uint32_t *>(&h);
    lo = *reinterpret_cast<uint32_t *>(&l);
}

// 8 consecutive K values of one row into the hi and lo K-major tiles.
__device__ __forceinline__ void st8_k(unsigned char *hi, unsigned char *lo, int row, int k0, int K, const float *v)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split2(v[2 * q], v[2 * q + 1], h[q], l[q]);
    const uint32_t off = tc::kmaj_off(row, k0, K);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// D (+)= A B^T over K (multiple of 16) with explicit strides between 8-row groups of A and B (K-major).
__device__ __forceinline__ void mma_k_sbo(uint32_t d, uint32_t a, uint32_t a_sbo, uint32_t b, uint32_t b_sbo, int K,
                                          uint32_t id, bool acc0)
{
    for (int ks = 0; ks < (K >> 4); ++ks) {
        const uint64_t ad = tc::smem_desc(a + ks * 256, 128, a_sbo);
        const uint64_t bd = tc::smem_desc(b + ks * 256, 128, b_sbo);
        const uint32_t acc = (acc0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ uint32_t unorm16_pair(float a, float b)
{
    const uint32_t qa = __float2uint_rn(fminf(fmaxf(a, 0.f), 1.f) * 65535.f);
    const uint32_t qb = __float2uint_rn(fminf(fmaxf(b, 0.f), 1.f) * 65535.f);
    return qa | (qb << 16);
}

}  // namespace

}  // namespace dp

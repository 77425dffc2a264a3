// Split-bf16 variant of the tensor-core embedding net (precision DP_MIX_BF16X3):
// the MIX-16 scheme of Sec. 4.1.3 with every product of the embedding net
// carried to FP32-class accuracy on the 5th-generation tensor cores.
//
// Each FP32 operand x is split as x = hi + lo with hi = bf16(x) and
// lo = bf16(x - hi) (16 significant bits in all, the FP32 exponent range), and
// a product A B is taken as hi(A) hi(B) + hi(A) lo(B) + lo(A) hi(B): three
// bf16 MMAs accumulating into one FP32 tensor-memory accumulator.  The term
// lo(A) lo(B) left out and the rounding of lo are both below 2^-16 of the
// product, against 2^-9 for plain bf16 operands: the error of the scheme is
// that of FP32 arithmetic with a 16-bit significand, small enough that the
// force error against FP64 stays below 1e-3 of the RMS force where plain
// bf16 and fp16 operands reach several times that.  tanh is the library's
// tanhf (the MIX-16 kernels use tanh.approx.f32, whose error is below that of
// their 16-bit operands but not below this scheme's).
//
// The layout and flow follow the MIX-16 kernels of tc.cu (same work list of
// 128-row tiles, same geometry records from the formatting kernel, same
// fusion of the contraction T = G^T R into the forward pass and of the force
// and virial scatter into the backward pass); the differences:
//  - every A operand (layer inputs, G^T and R^T of the contraction, dz3, dz2)
//    is written twice, hi and lo, and every weight tile is packed twice;
//  - the backward pass reads W3 and W2 for dE/dy2 = dz3 W3^T and
//    dE/dy1 = dz2 W2^T from the forward tiles W3^T, W2^T as MN-major
//    operands, so the weight image holds two tiles per net, not four;
//  - the descriptor and the fitting net between the passes run in FP32 on
//    the CUDA cores (the MIX-32 kernels), so the whole net is FP32-class.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "dp_internal.cuh"
#include "tc_common.cuh"
#include "tc_embed.cuh"

namespace dp {

namespace {

// Shared-memory layouts of the split-bf16 kernels for an embedding shape S.
template <class S>
struct X3 {
    static constexpr int cmin(int a, int b) { return a < b ? a : b; }
    // packed weights of one net: W2^T [N2][K2], W3^T [N3][N2] (hi), the same (lo), then the FP32 vectors
    static constexpr uint32_t B2 = 0, B3 = B2 + S::N2 * S::K2 * 2, B2L = B3 + S::N3 * S::N2 * 2,
                              B3L = B2L + S::N2 * S::K2 * 2, VEC = B3L + S::N3 * S::N2 * 2,
                              IMG = VEC + S::VEC_BYTES;
    // forward: image, then one region with A2 and A3 (hi, lo) until the layer-3 MMA has read them and
    // G^T and R^T (hi, lo) afterwards
    static constexpr uint32_t F_IMG = (IMG + 1023) / 1024 * 1024;
    static constexpr uint32_t F_A2 = F_IMG, F_A2L = F_A2 + 128 * S::K2 * 2, F_A3 = F_A2L + 128 * S::K2 * 2,
                              F_A3L = F_A3 + 128 * S::N2 * 2;
    static constexpr uint32_t F_GT = F_IMG, F_GTL = F_GT + 128 * 128 * 2, F_RT = F_GTL + 128 * 128 * 2,
                              F_RTL = F_RT + 16 * 128 * 2;
    static constexpr uint32_t F_ACT = 2 * (128 * S::K2 * 2 + 128 * S::N2 * 2);
    static constexpr uint32_t F_CON = 2 * (128 * 128 * 2 + 16 * 128 * 2);
    static constexpr uint32_t F_SMEM = F_IMG + (F_ACT > F_CON ? F_ACT : F_CON);
    static constexpr int F_CTAS = cmin(cmin((int)((227 * 1024) / (F_SMEM + 1024 + 256)), (int)(512 / S::F_TCOLS)), 4);
    // backward: image, then one region with A2, A3 (hi, lo) until the layer-3 MMA has read them, dz3
    // (hi, lo) until the dE/dy2 MMA has read it, dz2 (hi, lo) in A3's place after that; then dE/dT
    // per warp.  Tensor memory: 256 columns, z2 and dE/dy2 from column 0, z3 and dE/dy1 from N2.
    static constexpr uint32_t B_IMG = (IMG + 127) / 128 * 128;
    static constexpr uint32_t B_A2 = B_IMG, B_A2L = B_A2 + 128 * S::K2 * 2, B_A3 = B_A2L + 128 * S::K2 * 2,
                              B_A3L = B_A3 + 128 * S::N2 * 2;
    static constexpr uint32_t B_AB1 = B_IMG, B_AB1L = B_AB1 + 128 * S::N3 * 2;
    static constexpr uint32_t B_ACT = F_ACT > 2 * 128 * S::N3 * 2 ? F_ACT : 2 * 128 * S::N3 * 2;
    static constexpr uint32_t B_X = B_IMG + B_ACT;
    static constexpr uint32_t B_SMEM = B_X + S::BWD_SCRATCH;
    static constexpr uint32_t B_TCOLS = 256;
    static constexpr int B_CTAS = cmin((int)((227 * 1024) / (B_SMEM + 1024 + 256)), 2);
    static_assert(IMG % 16 == 0 && VEC % 16 == 0, "bulk copy alignment");
    static_assert(F_CTAS >= 1 && B_CTAS >= 1, "shared memory");
    static_assert(S::N2 + S::N3 <= (int)B_TCOLS && S::N3 <= (int)S::F_TCOLS, "tensor memory");
    static_assert(B_A3L + 128 * S::N2 * 2 <= B_X && F_RTL + 16 * 128 * 2 <= F_SMEM, "layout");
};

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

// 8 consecutive MN values (mn0 .. mn0 + 7) of K-row k into the hi and lo MN-major tiles.
__device__ __forceinline__ void st8_mn(unsigned char *hi, unsigned char *lo, int mn0, int k, int MN, const float *v)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split2(v[2 * q], v[2 * q + 1], h[q], l[q]);
    const uint32_t off = tc::mnmaj_off(mn0, k, MN);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// D (+)= A B^T as hi(A) hi(B) + hi(A) lo(B) + lo(A) hi(B), both operands K-major.
__device__ __forceinline__ void mma3_k(uint32_t d, const unsigned char *ah, const unsigned char *al,
                                       const unsigned char *bh, const unsigned char *bl, int K, uint32_t id)
{
    tc::mma_kloop(d, tc::smem_u32(ah), tc::smem_u32(bh), K, id, false);
    tc::mma_kloop(d, tc::smem_u32(ah), tc::smem_u32(bl), K, id, true);
    tc::mma_kloop(d, tc::smem_u32(al), tc::smem_u32(bh), K, id, true);
}

// The same with B MN-major of MN extent NB.
__device__ __forceinline__ void mma3_bmn(uint32_t d, const unsigned char *ah, const unsigned char *al,
                                         const unsigned char *bh, const unsigned char *bl, int NB, int K, uint32_t id)
{
    tc::mma_kloop_bmn(d, tc::smem_u32(ah), tc::smem_u32(bh), NB, K, id, false);
    tc::mma_kloop_bmn(d, tc::smem_u32(ah), tc::smem_u32(bl), NB, K, id, true);
    tc::mma_kloop_bmn(d, tc::smem_u32(al), tc::smem_u32(bh), NB, K, id, true);
}

// The environment row Rf = (s, s u) of this thread's row (zero on padded rows), its geometry, and
// layer 1 in FP32 (t1 = tanh(s W1 + b1)); the layer-2 input (with the skip of a 1- or 2-wide
// layer 1) into A2 hi / lo.
template <class S, bool BWD>
__device__ __forceinline__ void rows_layer1_x3(const RowIn &in, int lane, int row, const float *vec, unsigned char *A2,
                                               unsigned char *A2L, float Rf[4], float t1[S::E0], float geo[6], int &j,
                                               bool &valid)
{
    valid = in.ch.atom >= 0 && in.ch.c0 + lane < in.cnt;
    const float4 a = valid ? in.a : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 b = valid ? in.b : make_float2(0.f, 0.f);
    j = valid ? in.j : -1;
    Rf[0] = a.x;
    Rf[1] = a.x * a.y;
    Rf[2] = a.x * a.z;
    Rf[3] = a.x * a.w;
    geo[0] = a.y;
    geo[1] = a.z;
    geo[2] = a.w;
    geo[3] = b.x;
    geo[4] = b.y;
    geo[5] = (BWD && valid) ? a.x / b.y : 0.f;
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
                v = tanhf(fmaf(s, W1[k], b1[k]));
                t1[k] = v;
                if (S::E0 == 1 || S::E0 == 2) v += s;
            }
            buf[u] = v;
        }
        st8_k(A2, A2L, row, k0, S::K2, buf);
    }
}

// Layer-2 epilogue: t2 = tanh(z2 + b2), y2 = skip(t1) + t2 into A3 hi / lo.
template <class S>
__device__ __forceinline__ void epi_layer2_x3(uint32_t taddr, const float *vec, const float t1[S::E0],
                                              float t2[S::E1], unsigned char *A3, unsigned char *A3L, int row)
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
                const float t = tanhf(z[u] + b2[k]);
                t2[k] = t;
                v = skip_of<S::E0, S::E1>(t1, k) + t;
            }
            buf[u] = v;
        }
        st8_k(A3, A3L, row, c0, S::N2, buf);
        st8_k(A3, A3L, row, c0 + 8, S::N2, buf + 8);
    }
}

// One wait by every thread, then a block-wide vote; false (and *err set) when any thread gave up.
__device__ __forceinline__ bool wait_all(uint64_t *bar, uint32_t &ph, int tid, int *err)
{
    const bool ok = tc::mbar_wait(bar, ph, kWaitLimit);
    ph ^= 1;
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(err, 1);
        return false;
    }
    return true;
}

// Loads the packed weights of `net` (one bulk copy) when they change.
template <class S>
__device__ __forceinline__ bool load_net(unsigned char *img, const unsigned char *wimg, int net, int &cur_net,
                                         uint64_t *mbar_w, uint32_t &ph_w, int tid, int *err)
{
    using X = X3<S>;
    if (net == cur_net) return true;
    if (tid == 0) {
        tc::mbar_expect_tx(mbar_w, X::IMG);
        tc::bulk_g2s(img, wimg + (size_t)net * X::IMG, X::IMG, mbar_w);
    }
    if (!wait_all(mbar_w, ph_w, tid, err)) return false;
    cur_net = net;
    return true;
}

// Forward: rows -> layer 1 -> A2 -> z2 = A2 W2^T -> y2 -> A3 -> z3 = A3 W3^T -> G -> T_q = G^T R per
// chunk of 32 rows -> atomics into T [atom][M1][4].
template <class S>
__global__ void __launch_bounds__(kTcThreads) k_embed_fwd_x3(ModelDev md, const float4 *__restrict__ envA,
                                                            const int32_t *__restrict__ nlist,
                                                            const int32_t *__restrict__ nnei,
                                                            const int4 *__restrict__ chunks,
                                                            const int *__restrict__ ntiles_ptr,
                                                            const unsigned char *__restrict__ wimg,
                                                            float *__restrict__ T, int *err)
{
    using X = X3<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *img = smem;
    const float *vec = reinterpret_cast<const float *>(img + X::VEC);
    if (tid == 0) {
        tc::mbar_init(&mbar_mma, 1);
        tc::mbar_init(&mbar_w, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, S::F_TCOLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t id2 = tc::idesc_f16(128, S::N2, 1), id3 = tc::idesc_f16(128, S::N3, 1);
    const uint32_t idT = tc::idesc_f16_major(128, 16, 1, 1, 1);
    uint32_t ph_mma = 0, ph_w = 0;
    int cur_net = -1;
    const int ntiles = *ntiles_ptr;
    RowIn nxt = fetch_row<false>(md, chunks, blockIdx.x, ntiles, warp, lane, nnei, nlist, envA, nullptr);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const RowIn in = nxt;
        nxt = fetch_row<false>(md, chunks, tile + gridDim.x, ntiles, warp, lane, nnei, nlist, envA, nullptr);
        if (!load_net<S>(img, wimg, in.net, cur_net, &mbar_w, ph_w, tid, err)) break;
        float Rf[4], t1[S::E0], t2[S::E1], geo[6];
        int j;
        bool valid;
        rows_layer1_x3<S, false>(in, lane, tid, vec, smem + X::F_A2, smem + X::F_A2L, Rf, t1, geo, j, valid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            mma3_k(tmem, smem + X::F_A2, smem + X::F_A2L, img + X::B2, img + X::B2L, S::K2, id2);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        epi_layer2_x3<S>(taddr, vec, t1, t2, smem + X::F_A3, smem + X::F_A3L, tid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            mma3_k(tmem, smem + X::F_A3, smem + X::F_A3L, img + X::B3, img + X::B3L, S::N2, id3);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        // layer-3 epilogue: G = skip(y2) + tanh(z3 + b3) into G^T, this thread's row R into R^T (hi and
        // lo; channels m >= E2 and columns c >= 4 zero, all rewritten each tile)
        {
            unsigned char *GT = smem + X::F_GT, *GTL = smem + X::F_GTL;
            unsigned char *RT = smem + X::F_RT, *RTL = smem + X::F_RTL;
            const float *b3 = vec + 2 * S::K2 + S::N2;
            float y2[S::E1];
#pragma unroll
            for (int k = 0; k < S::E1; ++k) y2[k] = skip_of<S::E0, S::E1>(t1, k) + t2[k];
            {
                float r8[8] = {Rf[0], Rf[1], Rf[2], Rf[3], 0.f, 0.f, 0.f, 0.f};
                st8_mn(RT, RTL, 0, tid, 16, r8);
                const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(RT + tc::mnmaj_off(8, tid, 16)) = z4;
                *reinterpret_cast<uint4 *>(RTL + tc::mnmaj_off(8, tid, 16)) = z4;
#pragma unroll
                for (int c0 = S::N3; c0 < 128; c0 += 8) {
                    *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0, tid, 128)) = z4;
                    *reinterpret_cast<uint4 *>(GTL + tc::mnmaj_off(c0, tid, 128)) = z4;
                }
            }
#pragma unroll
            for (int c0 = 0; c0 < S::N3; c0 += 16) {
                float z[16];
                tc::tmem_ld16(taddr + c0, z);
                tc::tmem_ld_wait();
                float g[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int m = c0 + u;
                    g[u] = m < S::E2 ? skip_of<S::E1, S::E2>(y2, m) + tanhf(z[u] + b3[m]) : 0.f;
                }
                st8_mn(GT, GTL, c0, tid, 128, g);
                st8_mn(GT, GTL, c0 + 8, tid, 128, g + 8);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t gh = tc::smem_u32(smem + X::F_GT), gl = tc::smem_u32(smem + X::F_GTL);
            const uint32_t rh = tc::smem_u32(smem + X::F_RT), rl = tc::smem_u32(smem + X::F_RTL);
            // chunk q: T_q[m][c] = sum over its 32 rows of G[row][m] R[row][c]
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                tc::mma_kloop_mn(tmem + 16 * q, gh, 128, rh, 16, 32 * q, 32, idT, false);
                tc::mma_kloop_mn(tmem + 16 * q, gh, 128, rl, 16, 32 * q, 32, idT, true);
                tc::mma_kloop_mn(tmem + 16 * q, gl, 128, rh, 16, 32 * q, 32, idT, true);
            }
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        {
            const int m = warp * 32 + lane;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[4];
                tc::tmem_ld4(taddr + 16 * q, v);
                tc::tmem_ld_wait();
                const int atom = load_chunk(chunks, (int64_t)tile * 4 + q).x;
                if (atom >= 0 && m < S::E2) {
                    float *Tm = T + (int64_t)atom * 4 * S::E2 + 4 * m;
#pragma unroll
                    for (int c = 0; c < 4; ++c) atomicAdd(Tm + c, v[c]);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, S::F_TCOLS);
}

// Backward: the forward again (no stored activations), then dG = dT R, dR = dT^T G,
// dz3 = dG (1 - t3^2) -> dE/dy2 = dz3 W3^T + skip -> dz2 -> dE/dy1 = dz2 W2^T + skip -> ds ->
// g_ij -> FP64 force and virial atomics.
template <class S>
__global__ void __launch_bounds__(kTcThreads) k_embed_bwd_x3(ModelDev md, const float4 *__restrict__ envA,
                                                            const float2 *__restrict__ envB,
                                                            const int32_t *__restrict__ nlist,
                                                            const int32_t *__restrict__ nnei,
                                                            const int4 *__restrict__ chunks,
                                                            const int *__restrict__ ntiles_ptr,
                                                            const unsigned char *__restrict__ wimg,
                                                            const float *__restrict__ dT, double *__restrict__ force,
                                                            double *__restrict__ atom_virial, int *err)
{
    using X = X3<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *img = smem;
    float *sdT = reinterpret_cast<float *>(smem + X::B_X) + warp * 4 * S::E2;
    const float *vec = reinterpret_cast<const float *>(img + X::VEC);
    if (tid == 0) {
        tc::mbar_init(&mbar_mma, 1);
        tc::mbar_init(&mbar_w, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, X::B_TCOLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t kHi = (uint32_t)S::N2;   // column of the layer-3 and dE/dy1 products
    const uint32_t id2 = tc::idesc_f16(128, S::N2, 1), id3 = tc::idesc_f16(128, S::N3, 1);
    const uint32_t idb1 = tc::idesc_f16_major(128, S::N2, 1, 0, 1), idb2 = tc::idesc_f16_major(128, S::K2, 1, 0, 1);
    uint32_t ph_mma = 0, ph_w = 0;
    int cur_net = -1;
    const int ntiles = *ntiles_ptr;
    RowIn nxt = fetch_row<true>(md, chunks, blockIdx.x, ntiles, warp, lane, nnei, nlist, envA, envB);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const RowIn in = nxt;
        nxt = fetch_row<true>(md, chunks, tile + gridDim.x, ntiles, warp, lane, nnei, nlist, envA, envB);
        const TileCtx ch = in.ch;
        if (!load_net<S>(img, wimg, in.net, cur_net, &mbar_w, ph_w, tid, err)) break;
        // dE/dT of this warp's atom (already scaled by 1/sum(sel))
        for (int q = lane; q < 4 * S::E2; q += 32) sdT[q] = ch.atom >= 0 ? dT[(int64_t)ch.atom * 4 * S::E2 + q] : 0.f;
        float Rf[4], t1[S::E0], t2[S::E1], geo[6];
        int j;
        bool valid;
        rows_layer1_x3<S, true>(in, lane, tid, vec, smem + X::B_A2, smem + X::B_A2L, Rf, t1, geo, j, valid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            mma3_k(tmem, smem + X::B_A2, smem + X::B_A2L, img + X::B2, img + X::B2L, S::K2, id2);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        epi_layer2_x3<S>(taddr, vec, t1, t2, smem + X::B_A3, smem + X::B_A3L, tid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            mma3_k(tmem + kHi, smem + X::B_A3, smem + X::B_A3L, img + X::B3, img + X::B3L, S::N2, id3);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        // layer-3 epilogue fused with the start of the backward pass:
        //   G = skip(y2) + t3,  dG = dT R,  dR += dT^T G,  dz3 = dG (1 - t3^2)
        float dR[4] = {0.f, 0.f, 0.f, 0.f};
        float res2[S::E1];   // skip terms of dE/dy2
#pragma unroll
        for (int k = 0; k < S::E1; ++k) res2[k] = 0.f;
        {
            const float *b3 = vec + 2 * S::K2 + S::N2;
            float y2[S::E1];
#pragma unroll
            for (int k = 0; k < S::E1; ++k) y2[k] = skip_of<S::E0, S::E1>(t1, k) + t2[k];
#pragma unroll
            for (int c0 = 0; c0 < S::N3; c0 += 16) {
                float z[16];
                tc::tmem_ld16(taddr + kHi + c0, z);
                tc::tmem_ld_wait();
                float buf[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int m = c0 + u;
                    float v = 0.f;
                    if (m < S::E2) {
                        const float t = tanhf(z[u] + b3[m]);
                        const float G = skip_of<S::E1, S::E2>(y2, m) + t;
                        const float4 dt = *reinterpret_cast<const float4 *>(sdT + 4 * m);
                        dR[0] = fmaf(dt.x, G, dR[0]);
                        dR[1] = fmaf(dt.y, G, dR[1]);
                        dR[2] = fmaf(dt.z, G, dR[2]);
                        dR[3] = fmaf(dt.w, G, dR[3]);
                        const float dG = dt.x * Rf[0] + dt.y * Rf[1] + dt.z * Rf[2] + dt.w * Rf[3];
                        v = dG * (1.f - t * t);
                        if (S::E2 == S::E1) res2[m] += dG;
                        else if (S::E2 == 2 * S::E1) res2[m % S::E1] += dG;
                    }
                    buf[u] = v;
                }
                st8_k(smem + X::B_AB1, smem + X::B_AB1L, tid, c0, S::N3, buf);
                st8_k(smem + X::B_AB1, smem + X::B_AB1L, tid, c0 + 8, S::N3, buf + 8);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // dE/dy2 = dz3 W3^T: B = W3 [N2][N3], read from the W3^T tile as an MN-major operand
            mma3_bmn(tmem, smem + X::B_AB1, smem + X::B_AB1L, img + X::B3, img + X::B3L, S::N2, S::N3, idb1);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        float res1[S::E0];   // skip terms of dE/dy1
#pragma unroll
        for (int k = 0; k < S::E0; ++k) res1[k] = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < S::N2; c0 += 16) {
            float z[16];
            tc::tmem_ld16(taddr + c0, z);
            tc::tmem_ld_wait();
            float buf[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = c0 + u;
                float v = 0.f;
                if (k < S::E1) {
                    const float dy2 = z[u] + res2[k];
                    v = dy2 * (1.f - t2[k] * t2[k]);
                    if (S::E1 == S::E0) res1[k] += dy2;
                    else if (S::E1 == 2 * S::E0) res1[k % S::E0] += dy2;
                }
                buf[u] = v;
            }
            st8_k(smem + X::B_A3, smem + X::B_A3L, tid, c0, S::N2, buf);
            st8_k(smem + X::B_A3, smem + X::B_A3L, tid, c0 + 8, S::N2, buf + 8);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // dE/dy1 = dz2 W2^T: B = W2 [K2][N2], read from the W2^T tile as an MN-major operand
            mma3_bmn(tmem + kHi, smem + X::B_A3, smem + X::B_A3L, img + X::B2, img + X::B2L, S::K2, S::N2, idb2);
            tc::mma_commit(&mbar_mma);
        }
        if (!wait_all(&mbar_mma, ph_mma, tid, err)) break;
        tc::fence_after_sync();
        float ds = 0.f;
        {
            const float *W1 = vec;
#pragma unroll
            for (int c0 = 0; c0 < S::K2; c0 += 16) {
                float z[16];
                tc::tmem_ld16(taddr + kHi + c0, z);
                tc::tmem_ld_wait();
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int k = c0 + u;
                    if (k < S::E0) {
                        const float dy1 = z[u] + res1[k];
                        ds = fmaf(dy1 * (1.f - t1[k] * t1[k]), W1[k], ds);
                        if (S::E0 == 1 || S::E0 == 2) ds += dy1;
                    }
                }
            }
        }
        // g = (dR/dr_ij)^T dE/dR in FP32.  With R = (s, s u), u = d/r:
        //   g = u (dR0 s' + (s' - s/r) u.dR') + (s/r) dR',  dR' = (dR1, dR2, dR3);
        // F_j -= g, F_i += g, W_i -= d (x) g, accumulated in FP64.
        float gv[3] = {0.f, 0.f, 0.f}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.f;
        if (valid) {
            const float dR0 = dR[0] + ds;
            const float ud = geo[0] * dR[1] + geo[1] * dR[2] + geo[2] * dR[3];
            const float cu = fmaf(geo[3] - geo[5], ud, dR0 * geo[3]);
#pragma unroll
            for (int k = 0; k < 3; ++k) gv[k] = fmaf(cu, geo[k], geo[5] * dR[1 + k]);
#pragma unroll
            for (int k = 0; k < 3; ++k) atomicAdd(&force[3 * (int64_t)j + k], -(double)gv[k]);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) vir[3 * a + b] = -(geo[4] * geo[a]) * gv[b];
        }
        // the warp's rows all belong to one atom: reduce F_i and W_i over the warp
#pragma unroll
        for (int k = 0; k < 3; ++k)
            for (int s = 16; s > 0; s >>= 1) gv[k] += __shfl_xor_sync(0xffffffffu, gv[k], s);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            for (int s = 16; s > 0; s >>= 1) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], s);
        if (ch.atom >= 0) {
            if (lane < 3) {
                float v = lane == 0 ? gv[0] : (lane == 1 ? gv[1] : gv[2]);
                atomicAdd(&force[3 * (int64_t)ch.atom + lane], (double)v);
            }
            if (lane < 9) {
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < 9; ++q) v = (q == lane) ? vir[q] : v;
                atomicAdd(&atom_virial[9 * (int64_t)ch.atom + lane], (double)v);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, X::B_TCOLS);
}

// Packed weights of one net: hi = bf16(w), lo = bf16(w - hi) with w the FP64 weight (so lo also
// carries what an FP32 rounding of w would lose below 2^-16).
template <class S>
void pack_net_x3(const double *p, const NetLayout &L, unsigned char *out)
{
    using X = X3<S>;
    memset(out, 0, X::IMG);
    auto put = [&](uint32_t hi, uint32_t lo, int r, int k, int K, double w) {
        const __nv_bfloat16 h = __double2bfloat16(w);
        const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
        memcpy(out + hi + tc::kmaj_off(r, k, K), &h, 2);
        memcpy(out + lo + tc::kmaj_off(r, k, K), &l, 2);
    };
    const double *W1 = p + L.W[0], *b1 = p + L.b[0];
    const double *W2 = p + L.W[1], *b2 = p + L.b[1];
    const double *W3 = p + L.W[2], *b3 = p + L.b[2];
    for (int a = 0; a < S::E0; ++a)
        for (int o = 0; o < S::E1; ++o) put(X::B2, X::B2L, o, a, S::K2, W2[a * S::E1 + o]);   // W2^T
    for (int a = 0; a < S::E1; ++a)
        for (int o = 0; o < S::E2; ++o) put(X::B3, X::B3L, o, a, S::N2, W3[a * S::E2 + o]);   // W3^T
    float *vec = reinterpret_cast<float *>(out + X::VEC);
    for (int k = 0; k < S::E0; ++k) {
        vec[k] = (float)W1[k];
        vec[S::K2 + k] = (float)b1[k];
    }
    for (int k = 0; k < S::E1; ++k) vec[2 * S::K2 + k] = (float)b2[k];
    for (int k = 0; k < S::E2; ++k) vec[2 * S::K2 + S::N2 + k] = (float)b3[k];
}

template <class S>
dp_status pack_x3(dp_model *m)
{
    using X = X3<S>;
    const ModelDev &md = m->dev;
    const int nn = m->ntypes * m->ntypes;
    std::vector<unsigned char> img((size_t)nn * X::IMG);
    for (int q = 0; q < nn; ++q)
        pack_net_x3<S>(m->h_params.data() + md.emb_base + q * md.emb.size, md.emb, img.data() + (size_t)q * X::IMG);
    if (!m->d_tcw_x3) DP_CUDA(cudaMalloc((void **)&m->d_tcw_x3, img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_tcw_x3, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return DP_OK;
}

template <class S>
dp_status run_x3(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                 double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    using X = X3<S>;
    const ModelDev &md = m->dev;
    const int64_t n = nl->n;
    const int nn = md.ntypes * md.ntypes;
    const int64_t max_chunks = n * md.chunks_per_atom + 4 * nn + 4;
    size_t need = 0;
    auto sz = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    sz(sizeof(float) * 4 * md.m1 * n);   // T
    sz(sizeof(float) * 4 * md.m1 * n);   // dE/dT
    sz(sizeof(float) * md.desc_dim * n);   // D
    sz(sizeof(float) * md.desc_dim * n);   // dE/dD
    sz(sizeof(int4) * max_chunks);
    sz(sizeof(int) * 4);
    sz(chunks_batch_scratch(md, n));
    DP_TRY(ensure_workspace(m, need));
    char *w = m->ws;
    auto carve = [&](size_t bytes) {
        char *p = w;
        w += (bytes + 255) & ~(size_t)255;
        return p;
    };
    float *T = (float *)carve(sizeof(float) * 4 * md.m1 * n);
    float *dT = (float *)carve(sizeof(float) * 4 * md.m1 * n);
    float *D = (float *)carve(sizeof(float) * md.desc_dim * n);
    float *dD = (float *)carve(sizeof(float) * md.desc_dim * n);
    int4 *chunks = (int4 *)carve(sizeof(int4) * max_chunks);
    int *cnt = (int *)carve(sizeof(int) * 4);
    char *scratch = carve(chunks_batch_scratch(md, n));
    if (!nl->d_env) {
        set_error("split-bf16 path needs the neighbor geometry of the formatting kernel");
        return DP_ERR_ARG;
    }
    if (!m->d_tcw_x3) DP_TRY(pack_x3<S>(m));
    const float4 *envA = reinterpret_cast<const float4 *>(nl->d_env);
    const float2 *envB = reinterpret_cast<const float2 *>(nl->d_env + 4 * (size_t)n * md.nsel);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    DP_CUDA(cudaMemsetAsync(T, 0, sizeof(float) * 4 * md.m1 * n, st));
    DP_CUDA(cudaMemsetAsync(d_force, 0, sizeof(double) * 3 * n, st));
    DP_CUDA(cudaMemsetAsync(d_atom_virial, 0, sizeof(double) * 9 * n, st));
    {
        ProfScope ps(m->prof, PG_CHUNKS, 3, st);
        DP_TRY(build_chunks_batch(m, nl, 0, n, chunks, nullptr, cnt, scratch, st));
    }
    DP_CUDA(cudaFuncSetAttribute(k_embed_fwd_x3<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::F_SMEM));
    DP_CUDA(cudaFuncSetAttribute(k_embed_fwd_x3<S>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    DP_CUDA(cudaFuncSetAttribute(k_embed_bwd_x3<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::B_SMEM));
    DP_CUDA(cudaFuncSetAttribute(k_embed_bwd_x3<S>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    {
        ProfScope ps(m->prof, PG_EMBED_FWD, 1, st);
        k_embed_fwd_x3<S><<<(unsigned)(X::F_CTAS * nsm), kTcThreads, X::F_SMEM, st>>>(
            md, envA, nl->d_nlist, nl->d_nnei, chunks, cnt, m->d_tcw_x3, T, m->d_err);
    }
    DP_CUDA(cudaGetLastError());
    const int64_t nd = (int64_t)md.desc_dim * n, nq = (int64_t)4 * md.m1 * n;
    {
        ProfScope ps(m->prof, PG_DESC, 1, st);
        k_desc_f32<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(md, nl->d_order, n, T, D);
    }
    DP_CUDA(cudaGetLastError());
    DP_TRY(fit_f32(m, nl, D, dD, d_atom_energy, st));
    {
        ProfScope ps(m->prof, PG_DESC, 1, st);
        k_dT_f32<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(md, nl->d_order, n, T, dD, dT);
    }
    DP_CUDA(cudaGetLastError());
    {
        ProfScope ps(m->prof, PG_EMBED_BWD, 1, st);
        k_embed_bwd_x3<S><<<(unsigned)(X::B_CTAS * nsm), kTcThreads, X::B_SMEM, st>>>(
            md, envA, envB, nl->d_nlist, nl->d_nnei, chunks, cnt, m->d_tcw_x3, dT, d_force, d_atom_virial, m->d_err);
    }
    DP_CUDA(cudaGetLastError());
    ProfScope ps(m->prof, PG_REDUCE, 1, st);
    return reduce_energy_virial(d_atom_energy, d_atom_virial, centers_of(nl), d_energy, d_virial, m->d_red, st);
}

}  // namespace

dp_status pack_x3_weights(dp_model *m)
{
    const int *e = m->dev.emb.wout;
    if (e[0] == 25) return pack_x3<TcWater>(m);
    if (e[0] == 8) return pack_x3<TcStudent>(m);
    return pack_x3<TcPaper>(m);
}

dp_status compute_mix_x3(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                         double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    const int *e = m->dev.emb.wout;
    if (e[0] == 25) return run_x3<TcWater>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
    if (e[0] == 8) return run_x3<TcStudent>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
    return run_x3<TcPaper>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
}

}  // namespace dp

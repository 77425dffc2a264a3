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
#include <stdlib.h>
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
    // (j = -2 only in the bounds-checked build: a neighbor index outside the list, not used)
    valid = in.ch.atom >= 0 && in.ch.c0 + lane < in.cnt && in.j != -2;
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
                if (atom >= 0 && m < S::E2 && DP_IDX_OK(atom, md.n_list, BS_CHUNK_ATOM)) {
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

// ---------------------------------------------------------------------------------------------
// Fitting net in split bf16 on the tensor cores, fused with the descriptor and its adjoint (the
// structure of the MIX-16 fitting kernel in tc.cu: one CTA per SM walks tiles of 128 atoms of one
// center type, thread = atom row, accumulators in tensor memory).  The hi and lo weight tiles do not
// fit in shared memory whole, so every product streams its B operand in chunks (hi and lo of a chunk
// in one bulk copy) through a two-stage ring, the copy of chunk c + 1 overlapping the MMAs of chunk c;
// the A operand (D in K chunks for layer 1, else the 128 x F activations) is written hi and lo.
// tanh is tanhf; the derivative factors (1 - t1^2, 1 - t2^2) wait in tensor memory as 16-bit fixed
// point pairs (absolute error 2^-17 of a value in [0, 1]).

template <int M1_, int M2_, int F_>
struct FitX3 {
    static constexpr int M1 = M1_, M2 = M2_, F = F_, D = M1_ * M2_;
    static constexpr int KC1 = 32, NK1 = D / KC1;                   // layer-1 K chunks
    static constexpr int KC2 = (F % 48 == 0) ? 48 : 32, NK2 = F / KC2;   // K chunks of the F x F products
    static constexpr int NC = 32, NB1 = D / NC;                     // N chunks of dE/dD = dz1 W1^T
    static constexpr uint32_t C1 = F * KC1 * 4, C2 = F * KC2 * 4, CB1 = NC * F * 4;   // chunk bytes, hi + lo
    // global image per center type: chunks of W1^T [F][KC1], W2^T, W3^T [F][KC2] (K = input),
    // W3, W2 [F][KC2] (K = output), W1 [NC][F]; then b1, b2, b3, w_out [F], b_out (FP32)
    static constexpr uint32_t W1T = 0, W2T = W1T + NK1 * C1, W3T = W2T + NK2 * C2, W3B = W3T + NK2 * C2,
                              W2B = W3B + NK2 * C2, W1B = W2B + NK2 * C2, VEC = W1B + NB1 * CB1,
                              VEC_BYTES = (4 * F + 4) * 4, IMG = VEC + VEC_BYTES;
    static constexpr uint32_t cmax(uint32_t a, uint32_t b) { return a > b ? a : b; }
    static constexpr uint32_t STAGE = cmax(cmax(C1, C2), CB1);
    static constexpr uint32_t ACT = 2 * 128 * F * 2;                // activations hi | lo
    static constexpr uint32_t DCH = 2 * 128 * KC1 * 2;              // one D chunk hi | lo
    static constexpr uint32_t A_BYTES = cmax(ACT, 2 * DCH);
    static constexpr uint32_t A_OFF = 0, B_OFF = A_BYTES, V_OFF = B_OFF + 2 * STAGE, SMEM = V_OFF + VEC_BYTES;
    static_assert(D % KC1 == 0 && F % KC2 == 0 && D % NC == 0 && NC % M2_ == 0 && KC1 % M2_ == 0 &&
                      16 % M2_ == 0 && F_ % 16 == 0 && F_ <= 256 && IMG % 16 == 0 && STAGE % 16 == 0,
                  "fitting tile shape");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

using FitX3Water = FitX3<100, 16, 240>;
using FitX3Student = FitX3<32, 8, 64>;
using FitX3Paper = FitX3<128, 16, 240>;

template <class S>
__global__ void __launch_bounds__(128, 1) k_fit_x3(ModelDev md, const int32_t *__restrict__ order, int64_t pos_begin,
                                                  int64_t count, const float *__restrict__ T,
                                                  const unsigned char *__restrict__ img, double *__restrict__ E_atom,
                                                  float *__restrict__ dT, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_t[2], bar_m[2];
    __shared__ uint32_t tmem_base;
    constexpr int F = S::F, KC1 = S::KC1, KC2 = S::KC2, M2 = S::M2, M1 = S::M1;
    constexpr int AK = KC1 / M2;   // rows a of T per layer-1 chunk
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *Ah = smem + S::A_OFF, *Al = Ah + 128 * F * 2;
    unsigned char *Bst = smem + S::B_OFF;
    float *vec = reinterpret_cast<float *>(smem + S::V_OFF);
    const float *b1 = vec, *b2 = vec + F, *b3 = vec + 2 * F, *wo = vec + 3 * F;
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&bar_t[q], 1);
            tc::mbar_init(&bar_m[q], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    {
        const float *gv = reinterpret_cast<const float *>(img + S::VEC);
        for (int q = tid; q < 4 * F + 4; q += 128) vec[q] = gv[q];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    const uint32_t trow = tm + ((uint32_t)(warp * 32) << 16);
    const uint32_t tsc = trow + 256;   // t1 (FP32), then the derivative factors (1 - t1^2, 1 - t2^2)
    const float bout = vec[4 * F];
    const float inv2 = (float)(md.inv_nsel * md.inv_nsel);
    const uint32_t idF = tc::idesc_f16(128, F, 1), idN = tc::idesc_f16(128, S::NC, 1);
    uint32_t ph_t[2] = {0, 0}, ph_m[2] = {0, 0};
    bool loaded[2] = {false, false}, pend[2] = {false, false};
    bool dead = false;
    const int64_t ntiles = (count + 127) / 128;
    auto waitv = [&](uint64_t *bar, uint32_t &ph) {
        const bool ok = tc::mbar_wait(bar, ph, kWaitLimit);
        ph ^= 1;
        return __syncthreads_and(ok) != 0;
    };
    auto issue = [&](int s, uint32_t off, uint32_t bytes) {
        if (tid == 0) {
            tc::mbar_expect_tx(&bar_t[s], bytes);
            tc::bulk_g2s(Bst + s * S::STAGE, img + off, bytes, &bar_t[s]);
        }
        loaded[s] = true;
    };
    auto free_stage = [&](int s) {   // the MMAs that read stage s are done
        if (pend[s]) {
            pend[s] = false;
            if (!waitv(&bar_m[s], ph_m[s])) return false;
        }
        return true;
    };
    auto arrived = [&](int s) {   // the chunk copied into stage s is in shared memory
        loaded[s] = false;
        return waitv(&bar_t[s], ph_t[s]);
    };
    auto mma3_chunk = [&](uint32_t d, const unsigned char *ah, const unsigned char *al, uint32_t a_sbo, int s,
                          uint32_t half, uint32_t b_sbo, int K, uint32_t id, bool acc0) {
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t bh = tc::smem_u32(Bst + s * S::STAGE), bl = bh + half;
            mma_k_sbo(d, tc::smem_u32(ah), a_sbo, bh, b_sbo, K, id, acc0);
            mma_k_sbo(d, tc::smem_u32(ah), a_sbo, bl, b_sbo, K, id, true);
            mma_k_sbo(d, tc::smem_u32(al), a_sbo, bh, b_sbo, K, id, true);
            tc::mma_commit(&bar_m[s]);
        }
        pend[s] = true;
    };
    // d (+)= (the resident activations, K = F) x the B chunks at img + off + c * C2 (K chunks of KC2),
    // after every thread's A writes
    auto gemm_res = [&](uint32_t d, uint32_t off, bool acc0) -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        issue(0, off, S::C2);
        for (int c = 0; c < S::NK2; ++c) {
            const int s = c & 1;
            if (c + 1 < S::NK2) {
                if (!free_stage(1 - s)) return false;
                issue(1 - s, off + (uint32_t)(c + 1) * S::C2, S::C2);
            }
            if (!arrived(s)) return false;
            mma3_chunk(d, Ah + c * (KC2 / 8) * 128, Al + c * (KC2 / 8) * 128, (F / 8) * 128, s, F * KC2 * 2,
                       (KC2 / 8) * 128, KC2, idF, acc0 || c > 0);
        }
        for (int s = 0; s < 2; ++s)
            if (!free_stage(s)) return false;
        tc::fence_after_sync();
        return true;
    };
    for (int64_t tile = blockIdx.x; tile < ntiles && !dead; tile += gridDim.x) {
        const int64_t r0 = tile * 128 + tid;
        const bool valid = r0 < count;
        const int atom = valid ? order[pos_begin + r0] : 0;
        const float4 *Ta = reinterpret_cast<const float4 *>(T + (int64_t)atom * 4 * M1);
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 tb[M2];
#pragma unroll
        for (int b = 0; b < M2; ++b) tb[b] = valid ? Ta[b] : zero4;
        // ---- layer 1: z1 = D W1 in K chunks of KC1; D built chunk by chunk (hi, lo) while the tensor
        // core runs the previous chunk
        issue(0, S::W1T, S::C1);
        for (int c = 0; c < S::NK1 && !dead; ++c) {
            const int s = c & 1;
            unsigned char *sh = smem + S::A_OFF + s * S::DCH, *sl = sh + 128 * KC1 * 2;
            float4 cur[AK];
#pragma unroll
            for (int q = 0; q < AK; ++q) cur[q] = valid ? Ta[c * AK + q] : zero4;
#pragma unroll
            for (int c8 = 0; c8 < KC1; c8 += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 ta = cur[(c8 + u) / M2];
                    const float4 t2 = tb[(c8 + u) % M2];
                    v[u] = (ta.x * t2.x + ta.y * t2.y + ta.z * t2.z + ta.w * t2.w) * inv2;
                }
                st8_k(sh, sl, tid, c8, KC1, v);
            }
            tc::fence_async_smem();
            if (c + 1 < S::NK1) {
                if (!free_stage(1 - s)) { dead = true; break; }
                issue(1 - s, S::W1T + (uint32_t)(c + 1) * S::C1, S::C1);
            }
            tc::fence_before_sync();
            __syncthreads();
            if (!arrived(s)) { dead = true; break; }
            mma3_chunk(tm, sh, sl, (KC1 / 8) * 128, s, F * KC1 * 2, (KC1 / 8) * 128, KC1, idF, c > 0);
        }
        for (int s = 0; s < 2 && !dead; ++s)
            if (!free_stage(s)) dead = true;
        if (dead) break;
        tc::fence_after_sync();
        // layer-1 epilogue: t1 = tanh(z1 + b1) (plain layer), kept in tensor memory for layer 2
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            uint32_t w[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                v[u] = tanhf(z[u] + b1[c0 + u]);
                w[u] = __float_as_uint(v[u]);
            }
            tc::tmem_st16(tsc + c0, w);
            st8_k(Ah, Al, tid, c0, F, v);
            st8_k(Ah, Al, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_res(tm, S::W2T, false)) { dead = true; break; }
        // layer-2 epilogue: y2 = t1 + t2; E gets y2 . w now (y3 = y2 + t3); the derivative factors of
        // layers 1 and 2 replace t1
        float e = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], t1[16], v[16];
            uint32_t w[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld16(tsc + c0, t1);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = c0 + u;
                const float t = tanhf(z[u] + b2[k]);
                v[u] = t1[u] + t;
                e = fmaf(v[u], wo[k], e);
                w[u] = unorm16_pair(1.f - t1[u] * t1[u], 1.f - t * t);
            }
            tc::tmem_st16(tsc + c0, w);
            st8_k(Ah, Al, tid, c0, F, v);
            st8_k(Ah, Al, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_res(tm, S::W3T, false)) { dead = true; break; }
        // layer-3 epilogue: E_i = (y2 + t3) . w + b (FP32), dz3 = w (1 - t3^2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = c0 + u;
                const float t = tanhf(z[u] + b3[k]);
                e = fmaf(t, wo[k], e);
                v[u] = wo[k] * (1.f - t * t);
            }
            st8_k(Ah, Al, tid, c0, F, v);
            st8_k(Ah, Al, tid, c0 + 8, F, v + 8);
        }
        if (valid) E_atom[atom] = (double)(e + bout);
        if (!gemm_res(tm, S::W3B, false)) { dead = true; break; }
        // dE/dy2 epilogue: dy2 = dz3 W3^T + w (skip of layer 3), dz2 = dy2 (1 - t2^2); dy2 goes back
        // into the accumulator, so that the next product adds dz2 W2^T to it (the skip of layer 2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            uint32_t w[16], pk[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld16(tsc + c0, reinterpret_cast<float *>(pk));
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const float dy2 = z[u] + wo[c0 + u];
                v[u] = dy2 * ((float)(pk[u] >> 16) * (1.f / 65535.f));
                w[u] = __float_as_uint(dy2);
            }
            tc::tmem_st16(trow + c0, w);
            st8_k(Ah, Al, tid, c0, F, v);
            st8_k(Ah, Al, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_res(tm, S::W2B, true)) { dead = true; break; }
        // dE/dy1 epilogue: dy1 = dy2 + dz2 W2^T (from the accumulator), dz1 = dy1 (1 - t1^2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            uint32_t pk[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld16(tsc + c0, reinterpret_cast<float *>(pk));
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = z[u] * ((float)(pk[u] & 0xffffu) * (1.f / 65535.f));
            st8_k(Ah, Al, tid, c0, F, v);
            st8_k(Ah, Al, tid, c0 + 8, F, v + 8);
        }
        // dE/dD = dz1 W1^T in N chunks of NC, folded into dE/dT as soon as each chunk is read
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        float4 dtb[M2];
#pragma unroll
        for (int b = 0; b < M2; ++b) dtb[b] = zero4;
        float4 *dTa = reinterpret_cast<float4 *>(dT + (int64_t)atom * 4 * M1);
        issue(0, S::W1B, S::CB1);
        for (int j = 0; j < S::NB1 && !dead; ++j) {
            const int s = j & 1;
            if (j + 1 < S::NB1) {
                if (!free_stage(1 - s)) { dead = true; break; }
                issue(1 - s, S::W1B + (uint32_t)(j + 1) * S::CB1, S::CB1);
            }
            if (!arrived(s)) { dead = true; break; }
            const uint32_t reg = (uint32_t)s * 256;
            mma3_chunk(tm + reg, Ah, Al, (F / 8) * 128, s, S::NC * F * 2, (F / 8) * 128, F, idN, false);
            if (!free_stage(s)) { dead = true; break; }
            tc::fence_after_sync();
            constexpr int HS = M2 < 16 ? M2 : 16;
            const int a0 = (j * S::NC) / M2;
#pragma unroll
            for (int c0 = 0; c0 < S::NC; c0 += 16) {
                float z[16];
                tc::tmem_ld16(trow + reg + c0, z);
                tc::tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 16; h += HS) {
                    const int a = a0 + (c0 + h) / M2;
                    const float4 ta = valid ? Ta[a] : zero4;
                    float4 acc = zero4;
#pragma unroll
                    for (int u = 0; u < HS; ++u) {
                        const int b = (c0 + h + u) % M2;
                        const float dd = z[h + u];
                        acc.x = fmaf(dd, tb[b].x, acc.x);
                        acc.y = fmaf(dd, tb[b].y, acc.y);
                        acc.z = fmaf(dd, tb[b].z, acc.z);
                        acc.w = fmaf(dd, tb[b].w, acc.w);
                        dtb[b].x = fmaf(dd, ta.x, dtb[b].x);
                        dtb[b].y = fmaf(dd, ta.y, dtb[b].y);
                        dtb[b].z = fmaf(dd, ta.z, dtb[b].z);
                        dtb[b].w = fmaf(dd, ta.w, dtb[b].w);
                    }
                    if (valid) dTa[a] = make_float4(acc.x * inv2, acc.y * inv2, acc.z * inv2, acc.w * inv2);
                }
            }
        }
        if (dead) break;
        if (valid) {
#pragma unroll
            for (int b = 0; b < M2; ++b) {
                float4 o = dTa[b];
                o.x += dtb[b].x * inv2;
                o.y += dtb[b].y * inv2;
                o.z += dtb[b].z * inv2;
                o.w += dtb[b].w * inv2;
                dTa[b] = o;
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (dead) {
        // a wait gave up: flag it, then wait (bounded again) for this CTA's own copies and products
        // still in flight before the tensor memory is freed
        if (tid == 0) {
            atomicOr(err, 1);
            for (int s = 0; s < 2; ++s) {
                if (loaded[s]) tc::mbar_wait(&bar_t[s], ph_t[s], kWaitLimit);
                if (pend[s]) tc::mbar_wait(&bar_m[s], ph_m[s], kWaitLimit);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// hi and lo of w at element (r, k) of a K-major tile with K columns, in a chunk whose lo half starts
// `half` bytes after its hi half.
inline void put_x3(unsigned char *chunk, uint32_t half, int r, int k, int K, double w)
{
    const __nv_bfloat16 h = __double2bfloat16(w);
    const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
    memcpy(chunk + tc::kmaj_off(r, k, K), &h, 2);
    memcpy(chunk + half + tc::kmaj_off(r, k, K), &l, 2);
}

template <class FS>
void pack_fit_x3(const double *p, const NetLayout &L, unsigned char *out)
{
    memset(out, 0, FS::IMG);
    constexpr int F = FS::F, KC1 = FS::KC1, KC2 = FS::KC2, NC = FS::NC;
    const double *W1 = p + L.W[0], *W2 = p + L.W[1], *W3 = p + L.W[2];
    for (int d = 0; d < FS::D; ++d)
        for (int o = 0; o < F; ++o) {
            const double w = W1[(int64_t)d * F + o];
            put_x3(out + FS::W1T + (uint32_t)(d / KC1) * FS::C1, F * KC1 * 2, o, d % KC1, KC1, w);   // [o][d]
            put_x3(out + FS::W1B + (uint32_t)(d / NC) * FS::CB1, NC * F * 2, d % NC, o, F, w);       // [d][o]
        }
    for (int k = 0; k < F; ++k)
        for (int o = 0; o < F; ++o) {
            const double w2 = W2[k * F + o], w3 = W3[k * F + o];
            put_x3(out + FS::W2T + (uint32_t)(k / KC2) * FS::C2, F * KC2 * 2, o, k % KC2, KC2, w2);   // [o][k]
            put_x3(out + FS::W3T + (uint32_t)(k / KC2) * FS::C2, F * KC2 * 2, o, k % KC2, KC2, w3);
            put_x3(out + FS::W2B + (uint32_t)(o / KC2) * FS::C2, F * KC2 * 2, k, o % KC2, KC2, w2);   // [k][o]
            put_x3(out + FS::W3B + (uint32_t)(o / KC2) * FS::C2, F * KC2 * 2, k, o % KC2, KC2, w3);
        }
    float *vec = reinterpret_cast<float *>(out + FS::VEC);
    for (int k = 0; k < F; ++k) {
        vec[k] = (float)p[L.b[0] + k];
        vec[F + k] = (float)p[L.b[1] + k];
        vec[2 * F + k] = (float)p[L.b[2] + k];
        vec[3 * F + k] = (float)p[L.W[3] + k];
    }
    vec[4 * F] = (float)p[L.b[3]];
}

// 1, 2, 3: the fitting shapes with a split-bf16 tensor-core kernel (three equal hidden widths after a
// plain first layer); 0: none (the FP32 CUDA-core fitting net is used).
int fit_x3_kind(const ModelDev &md)
{
    if (md.n_fit != 3 || md.fit.wout[0] != md.fit.wout[1] || md.fit.wout[1] != md.fit.wout[2]) return 0;
    const int F = md.fit.wout[0];
    if (md.m1 == 100 && md.m2 == 16 && F == 240) return 1;
    if (md.m1 == 32 && md.m2 == 8 && F == 64) return 2;
    if (md.m1 == 128 && md.m2 == 16 && F == 240) return 3;
    return 0;
}

template <class FS>
dp_status pack_fit_x3_all(dp_model *m)
{
    const ModelDev &md = m->dev;
    std::vector<unsigned char> img((size_t)md.ntypes * FS::IMG);
    for (int t = 0; t < md.ntypes; ++t)
        pack_fit_x3<FS>(m->h_params.data() + md.fit_base + t * md.fit.size, md.fit, img.data() + (size_t)t * FS::IMG);
    if (!m->d_tcfit_x3) DP_CUDA(cudaMalloc((void **)&m->d_tcfit_x3, img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_tcfit_x3, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return DP_OK;
}

dp_status pack_fit_x3_weights(dp_model *m)
{
    switch (fit_x3_kind(m->dev)) {
    case 1: return pack_fit_x3_all<FitX3Water>(m);
    case 2: return pack_fit_x3_all<FitX3Student>(m);
    case 3: return pack_fit_x3_all<FitX3Paper>(m);
    default: return DP_OK;
    }
}

template <class FS>
dp_status launch_fit_x3(dp_model *m, dp_nlist *nl, const float *T, int grid, double *E_atom, float *dT,
                        cudaStream_t st)
{
    const ModelDev &md = m->dev;
    DP_CUDA(cudaFuncSetAttribute(k_fit_x3<FS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::SMEM));
    for (int t = 0; t < md.ntypes; ++t) {
        const int64_t b = nl->type_off[t], cnt = nl->type_count[t];
        if (cnt <= 0) continue;
        const int64_t tiles = (cnt + 127) / 128;
        const unsigned g = (unsigned)(tiles < grid ? tiles : grid);
        ProfScope ps(m->prof, PG_FIT, 1, st);
        k_fit_x3<FS><<<g, 128, FS::SMEM, st>>>(md, nl->d_order, b, cnt, T, m->d_tcfit_x3 + (size_t)t * FS::IMG,
                                               E_atom, dT, m->d_err);
        DP_CUDA(cudaGetLastError());
    }
    return DP_OK;
}

dp_status fit_x3(dp_model *m, dp_nlist *nl, const float *T, int grid, double *E_atom, float *dT, cudaStream_t st)
{
    if (fit_cluster_enabled()) {
        const dp_status s = fit_cluster(m, nl, 2, T, E_atom, dT, st);
        if (s != DP_ERR_UNSUPPORTED) return s;
    }
    if (!m->d_tcfit_x3) DP_TRY(pack_fit_x3_weights(m));
    switch (fit_x3_kind(m->dev)) {
    case 1: return launch_fit_x3<FitX3Water>(m, nl, T, grid, E_atom, dT, st);
    case 2: return launch_fit_x3<FitX3Student>(m, nl, T, grid, E_atom, dT, st);
    case 3: return launch_fit_x3<FitX3Paper>(m, nl, T, grid, E_atom, dT, st);
    default: set_error("no split-bf16 fitting kernel for this shape"); return DP_ERR_UNSUPPORTED;
    }
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
    if (fit_x3_kind(md) != 0 && getenv("DP_SIMT_FIT") == nullptr) {
        DP_TRY(fit_x3(m, nl, T, nsm, d_atom_energy, dT, st));
    } else {
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
    }
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

DP_BOUNDS_ACCESSOR(bounds_read_tc_x3)

dp_status pack_x3_weights(dp_model *m)
{
    const int *e = m->dev.emb.wout;
    if (e[0] == 25) DP_TRY(pack_x3<TcWater>(m));
    else if (e[0] == 8) DP_TRY(pack_x3<TcStudent>(m));
    else DP_TRY(pack_x3<TcPaper>(m));
    return m->d_tcfit_x3 ? pack_fit_x3_weights(m) : DP_OK;
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

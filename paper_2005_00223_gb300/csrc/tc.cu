// MIX-16 scheme of Sec. 4.1.3 on the 5th-generation tensor cores (tcgen05):
// embedding layers 2 and 3 and their input gradients run as M = 128 MMAs with
// fp16 or bf16 operands in shared memory and FP32 accumulators in tensor
// memory; the first embedding layer (K = 1, too small for the tensor cores),
// tanh and its derivative run in FP32 on the CUDA cores, as the paper does.
// The minimum image, the distance and the switching function s(r), ds/dr are
// evaluated in FP64 once per evaluation by the formatting kernel, which
// stores (s, u = d/r) and (ds/dr, r) per neighbor slot as FP32; here the
// environment row R = (s, s u) and the chain dE/dR -> g_ij run in FP32, and
// the force / virial accumulation is FP64.
//
// Work unit: a tile of 128 neighbor rows = 4 chunks of 32 rows, one chunk per
// warp; every chunk is up to 32 neighbors of one type of one atom, and the 4
// chunks of a tile share the (center type, neighbor type) net.  Tiles are
// listed per evaluation (k_cb_count / k_cb_plan / k_cb_write); persistent CTAs walk them.  Each
// CTA keeps the packed weights of the current net in shared memory, loaded
// by one bulk copy on the TMA engine.
//
// Per tile, forward (k_embed_fwd_tc):  rows R -> layer 1 (FP32) -> A2 ->
//   MMA (A2 x W2) -> tanh / skip epilogue -> A3 -> MMA (A3 x W3) -> epilogue
//   gives G (fp16) -> contraction T_q = G^T R per chunk as MMAs with
//   MN-major operands (FP32 accumulators) -> atomics into T.
// Backward (k_embed_bwd_tc) recomputes the forward (no activation storage),
//   then dG = dT R, dR = dT^T G, dz3 -> MMA (dz3 x W3^T) -> dz2 -> MMA
//   (dz2 x W2^T) -> ds -> g_ij -> FP64 force and virial atomics.
// The descriptor D = T T<^T, the fitting net and dE/dT sit between the two.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "dp_internal.cuh"
#include "geom.cuh"
#include "tc_common.cuh"
#include "tc_embed.cuh"

namespace dp {

namespace {

template <class S, int BF>
__global__ void __launch_bounds__(kTcThreads) k_embed_fwd_tc(ModelDev md, const float4 *__restrict__ envA,
                                                            const int32_t *__restrict__ nlist,
                                                            const int32_t *__restrict__ nnei,
                                                            const int4 *__restrict__ chunks,
                                                            const int *__restrict__ ntiles_ptr,
                                                            const unsigned char *__restrict__ wimg,
                                                            float *__restrict__ T, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];   // no-swizzle operands and bulk copies: 16 B
    __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *img = smem;
    unsigned char *A2 = smem + S::F_A2_OFF;
    unsigned char *A3 = smem + S::F_A3_OFF;
    unsigned char *GT = smem + S::F_GT_OFF;   // over A2 and A3 (dead once the layer-3 MMA completed)
    unsigned char *RT = smem + S::F_RT_OFF;
    const float *vec = reinterpret_cast<const float *>(img + S::F_VEC_OFF);
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
    const uint32_t id2 = tc::idesc_f16(128, S::N2, BF), id3 = tc::idesc_f16(128, S::N3, BF);
    const uint32_t idT = tc::idesc_f16_mn(128, 16);
    uint32_t ph_mma = 0, ph_w = 0;
    int cur_net = -1;
    const int ntiles = *ntiles_ptr;
    RowIn nxt = fetch_row<false>(md, chunks, blockIdx.x, ntiles, warp, lane, nnei, nlist, envA, nullptr);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const RowIn in = nxt;
        nxt = fetch_row<false>(md, chunks, tile + gridDim.x, ntiles, warp, lane, nnei, nlist, envA, nullptr);
        const int net = in.net;
        if (net != cur_net) {
            // starved (test of the bounded waits): no copy is issued, so nothing is in flight
            // when the wait below gives up
            const bool starve = md.wait_test == WT_EMBED_FWD_WEIGHTS;
            if (tid == 0 && !starve) {   // W2^T and W3^T, then the vectors right after them
                tc::mbar_expect_tx(&mbar_w, S::B3B_OFF + S::VEC_BYTES);
                tc::bulk_g2s(img, wimg + (size_t)net * S::IMG, S::B3B_OFF, &mbar_w);
                tc::bulk_g2s(img + S::F_VEC_OFF, wimg + (size_t)net * S::IMG + S::VEC_OFF, S::VEC_BYTES, &mbar_w);
            }
            bool ok = tc::mbar_wait(&mbar_w, ph_w, starve ? (long)md.wait_short : kWaitLimit);
            ph_w ^= 1;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicOr(err, 1);
                break;
            }
            cur_net = net;
        }
        float Rf[4], t1[S::E0], t2[S::E1], geo[6];
        int j;
        bool valid;
        rows_layer1<S, BF, false>(in, lane, tid, vec, A2, Rf, t1, geo, j, valid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            tc::mma_kloop(tmem, tc::smem_u32(A2), tc::smem_u32(img + S::B2_OFF), S::K2, id2);
            tc::mma_commit(&mbar_mma);
        }
        bool ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        epi_layer2<S, BF>(taddr, vec, t1, t2, A3, tid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            tc::mma_kloop(tmem, tc::smem_u32(A3), tc::smem_u32(img + S::B3_OFF), S::N2, id3);
            tc::mma_commit(&mbar_mma);
        }
        ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        // layer-3 epilogue: G = skip(y2) + tanh(z3 + b3) in fp16 into G^T, this
        // thread's row R (zero on padded rows) into R^T
        {
            const float *b3 = vec + 2 * S::K2 + S::N2;
            float y2[S::E1];
#pragma unroll
            for (int k = 0; k < S::E1; ++k) y2[k] = skip_of<S::E0, S::E1>(t1, k) + t2[k];
            // the row's R^T entries c = 0..15 (c >= 4 zero) and G^T entries m = 0..127 (m >= E2 zero)
            // are all rewritten each tile: the region held A2 and A3 before
            *reinterpret_cast<uint4 *>(RT + tc::mnmaj_off(0, tid, 16)) =
                make_uint4(pack2<0>(Rf[0], Rf[1]), pack2<0>(Rf[2], Rf[3]), 0u, 0u);
            *reinterpret_cast<uint4 *>(RT + tc::mnmaj_off(8, tid, 16)) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int c0 = S::N3; c0 < 128; c0 += 8)
                *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0, tid, 128)) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int c0 = 0; c0 < S::N3; c0 += 16) {
                float z[16];
                tc::tmem_ld16(taddr + c0, z);
                tc::tmem_ld_wait();
                float g[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int m = c0 + u;
                    g[u] = m < S::E2 ? skip_of<S::E1, S::E2>(y2, m) + tc::tanh_fast(z[u] + b3[m]) : 0.f;
                }
                *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0, tid, 128)) =
                    make_uint4(pack2<0>(g[0], g[1]), pack2<0>(g[2], g[3]), pack2<0>(g[4], g[5]), pack2<0>(g[6], g[7]));
                *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0 + 8, tid, 128)) = make_uint4(
                    pack2<0>(g[8], g[9]), pack2<0>(g[10], g[11]), pack2<0>(g[12], g[13]), pack2<0>(g[14], g[15]));
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // chunk q: T_q[m][c] = sum over its 32 rows of G[row][m] R[row][c]
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tc::mma_kloop_mn(tmem + 16 * q, tc::smem_u32(GT), 128, tc::smem_u32(RT), 16, 32 * q, 32, idT,
                                 false);
            tc::mma_commit(&mbar_mma);
        }
        ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        // warp w holds channels m = 32 w + lane of every chunk's T
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

template <class S, int BF>
__global__ void __launch_bounds__(kTcThreads, S::B_CTAS >= 3 ? S::B_CTAS : 1) k_embed_bwd_tc(ModelDev md, const float4 *__restrict__ envA,
                                                            const float2 *__restrict__ envB,
                                                            const int32_t *__restrict__ nlist,
                                                            const int32_t *__restrict__ nnei,
                                                            const int4 *__restrict__ chunks,
                                                            const int *__restrict__ ntiles_ptr,
                                                            const unsigned char *__restrict__ wimg,
                                                            const float *__restrict__ dT, double *__restrict__ force,
                                                            double *__restrict__ atom_virial, int *err,
                                                            const unsigned *__restrict__ dT_max)
{
    extern __shared__ __align__(128) unsigned char smem[];   // no-swizzle operands and bulk copies: 16 B
    __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // fp16 operands: dE/dT (which carries 1/sum(sel)^2) is scaled by a power of two 2^-e so that its
    // largest entry lies in [1, 2), keeping dz3 and dz2 in fp16's normal range; g is scaled back
    // exactly before the force and virial sums (bf16 has FP32's range and needs no scaling)
    float gscale = 1.f, ginv = 1.f;
    if (BF == 0 && dT_max != nullptr) {
        const unsigned bits = *dT_max;
        const int e = (int)((bits >> 23) & 0xffu) - 127;
        if (bits != 0u && e > -126 && e < 127) {
            gscale = __int_as_float((127 - e) << 23);
            ginv = __int_as_float((127 + e) << 23);
        }
    }
    unsigned char *img = smem;
    unsigned char *A2 = smem + S::B_A2_OFF;
    unsigned char *A3 = smem + S::B_A3_OFF;     // forward layer-3 input, then dz2
    unsigned char *AB1 = smem + S::B_AB1_OFF;   // dz3, over A2 and A3
    float *sdT = reinterpret_cast<float *>(smem + S::B_X_OFF) + warp * 4 * S::E2;
    const float *vec = reinterpret_cast<const float *>(img + S::VEC_OFF);
    if (tid == 0) {
        tc::mbar_init(&mbar_mma, 1);
        tc::mbar_init(&mbar_w, 1);
        tc::mbar_init_fence();
    }
    // With three CTAs per SM (128 TMEM columns each) every product starts at column 0 and the skip
    // terms of dY2 and dY1 go into the accumulator before their MMA; with two, the layer-3 and dY1
    // products sit after column N2 and the skip terms stay in registers (fewer TMEM round trips)
    constexpr bool kRes = S::B_CTAS >= 3;
    constexpr uint32_t kCols = kRes ? S::F_TCOLS : (uint32_t)kTmemCols;
    constexpr uint32_t kHi = kRes ? 0u : (uint32_t)S::N2;   // column of the layer-3 and dY1 products
    if (warp == 0) tc::tmem_alloc(&tmem_base, kCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t id2 = tc::idesc_f16(128, S::N2, BF), id3 = tc::idesc_f16(128, S::N3, BF);
    const uint32_t idb1 = tc::idesc_f16(128, S::N2, BF), idb2 = tc::idesc_f16(128, S::K2, BF);
    uint32_t ph_mma = 0, ph_w = 0;
    int cur_net = -1;
    const int ntiles = *ntiles_ptr;
    RowIn nxt = fetch_row<true>(md, chunks, blockIdx.x, ntiles, warp, lane, nnei, nlist, envA, envB);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const RowIn in = nxt;
        nxt = fetch_row<true>(md, chunks, tile + gridDim.x, ntiles, warp, lane, nnei, nlist, envA, envB);
        const int net = in.net;
        const TileCtx ch = in.ch;
        if (net != cur_net) {
            if (tid == 0) {
                tc::mbar_expect_tx(&mbar_w, S::IMG);
                tc::bulk_g2s(img, wimg + (size_t)net * S::IMG, S::IMG, &mbar_w);
            }
            bool ok = tc::mbar_wait(&mbar_w, ph_w, kWaitLimit);
            ph_w ^= 1;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicOr(err, 1);
                break;
            }
            cur_net = net;
        }
        // dE/dT of this warp's atom (already scaled by 1/sum(sel))
        for (int q = lane; q < 4 * S::E2; q += 32)
            sdT[q] = ch.atom >= 0 ? dT[(int64_t)ch.atom * 4 * S::E2 + q] * gscale : 0.f;
        float Rf[4], t1[S::E0], t2[S::E1], geo[6];
        int j;
        bool valid;
        rows_layer1<S, BF, true>(in, lane, tid, vec, A2, Rf, t1, geo, j, valid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            tc::mma_kloop(tmem, tc::smem_u32(A2), tc::smem_u32(img + S::B2_OFF), S::K2, id2);
            tc::mma_commit(&mbar_mma);
        }
        bool ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        epi_layer2<S, BF>(taddr, vec, t1, t2, A3, tid);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            tc::mma_kloop(tmem + kHi, tc::smem_u32(A3), tc::smem_u32(img + S::B3_OFF), S::N2, id3);
            tc::mma_commit(&mbar_mma);
        }
        ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        // layer-3 epilogue fused with the start of the backward pass:
        //   G = skip(y2) + t3,  dG = dT R,  dR += dT^T G,  dz3 = dG (1 - t3^2)
        float dR[4] = {0.f, 0.f, 0.f, 0.f};
        float res2[S::E1];   // skip terms of dE/dy2
#pragma unroll
        for (int k = 0; k < S::E1; ++k) res2[k] = 0.f;
        {
            const float *b3 = vec + 2 * S::K2 + S::N2;
            float y2[kRes ? 1 : S::E1];   // with two CTAs per SM the layer-2 outputs are materialised
            if constexpr (!kRes) {
#pragma unroll
                for (int k = 0; k < S::E1; ++k) y2[k] = skip_of<S::E0, S::E1>(t1, k) + t2[k];
            }
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
                        const float t = tc::tanh_fast(z[u] + b3[m]);
                        // skip of layer 3 from y2 = skip(t1) + t2 (with three CTAs per SM evaluated
                        // where it is used)
                        float sk = 0.f;
                        if constexpr (kRes) {
                            if (S::E2 == S::E1 || S::E2 == 2 * S::E1) {
                                const int k2 = m % S::E1;
                                sk = skip_of<S::E0, S::E1>(t1, k2) + t2[k2];
                            }
                        } else {
                            sk = skip_of<S::E1, S::E2>(y2, m);
                        }
                        const float G = sk + t;
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
                st_row8<BF>(AB1, tid, c0, S::N3, buf);
                st_row8<BF>(AB1, tid, c0 + 8, S::N3, buf + 8);
            }
            if (kRes) {   // this row's layer-3 accumulators are all read: its dY2 columns start as the skip terms
#pragma unroll
                for (int c0 = 0; c0 < S::N2; c0 += 16) {
                    uint32_t w[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) w[u] = __float_as_uint(c0 + u < S::E1 ? res2[c0 + u] : 0.f);
                    tc::tmem_st16(taddr + c0, w);
                }
                tc::tmem_st_wait();
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // dY2 = dz3 x W3^T: B rows are the outputs k of W3's input side (W3 [E1][E2] row-major)
            tc::mma_kloop(tmem, tc::smem_u32(AB1), tc::smem_u32(img + S::B3B_OFF), S::N3, idb1, kRes);
            tc::mma_commit(&mbar_mma);
        }
        ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        tc::fence_after_sync();
        float res1[S::E0];   // skip terms of dE/dy1
#pragma unroll
        for (int k = 0; k < S::E0; ++k) res1[k] = 0.f;
        {
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
                    const float dy2 = kRes ? z[u] : z[u] + res2[k];   // kRes: started from the skip terms
                    v = dy2 * (1.f - t2[k] * t2[k]);
                    if (S::E1 == S::E0) res1[k] += dy2;
                    else if (S::E1 == 2 * S::E0) res1[k % S::E0] += dy2;
                }
                buf[u] = v;
            }
            st_row8<BF>(A3, tid, c0, S::N2, buf);
            st_row8<BF>(A3, tid, c0 + 8, S::N2, buf + 8);
        }
        if (kRes) {   // this row's dY2 accumulators are all read: its dY1 columns start as the skip terms
#pragma unroll
            for (int c0 = 0; c0 < S::K2; c0 += 16) {
                uint32_t w[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) w[u] = __float_as_uint(c0 + u < S::E0 ? res1[c0 + u] : 0.f);
                tc::tmem_st16(taddr + c0, w);
            }
            tc::tmem_st_wait();
        }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            // dY1 = dz2 x W2^T
            tc::mma_kloop(tmem + kHi, tc::smem_u32(A3), tc::smem_u32(img + S::B2B_OFF), S::N2, idb2, kRes);
            tc::mma_commit(&mbar_mma);
        }
        ok = tc::mbar_wait(&mbar_mma, ph_mma, kWaitLimit);
        ph_mma ^= 1;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
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
                        const float dy1 = kRes ? z[u] : z[u] + res1[k];   // kRes: started from the skip terms
                        ds = fmaf(dy1 * (1.f - t1[k] * t1[k]), W1[k], ds);
                        if (S::E0 == 1) ds += dy1;
                        else if (S::E0 == 2) ds += dy1;
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
            for (int k = 0; k < 3; ++k) gv[k] = fmaf(cu, geo[k], geo[5] * dR[1 + k]) * ginv;
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
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// *out = bit pattern of max |x| over x [n] (non-negative floats order like their bits); *out zeroed
// by the caller.
__global__ void k_absmax_bits(int64_t n, const float *__restrict__ x, unsigned *out)
{
    unsigned m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned b = __float_as_uint(fabsf(x[i]));
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Work list: for each (center type, neighbor type) group, the 32-neighbor
// chunks of its atoms (type-sorted order), padded with empty chunks to a
// multiple of 4 so that a tile never mixes nets.  Entry = {atom, tj, first
// slot, net}.  Built by three kernels: per 1024 positions, an exclusive scan
// of the chunk counts (k_cb_count); one block scanning the block sums and
// placing the groups (k_cb_plan); the scatter of the entries (k_cb_write).
constexpr int kCbThreads = 1024;

// Exclusive scan of v over the block (kCbThreads threads); *total = sum.
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int *total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? warp_sums[w - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return incl - v;
}

// loc[tj][p] = chunks of positions [block start, p) for neighbor type tj;
// bsum[tj][block] = the block's total.
__global__ void __launch_bounds__(kCbThreads) k_cb_count(ModelDev md, int64_t n, const int32_t *__restrict__ order,
                                                        const int32_t *__restrict__ nnei, int *__restrict__ loc,
                                                        int *__restrict__ bsum, int nb)
{
    __shared__ int ws[32];
    const int64_t p = blockIdx.x * (int64_t)kCbThreads + threadIdx.x;
    const int a = p < n ? order[p] : 0;
    for (int tj = 0; tj < md.ntypes; ++tj) {
        const int c = p < n ? (nnei[(int64_t)a * md.ntypes + tj] + 31) >> 5 : 0;
        int total;
        const int ex = block_excl_scan(c, ws, &total);
        if (p < n) loc[(int64_t)tj * n + p] = ex;
        if (threadIdx.x == 0) bsum[tj * nb + blockIdx.x] = total;
    }
}

// One block: boff[tj][b] = exclusive scan of bsum[tj][.]; per group (ti, tj)
// its first entry gbase and the chunk prefix tstart at its first position;
// the padding entries; the tile count.
// The type ranges of the positions, passed by value (no host-to-device copy, which from pageable
// memory would wait for the stream).
struct TypeTab {
    int64_t off[kMaxTypes], cnt[kMaxTypes];
};

__global__ void __launch_bounds__(kCbThreads) k_cb_plan(ModelDev md, int64_t n, TypeTab tt,
                                                       const int *__restrict__ loc, const int *__restrict__ bsum,
                                                       int *__restrict__ boff, int nb, int *__restrict__ gtab,
                                                       int4 *__restrict__ chunks, int *__restrict__ ntiles)
{
    __shared__ int ws[32];
    __shared__ int tot[kMaxTypes];
    for (int tj = 0; tj < md.ntypes; ++tj) {
        int carry = 0;
        for (int b0 = 0; b0 < nb; b0 += kCbThreads) {
            const int b = b0 + threadIdx.x;
            const int v = b < nb ? bsum[tj * nb + b] : 0;
            int total;
            const int ex = block_excl_scan(v, ws, &total);
            if (b < nb) boff[tj * nb + b] = carry + ex;
            carry += total;
        }
        if (threadIdx.x == 0) tot[tj] = carry;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // prefix of neighbor type tj at position q (q <= n)
    auto prefix = [&](int tj, int64_t q) -> int {
        if (q >= n) return tot[tj];
        return boff[tj * nb + (int)(q / kCbThreads)] + loc[(int64_t)tj * n + q];
    };
    int base = 0;
    for (int ti = 0; ti < md.ntypes; ++ti) {
        for (int tj = 0; tj < md.ntypes; ++tj) {
            const int net = ti * md.ntypes + tj;
            const int s0 = prefix(tj, tt.off[ti]);
            const int s1 = prefix(tj, tt.off[ti] + tt.cnt[ti]);
            const int total = tt.cnt[ti] > 0 ? s1 - s0 : 0;
            gtab[2 * net] = base;
            gtab[2 * net + 1] = s0;
            for (int q = total; q % 4 != 0; ++q) chunks[base + q] = make_int4(-1, tj, 0, net);
            base += (total + 3) / 4 * 4;
        }
    }
    *ntiles = base / 4;
}

// Entry {atom, tj, first slot, net}; with firstc (the FP64 work list of a
// batch) {atom, position in the batch, first slot, net} instead, and
// firstc[p * ntypes + tj] = the index of the first chunk of (p, tj).
__global__ void __launch_bounds__(kCbThreads) k_cb_write(ModelDev md, int64_t n, const int32_t *__restrict__ order,
                                                        const int32_t *__restrict__ type,
                                                        const int32_t *__restrict__ nnei, const int *__restrict__ loc,
                                                        const int *__restrict__ boff, int nb,
                                                        const int *__restrict__ gtab, int4 *__restrict__ chunks,
                                                        int *__restrict__ firstc)
{
    const int64_t p = blockIdx.x * (int64_t)kCbThreads + threadIdx.x;
    if (p >= n) return;
    const int a = order[p], ti = type[a];
    for (int tj = 0; tj < md.ntypes; ++tj) {
        const int nch = (nnei[(int64_t)a * md.ntypes + tj] + 31) >> 5;
        const int net = ti * md.ntypes + tj;
        const int dst = gtab[2 * net] + boff[tj * nb + blockIdx.x] + loc[(int64_t)tj * n + p] - gtab[2 * net + 1];
        if (firstc) firstc[p * md.ntypes + tj] = dst;
        for (int c = 0; c < nch; ++c) chunks[dst + c] = make_int4(a, firstc ? (int)p : tj, c * 32, net);
    }
}

// Fitting net of the MIX-16 scheme on the tensor cores (tcgen05), fused with
// the descriptor and its adjoint.  One persistent CTA per SM walks tiles of
// 128 atoms of one center type (thread = atom row):
//   D = T T<^T (times 1/sum(sel)^2) is built straight into the A operand,
//     64 columns at a time, while the tensor core consumes the previous
//     chunk (two stages; W1^T chunks arrive by bulk copies on the TMA engine);
//   three hidden layers y_k = skip + tanh(z_k) with M = 128, N = K = F MMAs,
//     tanh, skip and bias in FP32 epilogues; E_i = y3 . w + b in FP32;
//   the backward: dz3 = w (1 - t3^2) -> MMA with W3 -> dz2 -> MMA with W2 ->
//     dz1 -> MMA with W1 in N-chunks -> dE/dD, folded at once into
//     dE/dT[a][c] = sum_b dD[a][b] T[b][c] + [a < M2] sum_a' dD[a'][a] T[a'][c].
// D and dE/dD never reach HBM.  Operands are fp16 or bf16, accumulators FP32
// in TMEM; the last layer and E_i stay FP32 as the paper prescribes.

template <int M1_, int M2_, int F_>
struct FitShape {
    static constexpr int M1 = M1_, M2 = M2_, F = F_, D = M1_ * M2_;
    static constexpr int KC = 64;                       // K chunk of layer 1
    static constexpr int NK1 = D / KC;
    static constexpr int NC = (D % 160 == 0) ? 160 : 128;   // N chunk of the layer-1 input gradient
    static constexpr int NB1 = D / NC;
    static_assert(D % KC == 0 && D % NC == 0 && NC % M2_ == 0 && KC % M2_ == 0 && 16 % M2_ == 0 && F_ % 16 == 0 &&
                      F_ <= 256, "fitting tile shape");
    // packed weight image per center type (bytes)
    static constexpr uint32_t W1T_OFF = 0;                                  // NK1 x [F][KC]
    static constexpr uint32_t W2T_OFF = W1T_OFF + NK1 * F * KC * 2;         // [F][F], (o, k) = W2[k][o]
    static constexpr uint32_t W3T_OFF = W2T_OFF + F * F * 2;
    static constexpr uint32_t W3B_OFF = W3T_OFF + F * F * 2;                // [F][F], (k, o) = W3[k][o]
    static constexpr uint32_t W2B_OFF = W3B_OFF + F * F * 2;
    static constexpr uint32_t W1B_OFF = W2B_OFF + F * F * 2;                // NB1 x [NC][F], (d, o) = W1[d][o]
    static constexpr uint32_t VEC_OFF = W1B_OFF + NB1 * NC * F * 2;         // b1, b2, b3, w_out [F]; b_out
    static constexpr uint32_t IMG = VEC_OFF + (4 * F + 4) * 4;
    // shared memory
    static constexpr uint32_t ABUF = (128 * F * 2 > 2 * 128 * KC * 2) ? 128 * F * 2 : 2 * 128 * KC * 2;
    static constexpr uint32_t BB1 = F * F * 2, BB2 = 2 * F * KC * 2, BB3 = NC * F * 2;
    static constexpr uint32_t BBUF = BB1 > BB2 ? (BB1 > BB3 ? BB1 : BB3) : (BB2 > BB3 ? BB2 : BB3);
    static constexpr uint32_t A_OFF = 0, B_OFF = ABUF, V_OFF = ABUF + BBUF;
    static constexpr uint32_t SMEM = V_OFF + (4 * F + 4) * 4;
};



template <class S, int BF>
__global__ void __launch_bounds__(128, 1) k_fit_tc(ModelDev md, const int32_t *__restrict__ order, int64_t pos_begin,
                                                  int64_t count, const float *__restrict__ T,
                                                  const unsigned char *__restrict__ img, double *__restrict__ E_atom,
                                                  float *__restrict__ dT, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_t[2], bar_m[2];
    __shared__ uint32_t tmem_base;
    constexpr int F = S::F, KC = S::KC, M2 = S::M2, M1 = S::M1;
    constexpr int AK = KC / M2;                 // rows a of T per K chunk of layer 1
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *A = smem + S::A_OFF, *B = smem + S::B_OFF;
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
        const float *gv = reinterpret_cast<const float *>(img + S::VEC_OFF);
        for (int q = tid; q < 4 * F + 4; q += 128) vec[q] = gv[q];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    const uint32_t trow = tm + ((uint32_t)(warp * 32) << 16);
    // columns 256.. of this row: t1 (FP32) after layer 1, then the packed
    // derivative factors (1 - t1^2, 1 - t2^2) as fp16 pairs until the backward
    const uint32_t tsc = trow + 256;
    const float bout = vec[4 * F];
    const float inv2 = (float)(md.inv_nsel * md.inv_nsel);
    const uint32_t idF = tc::idesc_f16(128, F, BF), idN = tc::idesc_f16(128, S::NC, BF);
    uint32_t ph_t[2] = {0, 0}, ph_m[2] = {0, 0};
    bool dead = false;
    const int64_t ntiles = (count + 127) / 128;
    // one wait by every thread, then a block-wide vote; false when any thread gave up
    auto waitv = [&](uint64_t *bar, uint32_t &ph) {
        bool ok = tc::mbar_wait(bar, ph, kWaitLimit);
        ph ^= 1;
        return __syncthreads_and(ok) != 0;
    };
    auto mma = [&](uint32_t d, const unsigned char *a, const unsigned char *b, int K, uint32_t id, bool acc0) {
        const uint32_t sbo = (uint32_t)(K >> 3) * 128;
        for (int ks = 0; ks < (K >> 4); ++ks) {
            uint64_t ad = tc::smem_desc(tc::smem_u32(a) + ks * 256, 128, sbo);
            uint64_t bd = tc::smem_desc(tc::smem_u32(b) + ks * 256, 128, sbo);
            uint32_t acc = (acc0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                "l"(ad), "l"(bd), "r"(id), "r"(acc));
        }
    };
    auto load_b = [&](int s, uint32_t off, uint32_t bytes, unsigned char *dst) {
        if (tid == 0) {
            tc::mbar_expect_tx(&bar_t[s], bytes);
            tc::bulk_g2s(dst, img + off, bytes, &bar_t[s]);
        }
    };
    // one GEMM over the full A tile (K = F) after the A (and TMEM) writes of every thread
    auto gemm_full = [&](uint32_t d, int N_id_is_F, bool acc0) -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (!waitv(&bar_t[0], ph_t[0])) return false;
        if (tid == 0) {
            tc::fence_after_sync();
            mma(d, A, B, F, N_id_is_F ? idF : idN, acc0);
            tc::mma_commit(&bar_m[0]);
        }
        if (!waitv(&bar_m[0], ph_m[0])) return false;
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
        // ---- layer 1: D x W1, K in chunks of KC, two stages; the T rows of
        // the next chunk are loaded while this one is built
        float4 nxt[AK];
#pragma unroll
        for (int q = 0; q < AK; ++q) nxt[q] = valid ? Ta[q] : zero4;
        for (int kc = 0; kc < S::NK1; ++kc) {
            const int s = kc & 1;
            if (kc >= 2 && !waitv(&bar_m[s], ph_m[s])) { dead = true; break; }
            load_b(s, S::W1T_OFF + (uint32_t)kc * F * KC * 2, F * KC * 2, B + s * F * KC * 2);
            float4 cur[AK];
#pragma unroll
            for (int q = 0; q < AK; ++q) cur[q] = nxt[q];
            if (kc + 1 < S::NK1) {
#pragma unroll
                for (int q = 0; q < AK; ++q) nxt[q] = valid ? Ta[(kc + 1) * AK + q] : zero4;
            }
            unsigned char *As = A + s * 128 * KC * 2;
#pragma unroll
            for (int c8 = 0; c8 < KC; c8 += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 ta = cur[(c8 + u) / M2];
                    const float4 t2 = tb[(c8 + u) % M2];
                    v[u] = (ta.x * t2.x + ta.y * t2.y + ta.z * t2.z + ta.w * t2.w) * inv2;
                }
                st_row8<BF>(As, tid, c8, KC, v);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (!waitv(&bar_t[s], ph_t[s])) { dead = true; break; }
            if (tid == 0) {
                tc::fence_after_sync();
                mma(tm, As, B + s * F * KC * 2, KC, idF, kc > 0);
                tc::mma_commit(&bar_m[s]);
            }
        }
        if (dead) break;
        for (int kc = (S::NK1 > 2 ? S::NK1 - 2 : 0); kc < S::NK1; ++kc)
            if (!waitv(&bar_m[kc & 1], ph_m[kc & 1])) { dead = true; break; }
        if (dead) break;
        tc::fence_after_sync();
        load_b(0, S::W2T_OFF, F * F * 2, B);
        // layer-1 epilogue: t1 = tanh(z + b1) (plain layer), kept in TMEM for layer 2
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            uint32_t w[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                v[u] = tc::tanh_fast(z[u] + b1[c0 + u]);
                w[u] = __float_as_uint(v[u]);
            }
            tc::tmem_st16(tsc + c0, w);
            st_row8<BF>(A, tid, c0, F, v);
            st_row8<BF>(A, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_full(tm, 1, false)) { dead = true; break; }
        load_b(0, S::W3T_OFF, F * F * 2, B);
        // layer-2 epilogue: y2 = t1 + t2; E gets y2 . w now (y3 = y2 + t3);
        // the derivative factors of layers 1 and 2 replace t1
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
                const float t = tc::tanh_fast(z[u] + b2[k]);
                v[u] = t1[u] + t;
                e = fmaf(v[u], wo[k], e);
                __half2 h = __floats2half2_rn(1.f - t1[u] * t1[u], 1.f - t * t);
                w[u] = *reinterpret_cast<uint32_t *>(&h);
            }
            tc::tmem_st16(tsc + c0, w);
            st_row8<BF>(A, tid, c0, F, v);
            st_row8<BF>(A, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_full(tm, 1, false)) { dead = true; break; }
        load_b(0, S::W3B_OFF, F * F * 2, B);
        // layer-3 epilogue: E_i = (y2 + t3) . w + b (FP32), dz3 = w (1 - t3^2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], v[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = c0 + u;
                const float t = tc::tanh_fast(z[u] + b3[k]);
                e = fmaf(t, wo[k], e);
                v[u] = wo[k] * (1.f - t * t);
            }
            st_row8<BF>(A, tid, c0, F, v);
            st_row8<BF>(A, tid, c0 + 8, F, v + 8);
        }
        if (valid) E_atom[atom] = (double)(e + bout);
        if (!gemm_full(tm, 1, false)) { dead = true; break; }
        load_b(0, S::W2B_OFF, F * F * 2, B);
        // dY2 epilogue: dy2 = dz3 W3^T + w (skip of layer 3), dz2 = dy2 (1 - t2^2);
        // dy2 goes back into the accumulator, so that the next MMA adds dz2 W2^T
        // to it (the skip of layer 2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], pk[16], v[16];
            uint32_t w[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld16(tsc + c0, pk);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const float dy2 = z[u] + wo[c0 + u];
                uint32_t bits = __float_as_uint(pk[u]);
                const float2 g = __half22float2(*reinterpret_cast<__half2 *>(&bits));
                v[u] = dy2 * g.y;
                w[u] = __float_as_uint(dy2);
            }
            tc::tmem_st16(trow + c0, w);
            st_row8<BF>(A, tid, c0, F, v);
            st_row8<BF>(A, tid, c0 + 8, F, v + 8);
        }
        tc::tmem_st_wait();
        if (!gemm_full(tm, 1, true)) { dead = true; break; }
        load_b(0, S::W1B_OFF, S::NC * F * 2, B);
        // dY1 epilogue: dy1 = dy2 + dz2 W2^T (from the accumulator), dz1 = dy1 (1 - t1^2)
#pragma unroll 1
        for (int c0 = 0; c0 < F; c0 += 16) {
            float z[16], pk[16], v[16];
            tc::tmem_ld16(trow + c0, z);
            tc::tmem_ld16(tsc + c0, pk);
            tc::tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                uint32_t bits = __float_as_uint(pk[u]);
                const float2 g = __half22float2(*reinterpret_cast<__half2 *>(&bits));
                v[u] = z[u] * g.x;
            }
            st_row8<BF>(A, tid, c0, F, v);
            st_row8<BF>(A, tid, c0 + 8, F, v + 8);
        }
        // dE/dD = dz1 W1^T in N chunks, folded into dE/dT
        float4 dtb[M2];
#pragma unroll
        for (int b = 0; b < M2; ++b) dtb[b] = zero4;
        float4 *dTa = reinterpret_cast<float4 *>(dT + (int64_t)atom * 4 * M1);
        for (int j = 0; j < S::NB1 && !dead; ++j) {
            const uint32_t reg = (uint32_t)(j & 1) * 256;
            if (!gemm_full(tm + reg, 0, false)) { dead = true; break; }
            if (j + 1 < S::NB1) load_b(0, S::W1B_OFF + (uint32_t)(j + 1) * S::NC * F * 2, S::NC * F * 2, B);
            // column block [c0 + h, c0 + h + HS) of this chunk is row a = a0 + (c0 + h) / M2 of T;
            // the next block's row is loaded ahead of its use
            constexpr int HS = M2 < 16 ? M2 : 16;
            const int a0 = (j * S::NC) / M2;
            float4 tan = valid ? Ta[a0] : zero4;
#pragma unroll
            for (int c0 = 0; c0 < S::NC; c0 += 16) {
                float z[16];
                tc::tmem_ld16(trow + reg + c0, z);
                tc::tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 16; h += HS) {
                    const int a = a0 + (c0 + h) / M2;
                    const float4 ta = tan;
                    if ((c0 + h) / M2 + 1 < S::NC / M2) tan = valid ? Ta[a + 1] : zero4;
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
                    // an M2-wide block of columns completes the first term of dE/dT for row a
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
    if (dead && tid == 0) atomicOr(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}


template <class S>
void pack_net(const double *p, const NetLayout &L, int bf16, unsigned char *out)
{
    memset(out, 0, S::IMG);
    auto put = [&](uint32_t base, int r, int k, int K, float v) {
        uint16_t h;
        if (bf16) {
            __nv_bfloat16 b = __float2bfloat16_rn(v);
            memcpy(&h, &b, 2);
        } else {
            __half b = __float2half_rn(v);
            memcpy(&h, &b, 2);
        }
        memcpy(out + base + tc::kmaj_off(r, k, K), &h, 2);
    };
    const double *W1 = p + L.W[0], *b1 = p + L.b[0];
    const double *W2 = p + L.W[1], *b2 = p + L.b[1];
    const double *W3 = p + L.W[2], *b3 = p + L.b[2];
    for (int a = 0; a < S::E0; ++a)
        for (int o = 0; o < S::E1; ++o) {
            float w = (float)W2[a * S::E1 + o];
            put(S::B2_OFF, o, a, S::K2, w);      // W2^T: row = output o, K = input a
            put(S::B2B_OFF, a, o, S::N2, w);     // W2:   row = input a,  K = output o
        }
    for (int a = 0; a < S::E1; ++a)
        for (int o = 0; o < S::E2; ++o) {
            float w = (float)W3[a * S::E2 + o];
            put(S::B3_OFF, o, a, S::N2, w);
            put(S::B3B_OFF, a, o, S::N3, w);
        }
    float *vec = reinterpret_cast<float *>(out + S::VEC_OFF);
    for (int k = 0; k < S::E0; ++k) {
        vec[k] = (float)W1[k];
        vec[S::K2 + k] = (float)b1[k];
    }
    for (int k = 0; k < S::E1; ++k) vec[2 * S::K2 + k] = (float)b2[k];
    for (int k = 0; k < S::E2; ++k) vec[2 * S::K2 + S::N2 + k] = (float)b3[k];
}

template <class S>
dp_status pack_all(dp_model *m)
{
    const ModelDev &md = m->dev;
    const int nn = m->ntypes * m->ntypes;
    std::vector<unsigned char> img((size_t)2 * nn * S::IMG);
    for (int bf = 0; bf < 2; ++bf)
        for (int q = 0; q < nn; ++q)
            pack_net<S>(m->h_params.data() + md.emb_base + q * md.emb.size, md.emb, bf,
                        img.data() + ((size_t)bf * nn + q) * S::IMG);
    if (!m->d_tcw) DP_CUDA(cudaMalloc((void **)&m->d_tcw, img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_tcw, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    m->tc_img_bytes = S::IMG;
    return DP_OK;
}


template <class FS>
void pack_fit_net(const double *p, const NetLayout &L, int bf16, unsigned char *out)
{
    memset(out, 0, FS::IMG);
    auto put = [&](uint32_t base, int r, int k, int K, float v) {
        uint16_t h;
        if (bf16) {
            __nv_bfloat16 b = __float2bfloat16_rn(v);
            memcpy(&h, &b, 2);
        } else {
            __half b = __float2half_rn(v);
            memcpy(&h, &b, 2);
        }
        memcpy(out + base + tc::kmaj_off(r, k, K), &h, 2);
    };
    constexpr int F = FS::F, KC = FS::KC, NC = FS::NC;
    const double *W1 = p + L.W[0], *W2 = p + L.W[1], *W3 = p + L.W[2];
    for (int d = 0; d < FS::D; ++d)
        for (int o = 0; o < F; ++o) {
            const float w = (float)W1[(int64_t)d * F + o];
            put(FS::W1T_OFF + (uint32_t)(d / KC) * F * KC * 2, o, d % KC, KC, w);   // B[n = o][k = d]
            put(FS::W1B_OFF + (uint32_t)(d / NC) * NC * F * 2, d % NC, o, F, w);    // B[n = d][k = o]
        }
    for (int k = 0; k < F; ++k)
        for (int o = 0; o < F; ++o) {
            const float w2 = (float)W2[k * F + o], w3 = (float)W3[k * F + o];
            put(FS::W2T_OFF, o, k, F, w2);
            put(FS::W3T_OFF, o, k, F, w3);
            put(FS::W2B_OFF, k, o, F, w2);
            put(FS::W3B_OFF, k, o, F, w3);
        }
    float *vec = reinterpret_cast<float *>(out + FS::VEC_OFF);
    for (int k = 0; k < F; ++k) {
        vec[k] = (float)p[L.b[0] + k];
        vec[F + k] = (float)p[L.b[1] + k];
        vec[2 * F + k] = (float)p[L.b[2] + k];
        vec[3 * F + k] = (float)p[L.W[3] + k];
    }
    vec[4 * F] = (float)p[L.b[3]];
}

template <class FS>
dp_status pack_fit_all(dp_model *m)
{
    const ModelDev &md = m->dev;
    std::vector<unsigned char> img((size_t)2 * md.ntypes * FS::IMG);
    for (int bf = 0; bf < 2; ++bf)
        for (int t = 0; t < md.ntypes; ++t)
            pack_fit_net<FS>(m->h_params.data() + md.fit_base + t * md.fit.size, md.fit, bf,
                             img.data() + ((size_t)bf * md.ntypes + t) * FS::IMG);
    if (!m->d_tcfit) DP_CUDA(cudaMalloc((void **)&m->d_tcfit, img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_tcfit, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return DP_OK;
}

using FitWater = FitShape<100, 16, 240>;
using FitStudent = FitShape<32, 8, 64>;
using FitPaper = FitShape<128, 16, 240>;
// descriptors of the wide embedding nets (M1 = 4w, wide.cu)
using FitW256 = FitShape<256, 16, 240>;
using FitW512 = FitShape<512, 16, 240>;
using FitW1024 = FitShape<1024, 16, 240>;
using FitW2048 = FitShape<2048, 16, 240>;

// The fused tensor-core fitting kernel covers three equal hidden widths F
// after a plain first layer (the configs' 240-240-240 and 64-64-64).
int fit_tc_kind(const ModelDev &md)
{
    if (md.n_fit != 3 || md.fit.wout[0] != md.fit.wout[1] || md.fit.wout[1] != md.fit.wout[2]) return 0;
    const int F = md.fit.wout[0];
    if (md.m1 == 100 && md.m2 == 16 && F == 240) return 1;
    if (md.m1 == 32 && md.m2 == 8 && F == 64) return 2;
    if (md.m1 == 128 && md.m2 == 16 && F == 240) return 3;
    if (md.m2 == 16 && F == 240) {
        if (md.m1 == 256) return 4;
        if (md.m1 == 512) return 5;
        if (md.m1 == 1024) return 6;
        if (md.m1 == 2048) return 7;
    }
    return 0;
}

template <class FS, int BF>
dp_status launch_fit_tc(dp_model *m, dp_nlist *nl, const float *T, int grid, double *E_atom, float *dT,
                        cudaStream_t st)
{
    const ModelDev &md = m->dev;
    DP_CUDA(cudaFuncSetAttribute(k_fit_tc<FS, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS::SMEM));
    for (int t = 0; t < md.ntypes; ++t) {
        const int64_t b = nl->type_off[t], cnt = nl->type_count[t];
        if (cnt <= 0) continue;
        const int64_t tiles = (cnt + 127) / 128;
        const unsigned g = (unsigned)(tiles < grid ? tiles : grid);
        const unsigned char *img = m->d_tcfit + ((size_t)BF * md.ntypes + t) * FS::IMG;
        ProfScope ps(m->prof, PG_FIT, 1, st);
        k_fit_tc<FS, BF><<<g, 128, FS::SMEM, st>>>(md, nl->d_order, b, cnt, T, img, E_atom, dT, m->d_err);
        DP_CUDA(cudaGetLastError());
    }
    return DP_OK;
}

template <int BF>
dp_status fit_tc(dp_model *m, dp_nlist *nl, const float *T, int grid, double *E_atom, float *dT,
                 cudaStream_t st)
{
    if (fit_cluster_enabled()) {
        const dp_status s = fit_cluster(m, nl, BF, T, E_atom, dT, st);
        if (s != DP_ERR_UNSUPPORTED) return s;
    }
    switch (fit_tc_kind(m->dev)) {
    case 1: return launch_fit_tc<FitWater, BF>(m, nl, T, grid, E_atom, dT, st);
    case 2: return launch_fit_tc<FitStudent, BF>(m, nl, T, grid, E_atom, dT, st);
    case 3: return launch_fit_tc<FitPaper, BF>(m, nl, T, grid, E_atom, dT, st);
    default: break;
    }
    if constexpr (BF == 1) {   // the wide nets' descriptors (bf16 only)
        switch (fit_tc_kind(m->dev)) {
        case 4: return launch_fit_tc<FitW256, 1>(m, nl, T, grid, E_atom, dT, st);
        case 5: return launch_fit_tc<FitW512, 1>(m, nl, T, grid, E_atom, dT, st);
        case 6: return launch_fit_tc<FitW1024, 1>(m, nl, T, grid, E_atom, dT, st);
        case 7: return launch_fit_tc<FitW2048, 1>(m, nl, T, grid, E_atom, dT, st);
        default: break;
        }
    }
    set_error("no tensor-core fitting kernel for this shape");
    return DP_ERR_UNSUPPORTED;
}

template <class S, int BF>
dp_status run_tc(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                 double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int64_t n = nl->n;
    const int nn = md.ntypes * md.ntypes;
    const int64_t max_chunks = n * md.chunks_per_atom + 4 * nn + 4;
    // workspace: T, dT [n][4 M1] f32; D, dD [n][desc] f32; chunks; counters; type tables
    size_t need = 0;
    auto sz = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    sz(sizeof(float) * 4 * md.m1 * n);
    sz(sizeof(float) * 4 * md.m1 * n);
    sz(sizeof(float) * md.desc_dim * n);
    sz(sizeof(float) * md.desc_dim * n);
    sz(sizeof(int4) * max_chunks);
    sz(sizeof(int) * 4);
    sz(sizeof(unsigned) * 4);   // max |dE/dT| (fp16 gradient scaling)
    const int nb = (int)((n + kCbThreads - 1) / kCbThreads);
    sz(sizeof(int) * (size_t)md.ntypes * n);             // chunk-count scans
    sz(sizeof(int) * (size_t)2 * md.ntypes * nb);        // block sums and offsets
    sz(sizeof(int) * 2 * kMaxTypes * kMaxTypes);          // group placement
    sz(sizeof(int64_t) * 2 * kMaxTypes);
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    const bool tcfit = fit_tc_kind(md) != 0 && getenv("DP_SIMT_FIT") == nullptr;
    const int fgrid = nsm;
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
    unsigned *dT_max = (unsigned *)carve(sizeof(unsigned) * 4);
    int *cb_loc = (int *)carve(sizeof(int) * (size_t)md.ntypes * n);
    int *cb_bsum = (int *)carve(sizeof(int) * (size_t)2 * md.ntypes * nb);
    int *cb_boff = cb_bsum + (size_t)md.ntypes * nb;
    int *cb_gtab = (int *)carve(sizeof(int) * 2 * kMaxTypes * kMaxTypes);
    TypeTab tt = {};
    for (int t = 0; t < md.ntypes; ++t) {
        tt.off[t] = nl->type_off[t];
        tt.cnt[t] = nl->type_count[t];
    }
    DP_CUDA(cudaMemsetAsync(T, 0, sizeof(float) * 4 * md.m1 * n, st));
    DP_CUDA(cudaMemsetAsync(d_force, 0, sizeof(double) * 3 * n, st));
    DP_CUDA(cudaMemsetAsync(d_atom_virial, 0, sizeof(double) * 9 * n, st));
    const unsigned char *wimg = m->d_tcw + (size_t)BF * nn * S::IMG;
    if (!nl->d_env) {
        set_error("tensor-core path needs the neighbor geometry of the formatting kernel");
        return DP_ERR_ARG;
    }
    const float4 *envA = reinterpret_cast<const float4 *>(nl->d_env);
    const float2 *envB = reinterpret_cast<const float2 *>(nl->d_env + 4 * (size_t)n * md.nsel);
    {
        ProfScope ps(m->prof, PG_CHUNKS, 3, st);
        k_cb_count<<<nb, kCbThreads, 0, st>>>(md, n, nl->d_order, nl->d_nnei, cb_loc, cb_bsum, nb);
        k_cb_plan<<<1, kCbThreads, 0, st>>>(md, n, tt, cb_loc, cb_bsum, cb_boff, nb, cb_gtab,
                                            chunks, cnt);
        k_cb_write<<<nb, kCbThreads, 0, st>>>(md, n, nl->d_order, nl->d_type, nl->d_nnei, cb_loc, cb_boff, nb,
                                              cb_gtab, chunks, nullptr);
    }
    DP_CUDA(cudaGetLastError());
    DP_CUDA(cudaFuncSetAttribute(k_embed_fwd_tc<S, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::F_SMEM));
    DP_CUDA(cudaFuncSetAttribute(k_embed_fwd_tc<S, BF>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    DP_CUDA(cudaFuncSetAttribute(k_embed_bwd_tc<S, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::B_SMEM));
    DP_CUDA(cudaFuncSetAttribute(k_embed_bwd_tc<S, BF>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    {
        ProfScope ps(m->prof, PG_EMBED_FWD, 1, st);
        k_embed_fwd_tc<S, BF><<<(unsigned)(S::F_CTAS * nsm), kTcThreads, S::F_SMEM, st>>>(md, envA, nl->d_nlist, nl->d_nnei, chunks,
                                                                     cnt, wimg, T, m->d_err);
    }
    DP_CUDA(cudaGetLastError());
    const int64_t nd = (int64_t)md.desc_dim * n, nq = (int64_t)4 * md.m1 * n;
    if (tcfit) {
        DP_TRY(fit_tc<BF>(m, nl, T, fgrid, d_atom_energy, dT, st));
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
    if (BF == 0) {   // the scale of dE/dT for the fp16 backward operands
        ProfScope ps(m->prof, PG_DESC, 1, st);
        DP_CUDA(cudaMemsetAsync(dT_max, 0, sizeof(unsigned), st));
        k_absmax_bits<<<(unsigned)(2 * nsm), 256, 0, st>>>(nq, dT, dT_max);
        DP_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(m->prof, PG_EMBED_BWD, 1, st);
        k_embed_bwd_tc<S, BF><<<(unsigned)(S::B_CTAS * nsm), kTcThreads, S::B_SMEM, st>>>(md, envA, envB, nl->d_nlist, nl->d_nnei, chunks,
                                                                     cnt, wimg, dT, d_force, d_atom_virial, m->d_err,
                                                                     BF == 0 ? dT_max : nullptr);
    }
    DP_CUDA(cudaGetLastError());
    ProfScope ps(m->prof, PG_REDUCE, 1, st);
    return reduce_energy_virial(d_atom_energy, d_atom_virial, centers_of(nl), d_energy, d_virial, m->d_red, st);
}

}  // namespace

DP_BOUNDS_ACCESSOR(bounds_read_tc)

// Scratch of build_chunks_batch for nb positions.
size_t chunks_batch_scratch(const ModelDev &md, int64_t nb)
{
    const int64_t blocks = (nb + kCbThreads - 1) / kCbThreads;
    return 256 * 4 + sizeof(int) * (size_t)md.ntypes * nb + sizeof(int) * (size_t)2 * md.ntypes * blocks +
           sizeof(int) * 2 * kMaxTypes * kMaxTypes + sizeof(int64_t) * 2 * kMaxTypes;
}

// Work list of the 32-neighbor chunks of positions [p0, p0 + nb) of the
// type-sorted order, grouped by net and padded to tiles of 4 chunks of one
// net: entry {atom, batch position, first slot, net} (atom -1: padding),
// firstc[q * ntypes + tj] = first chunk of (p0 + q, tj), *ntiles on the
// device.  At most nb * chunks_per_atom + 3 ntypes^2 entries.
dp_status build_chunks_batch(dp_model *m, dp_nlist *nl, int64_t p0, int64_t nb, int4 *chunks, int *firstc,
                             int *ntiles, char *scratch, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const int blocks = (int)((nb + kCbThreads - 1) / kCbThreads);
    auto carve = [&](size_t bytes) {
        char *p = scratch;
        scratch += (bytes + 255) & ~(size_t)255;
        return p;
    };
    int *loc = (int *)carve(sizeof(int) * (size_t)md.ntypes * nb);
    int *bsum = (int *)carve(sizeof(int) * (size_t)2 * md.ntypes * blocks);
    int *boff = bsum + (size_t)md.ntypes * blocks;
    int *gtab = (int *)carve(sizeof(int) * 2 * kMaxTypes * kMaxTypes);
    TypeTab tt = {};
    for (int t = 0; t < md.ntypes; ++t) {
        int64_t b = nl->type_off[t] - p0, e = nl->type_off[t] + nl->type_count[t] - p0;
        b = b < 0 ? 0 : (b > nb ? nb : b);
        e = e < 0 ? 0 : (e > nb ? nb : e);
        tt.off[t] = b;
        tt.cnt[t] = e - b;
    }
    const int32_t *order = nl->d_order + p0;
    k_cb_count<<<blocks, kCbThreads, 0, st>>>(md, nb, order, nl->d_nnei, loc, bsum, blocks);
    k_cb_plan<<<1, kCbThreads, 0, st>>>(md, nb, tt, loc, bsum, boff, blocks, gtab, chunks,
                                        ntiles);
    k_cb_write<<<blocks, kCbThreads, 0, st>>>(md, nb, order, nl->d_type, nl->d_nnei, loc, boff, blocks, gtab, chunks,
                                              firstc);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

dp_status pack_tc_weights(dp_model *m)
{
    const int *e = m->dev.emb.wout;
    DP_TRY(pack_fit_cluster_weights(m));
    if (embed_is_wide(m->n_embed, m->embed)) {
        if (m->d_wide) DP_TRY(pack_wide_weights(m));
    } else {
        if (m->d_tcw_x3) DP_TRY(pack_x3_weights(m));
        if (e[0] == 25) DP_TRY(pack_all<TcWater>(m));
        else if (e[0] == 8) DP_TRY(pack_all<TcStudent>(m));
        else DP_TRY(pack_all<TcPaper>(m));
    }
    switch (fit_tc_kind(m->dev)) {
    case 1: return pack_fit_all<FitWater>(m);
    case 2: return pack_fit_all<FitStudent>(m);
    case 3: return pack_fit_all<FitPaper>(m);
    case 4: return pack_fit_all<FitW256>(m);
    case 5: return pack_fit_all<FitW512>(m);
    case 6: return pack_fit_all<FitW1024>(m);
    case 7: return pack_fit_all<FitW2048>(m);
    default: return DP_OK;
    }
}

dp_status fit_mix16_bf16(dp_model *m, dp_nlist *nl, const float *T, double *E_atom, float *dT, cudaStream_t st)
{
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    return fit_tc<1>(m, nl, T, nsm, E_atom, dT, st);
}

dp_status compute_mix16(dp_model *m, dp_nlist *nl, int bf16, double *d_energy, double *d_atom_energy,
                        double *d_force, double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    const int *e = m->dev.emb.wout;
    if (e[0] == 25)
        return bf16 ? run_tc<TcWater, 1>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st)
                    : run_tc<TcWater, 0>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
    if (e[0] == 8)
        return bf16 ? run_tc<TcStudent, 1>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st)
                    : run_tc<TcStudent, 0>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
    return bf16 ? run_tc<TcPaper, 1>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st)
                : run_tc<TcPaper, 0>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
}

}  // namespace dp

// Fitting net on the tensor cores with one 128-atom tile split over a thread-block cluster.
//
// The computation is that of the fused fitting kernels of tc.cu (MIX-16 of Sec. 4.1.3: fp16 or bf16
// operands, FP32 accumulators) and tc_x3.cu (split bf16: every product as hi*hi + hi*lo + lo*hi):
// the descriptor D = T T<^T (Sec. 2.2) built straight into the A operand, the three hidden layers of
// width F with their skips, E_i = y3 . w + b in FP32, and the adjoint dE_i/dT_i through dz3, dz2,
// dz1 and dE/dD.  What changes is who does which part of a tile: its 128 atom rows are shared by the
// NS CTAs of a cluster, and
//  - CTA r owns the output columns [r F/NS, (r+1) F/NS) of the three layers and of the two backward
//    F x F products, and the 64-column blocks r, r + NS, r + 2 NS, ... of dE/dD;
//  - every CTA builds the whole D tile (the K dimension of layer 1) itself, chunk by chunk, in a ring
//    of shared-memory stages that the tensor core drains behind it;
//  - after each epilogue every CTA writes its columns of the next A operand (t1, y2, dz3, dz2, dz1;
//    hi and lo planes in split mode) into the shared memory of all CTAs of the cluster, between two
//    cluster barriers: the products that read the old A are complete everywhere before the first,
//    and all columns of the new A are in place after the second;
//  - one thread per CTA streams that CTA's slices of the weights through a ring of bulk copies that
//    runs ahead of the tensor core across layers and tiles (the weights do not depend on the data);
//  - E_i and the term of dE/dT that rows a < M2 of T receive through T< are summed over the cluster
//    at the end of the tile, from partial sums each CTA leaves in its own shared memory, in a fixed
//    order.
// Persistent clusters walk the tiles of one center type.  With clusters of 3, the 32 tiles of 4,000
// atoms keep 96 SMs busy where the single-CTA kernels kept 32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "dp_internal.cuh"
#include "tc_common.cuh"
#include "tc_embed.cuh"

namespace dp {

namespace {

constexpr unsigned long long kWaitNs = 1000000000ull;   // a wait of the cluster kernel gives up after 1 s

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of all CTAs of the cluster; memory operations before it (shared, distributed shared
// and global) are visible to every thread of the cluster after it.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address in the shared memory of CTA `rank` of the cluster of the same variable as local `saddr`.
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cl_st16(uint32_t addr, uint4 v)
{
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ float4 cl_ld16(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ float cl_ld4(uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// d (+)= A B^T over KS steps of K = 16 (K-major no-swizzle operands): the descriptors of the first step
// advance by 256 bytes (16 in their address field, which cannot carry below 256 KB) per step.
template <int KS>
__device__ __forceinline__ void mma_steps(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc0)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(id), "r"(acc0));
#pragma unroll
    for (int ks = 1; ks < KS; ++ks)
        asm volatile(
            "{\n .reg .pred p;\n setp.eq.u32 p, 0, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(ad + 16u * ks), "l"(bd + 16u * ks), "r"(id));
}

// Tile shape: descriptor M1 x M2 (D = M1 M2 columns), hidden width F, NS CTAs per cluster, P operand
// planes (1: fp16 / bf16, 2: split bf16 hi and lo).
template <int M1_, int M2_, int F_, int NS_, int P_>
struct FitCl {
    static constexpr int M1 = M1_, M2 = M2_, F = F_, D = M1_ * M2_, NS = NS_, P = P_;
    static constexpr int FS = F / NS;                                    // output columns per CTA
    static constexpr int KC1 = P == 2 ? 32 : 64, NK1 = D / KC1;          // layer-1 K chunks
    static constexpr int KC2 = (F % 48 == 0) ? 48 : 32, NK2 = F / KC2;   // K chunks of the F-wide products
    static constexpr int NBW = 64, NBLK = D / NBW, BPR = (NBLK + NS - 1) / NS;   // dE/dD column blocks
    static constexpr uint32_t CH1 = FS * KC1 * 2 * P, CH2 = FS * KC2 * 2 * P, CHB = NBW * KC2 * 2 * P;
    // weight image of CTA rank r, in the order the chunks are consumed: layer-1 chunks of W1 (rows o
    // of the slice, K = d), W2^T and W3^T (rows o, K = k), W3 and W2 (rows k of the slice, K = o), then
    // the rank's dE/dD blocks of W1 (rows d, K = o), then b1, b2, b3, w_out (all F) and b_out (FP32)
    static constexpr uint32_t O1 = 0, O2 = O1 + NK1 * CH1, O3 = O2 + NK2 * CH2, O4 = O3 + NK2 * CH2,
                              O5 = O4 + NK2 * CH2, O6 = O5 + NK2 * CH2, O7 = O6 + BPR * NK2 * CHB;
    static constexpr uint32_t VEC_BYTES = ((4 * F + 4) * 4 + 15) / 16 * 16, IMG_R = O7 + VEC_BYTES;
    static constexpr uint32_t cmax(uint32_t a, uint32_t b) { return a > b ? a : b; }
    // shared memory: A region (the [128][F] activations, P planes; in layer 1 a ring of D chunks; at
    // the end of a tile the partial sums), the weight ring, the vectors
    static constexpr uint32_t ACT = 128 * F * 2 * P, DCH = 128 * KC1 * 2 * P, PART = 128 * M2 * 16 + 128 * 4;
    static constexpr uint32_t AREG = cmax(cmax(ACT, 2 * DCH), PART);
    static constexpr int SA = (int)(AREG / DCH) < 4 ? (int)(AREG / DCH) : 4;
    static constexpr uint32_t STAGE = cmax(cmax(CH1, CH2), CHB);
    static constexpr uint32_t B_OFF = AREG, RING = 227 * 1024 - AREG - VEC_BYTES - 1024;
    static constexpr int SB = (int)(RING / STAGE) < 8 ? (int)(RING / STAGE) : 8;
    static constexpr uint32_t V_OFF = B_OFF + SB * STAGE, SMEM = V_OFF + VEC_BYTES;
    // launched with at least 120 KB so that one CTA runs per SM: each holds 512 tensor-memory columns,
    // and a CTA waiting for columns held by a CTA of another cluster could wait on a cluster barrier
    static constexpr uint32_t SMEM_LAUNCH = cmax(SMEM, 120 * 1024);
    static_assert(F % NS == 0 && FS % 16 == 0 && FS >= 16 && FS <= 128, "column split");
    static_assert(D % KC1 == 0 && KC1 % M2 == 0 && F % KC2 == 0 && D % NBW == 0 && NBW % M2 == 0 &&
                      16 % M2 == 0 && NBLK >= NS,
                  "chunks");
    static_assert(SA >= 2 && SB >= 3 && SMEM <= 227 * 1024, "shared memory");
    static_assert(IMG_R % 16 == 0 && CH1 % 16 == 0 && CH2 % 16 == 0 && CHB % 16 == 0 && AREG % 128 == 0 &&
                      STAGE % 128 == 0,
                  "bulk copy alignment");
};

// MODE 0: fp16 operands, 1: bf16, 2: split bf16 (P = 2).
//
// Roles: warps 0-3 are the workers (thread = atom row: D chunks, epilogues, dE/dD folds); lane 0 of
// warp 4 issues the products; lane 0 of warp 5 streams the weight chunks.  All hand-overs go through
// mbarriers: inside the CTA for copies, products and D chunks, and across the cluster for the
// exchanges (the workers of every CTA arrive on the barriers of every CTA), so the copy thread runs
// ahead through layers and tiles and no thread waits for more than what it consumes.
template <class S, int MODE>
__global__ void __launch_bounds__(192, 1) k_fit_cl(ModelDev md, const int32_t *__restrict__ order, int64_t pos_begin,
                                                  int64_t count, const float *__restrict__ T,
                                                  const unsigned char *__restrict__ img_type,
                                                  double *__restrict__ E_atom, float *__restrict__ dT, int *err)
{
    static_assert((MODE == 2) == (S::P == 2), "operand planes");
    constexpr int P = S::P, F = S::F, FS = S::FS, NS = S::NS, M1 = S::M1, M2 = S::M2, KC1 = S::KC1,
                  KC2 = S::KC2, NK1 = S::NK1, NK2 = S::NK2, NBW = S::NBW, SB = S::SB, SA = S::SA;
    constexpr int BF = MODE == 0 ? 0 : 1, AK = KC1 / M2, PF = 8 / AK > 2 ? 8 / AK : 2;
    constexpr uint32_t XW = 128u * NS;   // arrivals per phase of a cluster-wide barrier
    extern __shared__ __align__(128) unsigned char smem[];
    // in the CTA: weight ring (full: copy landed; empty: its products done), D stages (dfull: written;
    // dfree: its products done), layer accumulator (acc), dE/dD accumulators (dready: products done;
    // drel: read by the workers).  Over the cluster: pfree (every CTA's products that read A are done),
    // aready (every CTA's columns of the new A are written), partr / partd (end-of-tile partial sums
    // written / read).
    __shared__ __align__(8) uint64_t bar_full[SB], bar_empty[SB], bar_dfull[SA], bar_dfree[SA], bar_acc,
        bar_dready[2], bar_drel[2], bar_pfree, bar_aready, bar_partr, bar_partd;
    __shared__ uint32_t tmem_base;
    __shared__ int s_dead;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool worker = warp < 4, mma_thread = tid == 128, copy_thread = tid == 160;
    const uint32_t rank = cl_rank();
    const unsigned char *img = img_type + (size_t)rank * S::IMG_R;
    unsigned char *A = smem, *Bst = smem + S::B_OFF;
    float *vec = reinterpret_cast<float *>(smem + S::V_OFF);
    const float *b1 = vec, *b2 = vec + F, *b3 = vec + 2 * F, *wo = vec + 3 * F;
    if (tid == 0) {
        for (int q = 0; q < SB; ++q) {
            tc::mbar_init(&bar_full[q], 1);
            tc::mbar_init(&bar_empty[q], 1);
        }
        for (int q = 0; q < SA; ++q) {
            tc::mbar_init(&bar_dfull[q], 128);
            tc::mbar_init(&bar_dfree[q], 1);
        }
        tc::mbar_init(&bar_acc, 1);
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&bar_dready[q], 1);
            tc::mbar_init(&bar_drel[q], 128);
        }
        tc::mbar_init(&bar_pfree, XW);
        tc::mbar_init(&bar_aready, XW);
        tc::mbar_init(&bar_partr, XW);
        tc::mbar_init(&bar_partd, XW);
        s_dead = 0;
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    {
        const float *gv = reinterpret_cast<const float *>(img + S::O7);
        for (int q = tid; q < 4 * F + 4; q += 192) vec[q] = gv[q];
    }
    tc::fence_before_sync();
    __syncthreads();
    cl_sync();   // every CTA of the cluster is running, its barriers initialised, before any remote access
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    // tensor memory: the layer accumulator (FS columns) at 0, t1 and then the derivative factors of
    // layers 1 and 2 at 128, two dE/dD block accumulators at 256 and 256 + NBW
    const uint32_t trow = tm + ((uint32_t)((warp & 3) * 32) << 16), tsc = trow + 128;
    const float bout = vec[4 * F];
    const float inv2 = (float)(md.inv_nsel * md.inv_nsel);
    const uint32_t idS = tc::idesc_f16(128, FS, BF), idB = tc::idesc_f16(128, NBW, BF);
    const uint32_t a_u32 = tc::smem_u32(A), b_u32 = tc::smem_u32(Bst);
    const int col0 = (int)rank * FS;
    uint32_t a_rem[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) a_rem[q] = cl_map(a_u32, (uint32_t)q);
    const int ntiles = (int)((count + 127) / 128);
    const int cid = (int)(blockIdx.x / NS), ncl = (int)(gridDim.x / NS);
    const int my_tiles = cid < ntiles ? (ntiles - 1 - cid) / ncl + 1 : 0;
    const int nb_r = (S::NBLK - (int)rank + NS - 1) / NS;   // this CTA's dE/dD blocks
    const int nch = NK1 + 4 * NK2 + nb_r * NK2;              // weight chunks per tile

    // Polls an mbarrier phase (acquire at CTA or cluster scope); gives up after about a second or as
    // soon as another thread of the CTA gave up, and then marks the CTA failed.
    auto wait = [&](uint64_t *bar, uint32_t parity, bool cluster = false) -> bool {
        const uint32_t a = tc::smem_u32(bar);
        unsigned long long t0 = 0;
        for (uint32_t it = 1;; ++it) {
            uint32_t done;
            if (cluster)
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done)
                    : "r"(a), "r"(parity)
                    : "memory");
            else
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done)
                    : "r"(a), "r"(parity)
                    : "memory");
            if (done) return true;
            if (*(volatile int *)&s_dead) return false;
            if ((it & 255u) == 0) {
                unsigned long long now;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > kWaitNs) {
                    *(volatile int *)&s_dead = 1;
                    return false;
                }
            }
        }
    };
    auto dead = [&]() { return *(volatile int *)&s_dead != 0; };
    // the same, one answer for the whole warp (all its lanes call it): guards of .sync.aligned code
    auto dead_w = [&]() { return __any_sync(0xffffffffu, dead()) != 0; };
    // one arrival (release at cluster scope) on the same barrier of every CTA of the cluster
    auto arrive_all = [&](uint64_t *bar) {
        const uint32_t a = tc::smem_u32(bar);
#pragma unroll
        for (int q = 0; q < NS; ++q)
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_map(a, (uint32_t)q))
                         : "memory");
    };
    auto tanh_ = [](float x) -> float {
        if constexpr (MODE == 2) return tanhf(x);
        else return tc::tanh_fast(x);
    };
    // the derivative factors (1 - t1^2, 1 - t2^2) of one column as one 32-bit word
    auto fac_pack = [](float a, float b) -> uint32_t {
        if constexpr (MODE == 2) {
            return unorm16_pair(a, b);
        } else {
            __half2 h = __floats2half2_rn(a, b);
            return *reinterpret_cast<uint32_t *>(&h);
        }
    };
    auto fac1 = [](uint32_t w) -> float {
        if constexpr (MODE == 2) {
            return (float)(w & 0xffffu) * (1.f / 65535.f);
        } else {
            return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
        }
    };
    auto fac2 = [](uint32_t w) -> float {
        if constexpr (MODE == 2) {
            return (float)(w >> 16) * (1.f / 65535.f);
        } else {
            return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
        }
    };
    // 8 values of K-columns k0 .. k0 + 7 of this thread's row into a K-major tile with K columns
    auto st8 = [&](unsigned char *tile, uint32_t plane, int k0, int K, const float *v) {
        if constexpr (P == 2) st8_k(tile, tile + plane, tid, k0, K, v);
        else st_row8<BF>(tile, tid, k0, K, v);
    };
    // the same into the A operand ([128][F]) of every CTA of the cluster
    auto put8 = [&](int k0, const float *v) {
        const uint32_t off = tc::kmaj_off(tid, k0, F);
        uint4 h, l;
        if constexpr (P == 2) {
            split2(v[0], v[1], h.x, l.x);
            split2(v[2], v[3], h.y, l.y);
            split2(v[4], v[5], h.z, l.z);
            split2(v[6], v[7], h.w, l.w);
        } else {
            h = make_uint4(pack2<BF>(v[0], v[1]), pack2<BF>(v[2], v[3]), pack2<BF>(v[4], v[5]), pack2<BF>(v[6], v[7]));
            l = h;
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            cl_st16(a_rem[q] + off, h);
            if constexpr (P == 2) cl_st16(a_rem[q] + 128 * F * 2 + off, l);
        }
    };

    if (copy_thread) {
        // ---- the weight chunks of every tile in consumption order, each into the next ring stage once
        // the products that read the stage's previous chunk are done
        int pos = 0, issued = 0;
        for (int g = 0, total = my_tiles * nch; g < total; ++g) {
            const int s = g % SB;
            if (g >= SB && !wait(&bar_empty[s], (uint32_t)(g / SB - 1) & 1u)) break;
            uint32_t off, bytes;
            if (pos < NK1) {
                off = S::O1 + (uint32_t)pos * S::CH1;
                bytes = S::CH1;
            } else if (pos < NK1 + 4 * NK2) {
                off = S::O2 + (uint32_t)(pos - NK1) * S::CH2;
                bytes = S::CH2;
            } else {
                off = S::O6 + (uint32_t)(pos - NK1 - 4 * NK2) * S::CHB;
                bytes = S::CHB;
            }
            tc::mbar_expect_tx(&bar_full[s], bytes);
            tc::bulk_g2s(Bst + (uint32_t)s * S::STAGE, img + off, bytes, &bar_full[s]);
            if (++pos == nch) pos = 0;
            issued = g + 1;
        }
        if (dead()) {
            // a wait gave up: the copies still in flight land (bounded wait) before the memory is released
            for (int g = issued > SB ? issued - SB : 0; g < issued; ++g)
                tc::mbar_wait(&bar_full[g % SB], (uint32_t)(g / SB) & 1u, kWaitLimit);
        }
    } else if (mma_thread) {
        // ---- all products, in the order the copies arrive
        int g = 0;             // weight chunks consumed
        uint32_t ca = 0;       // D chunks
        uint32_t x = 0;        // exchanges (aready phases)
        uint32_t cd = 0;       // dE/dD blocks
        int lc = -1;           // the last chunk whose products were committed
        // d (+)= A B^T with the next weight chunk (B_ROWS x K) as B; three products in split mode
        auto chunk = [&](auto kc, auto brows, uint32_t d, uint32_t a, uint32_t a_plane, uint32_t a_sbo, uint32_t id,
                         bool acc0) -> bool {
            constexpr int K = decltype(kc)::value, B_ROWS = decltype(brows)::value;
            const int s = g % SB;
            if (!wait(&bar_full[s], (uint32_t)(g / SB) & 1u)) return false;
            tc::fence_after_sync();
            const uint32_t b = b_u32 + (uint32_t)s * S::STAGE;
            const uint64_t ad = tc::smem_desc(a, 128, a_sbo), bd = tc::smem_desc(b, 128, (K / 8) * 128);
            mma_steps<K / 16>(d, ad, bd, id, acc0 ? 1u : 0u);
            if constexpr (P == 2) {
                mma_steps<K / 16>(d, ad, bd + (uint64_t)((B_ROWS * K * 2) >> 4), id, 1u);
                mma_steps<K / 16>(d, ad + (uint64_t)(a_plane >> 4), bd, id, 1u);
            }
            tc::mma_commit(&bar_empty[s]);
            lc = g++;
            return true;
        };
        using KC1_t = std::integral_constant<int, KC1>;
        using KC2_t = std::integral_constant<int, KC2>;
        using FS_t = std::integral_constant<int, FS>;
        using NBW_t = std::integral_constant<int, NBW>;
        // acc (+)= A (K = F, the columns of all CTAs) x the next NK2 weight chunks, once A is complete
        auto gemm_res = [&](bool acc0) -> bool {
            if (!wait(&bar_aready, x++ & 1u, true)) return false;
            tc::fence_async_smem();
            tc::fence_after_sync();
            for (int c = 0; c < NK2; ++c)
                if (!chunk(KC2_t{}, FS_t{}, tm, a_u32 + (uint32_t)c * (KC2 / 8) * 128, 128 * F * 2, (F / 8) * 128, idS,
                           acc0 || c > 0))
                    return false;
            tc::mma_commit(&bar_acc);
            return true;
        };
        for (int it = 0; it < my_tiles && !dead(); ++it) {
            bool ok = true;
            for (int c = 0; c < NK1 && ok; ++c, ++ca) {
                const int sa = (int)(ca % SA);
                ok = wait(&bar_dfull[sa], (ca / SA) & 1u);
                if (!ok) break;
                tc::fence_after_sync();
                ok = chunk(KC1_t{}, FS_t{}, tm, a_u32 + (uint32_t)sa * S::DCH, 128 * KC1 * 2, (KC1 / 8) * 128, idS, c > 0);
                if (!ok) break;
                tc::mma_commit(&bar_dfree[sa]);
            }
            if (!ok) break;
            tc::mma_commit(&bar_acc);
            if (!gemm_res(false) || !gemm_res(false) || !gemm_res(false) || !gemm_res(true)) break;
            if (!wait(&bar_aready, x++ & 1u, true)) break;   // dz1 complete
            tc::fence_async_smem();
            for (int i = 0; i < nb_r && ok; ++i, ++cd) {
                const uint32_t buf = cd & 1u;
                if (cd >= 2 && !wait(&bar_drel[buf], ((cd >> 1) - 1) & 1u)) ok = false;
                if (!ok) break;
                tc::fence_after_sync();
                for (int c = 0; c < NK2 && ok; ++c)
                    ok = chunk(KC2_t{}, NBW_t{}, tm + 256 + buf * NBW, a_u32 + (uint32_t)c * (KC2 / 8) * 128, 128 * F * 2,
                               (F / 8) * 128, idB, c > 0);
                if (ok) tc::mma_commit(&bar_dready[buf]);
            }
            if (!ok) break;
        }
        if (dead() && lc >= 0) {
            // a wait gave up: wait (bounded) for the products in flight before the memory is released
            atomicOr(err, 1);
            tc::mbar_wait(&bar_empty[lc % SB], (uint32_t)(lc / SB) & 1u, kWaitLimit);
        }
    } else if (worker) {
        uint32_t ca = 0, nacc = 0, x = 0, cd = 0;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        // every worker: my CTA's products that read A are done (after an accumulator wait) -> tell every
        // CTA; then wait until every CTA has said so, before writing into their A operands
        auto exchange_begin = [&]() {
            tc::fence_before_sync();
            arrive_all(&bar_pfree);
            wait(&bar_pfree, x & 1u, true);
            tc::fence_after_sync();
        };
        // my columns of the new A operand are in every CTA (and my tensor-memory accesses are done)
        auto exchange_end = [&]() {
            tc::fence_before_sync();
            arrive_all(&bar_aready);
            ++x;
        };
        auto acc_wait = [&]() {
            if (!dead()) wait(&bar_acc, nacc & 1u);
            ++nacc;
            tc::fence_after_sync();
        };
        for (int it = 0; it < my_tiles; ++it) {
            const int64_t r0 = (int64_t)(cid + it * ncl) * 128 + tid;
            const bool valid = r0 < count;
            const int atom = valid ? order[pos_begin + r0] : 0;
            const float4 *Ta = reinterpret_cast<const float4 *>(T + (int64_t)atom * 4 * M1);
            float4 tb[M2];   // rows b < M2 of T (the T< factor) times 1/sum(sel)^2
#pragma unroll
            for (int b = 0; b < M2; ++b) {
                const float4 t = valid ? Ta[b] : zero4;
                tb[b] = make_float4(t.x * inv2, t.y * inv2, t.z * inv2, t.w * inv2);
            }
            // the peers have read this CTA's partial sums of the previous tile (in the A region)
            if (it > 0 && !dead()) wait(&bar_partd, (uint32_t)(it - 1) & 1u, true);
            // ---- layer 1: D (times 1/sum(sel)^2) into a ring of SA stages, T rows PF chunks ahead
            {
                float4 ring[PF][AK];
#pragma unroll
                for (int j = 0; j < PF; ++j)
#pragma unroll
                    for (int q = 0; q < AK; ++q) ring[j][q] = (valid && j < NK1) ? Ta[j * AK + q] : zero4;
                for (int c0 = 0; c0 < NK1; c0 += PF) {
#pragma unroll
                    for (int j = 0; j < PF; ++j) {
                        const int c = c0 + j;
                        if (c >= NK1) break;
                        const int sa = (int)(ca % SA);
                        if (ca >= (uint32_t)SA && !dead()) wait(&bar_dfree[sa], ((ca / SA) - 1) & 1u);
                        ++ca;
                        float4 cur[AK];
#pragma unroll
                        for (int q = 0; q < AK; ++q) cur[q] = ring[j][q];
                        if (c + PF < NK1) {
#pragma unroll
                            for (int q = 0; q < AK; ++q) ring[j][q] = valid ? Ta[(c + PF) * AK + q] : zero4;
                        }
                        unsigned char *Ds = A + (uint32_t)sa * S::DCH;
#pragma unroll
                        for (int c8 = 0; c8 < KC1; c8 += 8) {
                            float v[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const float4 ta = cur[(c8 + u) / M2];
                                const float4 t2 = tb[(c8 + u) % M2];
                                v[u] = ta.x * t2.x + ta.y * t2.y + ta.z * t2.z + ta.w * t2.w;
                            }
                            st8(Ds, 128 * KC1 * 2, c8, KC1, v);
                        }
                        tc::fence_async_smem();
                        tc::mbar_arrive(&bar_dfull[sa]);
                    }
                }
            }
            acc_wait();
            exchange_begin();
            // layer-1 epilogue: t1 = tanh(z1 + b1) (plain layer), kept in tensor memory for layer 2
            if (!dead_w()) {
#pragma unroll 1
                for (int c0 = 0; c0 < FS; c0 += 16) {
                    float z[16], v[16];
                    uint32_t w[16];
                    tc::tmem_ld16(trow + c0, z);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        v[u] = tanh_(z[u] + b1[col0 + c0 + u]);
                        w[u] = __float_as_uint(v[u]);
                    }
                    tc::tmem_st16(tsc + c0, w);
                    put8(col0 + c0, v);
                    put8(col0 + c0 + 8, v + 8);
                }
                tc::tmem_st_wait();
            }
            exchange_end();
            acc_wait();
            exchange_begin();
            // layer-2 epilogue: y2 = t1 + t2; E gets y2 . w now (y3 = y2 + t3); the derivative factors of
            // layers 1 and 2 replace t1
            float e = 0.f;
            if (!dead_w()) {
#pragma unroll 1
                for (int c0 = 0; c0 < FS; c0 += 16) {
                    float z[16], t1[16], v[16];
                    uint32_t w[16];
                    tc::tmem_ld16(trow + c0, z);
                    tc::tmem_ld16(tsc + c0, t1);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int k = col0 + c0 + u;
                        const float t = tanh_(z[u] + b2[k]);
                        v[u] = t1[u] + t;
                        e = fmaf(v[u], wo[k], e);
                        w[u] = fac_pack(1.f - t1[u] * t1[u], 1.f - t * t);
                    }
                    tc::tmem_st16(tsc + c0, w);
                    put8(col0 + c0, v);
                    put8(col0 + c0 + 8, v + 8);
                }
                tc::tmem_st_wait();
            }
            exchange_end();
            acc_wait();
            exchange_begin();
            // layer-3 epilogue: E_i gets t3 . w (with y2 . w above, E_i = y3 . w + b), dz3 = w (1 - t3^2)
            if (!dead_w()) {
#pragma unroll 1
                for (int c0 = 0; c0 < FS; c0 += 16) {
                    float z[16], v[16];
                    tc::tmem_ld16(trow + c0, z);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int k = col0 + c0 + u;
                        const float t = tanh_(z[u] + b3[k]);
                        e = fmaf(t, wo[k], e);
                        v[u] = wo[k] * (1.f - t * t);
                    }
                    put8(col0 + c0, v);
                    put8(col0 + c0 + 8, v + 8);
                }
            }
            exchange_end();
            acc_wait();
            exchange_begin();
            // dE/dy2 epilogue: dy2 = dz3 W3^T + w (skip of layer 3), dz2 = dy2 (1 - t2^2); dy2 goes back
            // into the accumulator, so that the next product adds dz2 W2^T to it (the skip of layer 2)
            if (!dead_w()) {
#pragma unroll 1
                for (int c0 = 0; c0 < FS; c0 += 16) {
                    float z[16], v[16];
                    uint32_t w[16], pk[16];
                    tc::tmem_ld16(trow + c0, z);
                    tc::tmem_ld16(tsc + c0, reinterpret_cast<float *>(pk));
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const float dy2 = z[u] + wo[col0 + c0 + u];
                        v[u] = dy2 * fac2(pk[u]);
                        w[u] = __float_as_uint(dy2);
                    }
                    tc::tmem_st16(trow + c0, w);
                    put8(col0 + c0, v);
                    put8(col0 + c0 + 8, v + 8);
                }
                tc::tmem_st_wait();
            }
            exchange_end();
            acc_wait();
            exchange_begin();
            // dE/dy1 epilogue: dy1 = dy2 + dz2 W2^T (from the accumulator), dz1 = dy1 (1 - t1^2)
            if (!dead_w()) {
#pragma unroll 1
                for (int c0 = 0; c0 < FS; c0 += 16) {
                    float z[16], v[16];
                    uint32_t pk[16];
                    tc::tmem_ld16(trow + c0, z);
                    tc::tmem_ld16(tsc + c0, reinterpret_cast<float *>(pk));
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) v[u] = z[u] * fac1(pk[u]);
                    put8(col0 + c0, v);
                    put8(col0 + c0 + 8, v + 8);
                }
            }
            exchange_end();
            // ---- dE/dD = dz1 W1^T over this CTA's column blocks, each folded into dE/dT once read:
            // dE/dT[a] = sum_b dD[a][b] T[b] (all rows a), and sum_a dD[a][b] T[a] for rows b < M2
            float4 dtb[M2];
#pragma unroll
            for (int b = 0; b < M2; ++b) dtb[b] = zero4;
            float4 *dTa = reinterpret_cast<float4 *>(dT + (int64_t)atom * 4 * M1);
            {
                constexpr int RB = NBW / M2, HS = M2 < 16 ? M2 : 16;
                for (int i = 0; i < nb_r; ++i, ++cd) {
                    const uint32_t buf = cd & 1u;
                    const int a0 = ((int)rank + i * NS) * RB;
                    float4 trow_b[RB];   // the block's rows a of T, loaded while its products run
#pragma unroll
                    for (int q = 0; q < RB; ++q) trow_b[q] = valid ? Ta[a0 + q] : zero4;
                    const bool ok = !dead_w() && wait(&bar_dready[buf], (cd >> 1) & 1u);
                    tc::fence_after_sync();
                    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
                        for (int c0 = 0; c0 < NBW; c0 += 16) {
                            float z[16];
                            tc::tmem_ld16(trow + 256 + buf * NBW + c0, z);
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int h = 0; h < 16; h += HS) {
                                const int a = a0 + (c0 + h) / M2;
                                const float4 ta = trow_b[(c0 + h) / M2];
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
                                if (valid) dTa[a] = acc;
                            }
                        }
                    }
                    tc::fence_before_sync();
                    tc::mbar_arrive(&bar_drel[buf]);
                }
            }
            // ---- cluster sums: this CTA's partial sums into its A region (all its products are done),
            // then E_i by rank 0 and the T< term of rows b < M2 by the owner of the block holding row
            // a = b, each adding the NS partial sums in rank order
            {
                float4 *part = reinterpret_cast<float4 *>(A);
#pragma unroll
                for (int b = 0; b < M2; ++b) part[tid * M2 + b] = dtb[b];
                reinterpret_cast<float *>(A + 128 * M2 * 16)[tid] = e;
            }
            // this thread's own rows b < M2 of dE/dT (written above), read while the partial sums gather
            float4 own[M2];
#pragma unroll
            for (int b = 0; b < M2; ++b)
                own[b] = (valid && ((b * M2) / NBW) % NS == (int)rank) ? dTa[b] : zero4;
            arrive_all(&bar_partr);
            if (!dead()) wait(&bar_partr, (uint32_t)it & 1u, true);
            if (valid && !dead()) {
                if (rank == 0) {
                    float s = 0.f;
#pragma unroll
                    for (int q = 0; q < NS; ++q) s += cl_ld4(a_rem[q] + 128 * M2 * 16 + tid * 4);
                    E_atom[atom] = (double)(s + bout);
                }
#pragma unroll
                for (int b = 0; b < M2; ++b) {
                    if (((b * M2) / NBW) % NS != (int)rank) continue;
                    float4 s = zero4;
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        const float4 p = cl_ld16(a_rem[q] + (uint32_t)(tid * M2 + b) * 16);
                        s.x += p.x;
                        s.y += p.y;
                        s.z += p.z;
                        s.w += p.w;
                    }
                    dTa[b] = make_float4(own[b].x + s.x * inv2, own[b].y + s.y * inv2, own[b].z + s.z * inv2,
                                         own[b].w + s.w * inv2);
                }
            }
            arrive_all(&bar_partd);
        }
        // the peers have read the last tile's partial sums
        if (my_tiles > 0 && !dead()) wait(&bar_partd, (uint32_t)(my_tiles - 1) & 1u, true);
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && dead()) atomicOr(err, 1);
    cl_sync();   // no CTA leaves while another may still access its shared memory
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// ---------------------------------------------------------------------------------------------
// Host side: per-rank weight images and the cluster launch.

using ClWater16 = FitCl<100, 16, 240, 3, 1>;
using ClStudent16 = FitCl<32, 8, 64, 2, 1>;
using ClPaper16 = FitCl<128, 16, 240, 3, 1>;
using ClW256 = FitCl<256, 16, 240, 3, 1>;
using ClW512 = FitCl<512, 16, 240, 3, 1>;
using ClW1024 = FitCl<1024, 16, 240, 3, 1>;
using ClW2048 = FitCl<2048, 16, 240, 3, 1>;
using ClWaterX3 = FitCl<100, 16, 240, 3, 2>;
using ClStudentX3 = FitCl<32, 8, 64, 2, 2>;
using ClPaperX3 = FitCl<128, 16, 240, 3, 2>;

// Element w at (row, k) of a K-major chunk [rows][K] (planes of rows * K * 2 bytes): fp16, bf16 (the
// value rounded to FP32 first, as the single-CTA kernels' images), or hi and lo of split bf16.
template <int MODE>
void put_w(unsigned char *chunk, int rows, int r, int k, int K, double w)
{
    const uint32_t off = tc::kmaj_off(r, k, K);
    if (MODE == 2) {
        const __nv_bfloat16 h = __double2bfloat16(w);
        const __nv_bfloat16 l = __double2bfloat16(w - (double)__bfloat162float(h));
        memcpy(chunk + off, &h, 2);
        memcpy(chunk + (size_t)rows * K * 2 + off, &l, 2);
    } else if (MODE == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)w);
        memcpy(chunk + off, &h, 2);
    } else {
        const __half h = __float2half_rn((float)w);
        memcpy(chunk + off, &h, 2);
    }
}

template <class S, int MODE>
void pack_cl(const double *p, const NetLayout &L, unsigned char *out)
{
    constexpr int F = S::F, FS = S::FS, KC1 = S::KC1, KC2 = S::KC2, NBW = S::NBW, NS = S::NS;
    memset(out, 0, (size_t)NS * S::IMG_R);
    const double *W1 = p + L.W[0], *W2 = p + L.W[1], *W3 = p + L.W[2];
    for (int r = 0; r < NS; ++r) {
        unsigned char *img = out + (size_t)r * S::IMG_R;
        for (int d = 0; d < S::D; ++d)
            for (int ol = 0; ol < FS; ++ol)   // z1 = D W1: B[o][d] = W1[d][o]
                put_w<MODE>(img + S::O1 + (uint32_t)(d / KC1) * S::CH1, FS, ol, d % KC1, KC1,
                            W1[(int64_t)d * F + r * FS + ol]);
        for (int k = 0; k < F; ++k)
            for (int ol = 0; ol < FS; ++ol) {   // z2 = y1 W2, z3 = y2 W3: B[o][k] = W[k][o]
                const int o = r * FS + ol;
                put_w<MODE>(img + S::O2 + (uint32_t)(k / KC2) * S::CH2, FS, ol, k % KC2, KC2, W2[k * F + o]);
                put_w<MODE>(img + S::O3 + (uint32_t)(k / KC2) * S::CH2, FS, ol, k % KC2, KC2, W3[k * F + o]);
            }
        for (int kl = 0; kl < FS; ++kl)
            for (int o = 0; o < F; ++o) {   // dy2 = dz3 W3^T, dy1 += dz2 W2^T: B[k][o] = W[k][o]
                const int k = r * FS + kl;
                put_w<MODE>(img + S::O4 + (uint32_t)(o / KC2) * S::CH2, FS, kl, o % KC2, KC2, W3[k * F + o]);
                put_w<MODE>(img + S::O5 + (uint32_t)(o / KC2) * S::CH2, FS, kl, o % KC2, KC2, W2[k * F + o]);
            }
        for (int i = 0; r + i * NS < S::NBLK; ++i)
            for (int dl = 0; dl < NBW; ++dl)
                for (int o = 0; o < F; ++o) {   // dE/dD = dz1 W1^T: B[d][o] = W1[d][o]
                    const int64_t d = (int64_t)(r + i * NS) * NBW + dl;
                    put_w<MODE>(img + S::O6 + (uint32_t)(i * S::NK2 + o / KC2) * S::CHB, NBW, dl, o % KC2, KC2,
                                W1[d * F + o]);
                }
        float *vec = reinterpret_cast<float *>(img + S::O7);
        for (int k = 0; k < F; ++k) {
            vec[k] = (float)p[L.b[0] + k];
            vec[F + k] = (float)p[L.b[1] + k];
            vec[2 * F + k] = (float)p[L.b[2] + k];
            vec[3 * F + k] = (float)p[L.W[3] + k];
        }
        vec[4 * F] = (float)p[L.b[3]];
    }
}

template <class S, int MODE>
dp_status pack_cl_all(dp_model *m)
{
    const ModelDev &md = m->dev;
    const size_t per = (size_t)S::NS * S::IMG_R;
    std::vector<unsigned char> img(per * md.ntypes);
    for (int t = 0; t < md.ntypes; ++t)
        pack_cl<S, MODE>(m->h_params.data() + md.fit_base + t * md.fit.size, md.fit, img.data() + per * t);
    if (!m->d_fitcl[MODE]) DP_CUDA(cudaMalloc((void **)&m->d_fitcl[MODE], img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_fitcl[MODE], img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return DP_OK;
}

template <class S, int MODE>
dp_status launch_cl(dp_model *m, dp_nlist *nl, const float *T, double *E_atom, float *dT, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    auto kern = k_fit_cl<S, MODE>;
    DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM_LAUNCH));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S::NS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM_LAUNCH;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters = 0;   // clusters resident at once on this GPU (one CTA per SM)
    if (max_clusters == 0) {
        cfg.gridDim = dim3(S::NS * 256, 1, 1);
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, kern, &cfg) != cudaSuccess || c < 1) {
            (void)cudaGetLastError();
            int nsm = 0;
            DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
            c = nsm / S::NS > 0 ? nsm / S::NS : 1;
        }
        max_clusters = c;
    }
    // Clusters pay for their exchanges with more SM time per tile than one CTA spends; they win only
    // while there are SMs the one-CTA kernel leaves idle, i.e. at most one tile per cluster.
    for (int t = 0; t < md.ntypes; ++t)
        if ((nl->type_count[t] + 127) / 128 > max_clusters) return DP_ERR_UNSUPPORTED;
    if (!m->d_fitcl[MODE]) DP_TRY((pack_cl_all<S, MODE>(m)));
    const size_t per = (size_t)S::NS * S::IMG_R;
    for (int t = 0; t < md.ntypes; ++t) {
        const int64_t b = nl->type_off[t], cnt = nl->type_count[t];
        if (cnt <= 0) continue;
        const int64_t tiles = (cnt + 127) / 128;
        const int64_t ncl = tiles < max_clusters ? tiles : max_clusters;
        cfg.gridDim = dim3((unsigned)(ncl * S::NS), 1, 1);
        const unsigned char *img = m->d_fitcl[MODE] + per * t;
        ProfScope ps(m->prof, PG_FIT, 1, st);
        DP_CUDA(cudaLaunchKernelEx(&cfg, kern, md, (const int32_t *)nl->d_order, b, cnt, T, img, E_atom, dT,
                                   m->d_err));
    }
    return DP_OK;
}

template <int MODE>
dp_status run_cl(dp_model *m, dp_nlist *nl, const float *T, double *E_atom, float *dT, cudaStream_t st, bool pack)
{
    const ModelDev &md = m->dev;
    if (md.n_fit != 3 || md.fit.wout[0] != md.fit.wout[1] || md.fit.wout[1] != md.fit.wout[2])
        return DP_ERR_UNSUPPORTED;
    const int F = md.fit.wout[0], m1 = md.m1, m2 = md.m2;
#define DP_CL_CASE(SHAPE)                                                                     \
    return pack ? pack_cl_all<SHAPE, MODE>(m) : launch_cl<SHAPE, MODE>(m, nl, T, E_atom, dT, st)
    if constexpr (MODE == 2) {
        if (m1 == 100 && m2 == 16 && F == 240) DP_CL_CASE(ClWaterX3);
        if (m1 == 32 && m2 == 8 && F == 64) DP_CL_CASE(ClStudentX3);
        if (m1 == 128 && m2 == 16 && F == 240) DP_CL_CASE(ClPaperX3);
    } else {
        if (m1 == 100 && m2 == 16 && F == 240) DP_CL_CASE(ClWater16);
        if (m1 == 32 && m2 == 8 && F == 64) DP_CL_CASE(ClStudent16);
        if (m1 == 128 && m2 == 16 && F == 240) DP_CL_CASE(ClPaper16);
        if constexpr (MODE == 1) {   // the wide embedding nets' descriptors (bf16 only)
            if (m2 == 16 && F == 240) {
                if (m1 == 256) DP_CL_CASE(ClW256);
                if (m1 == 512) DP_CL_CASE(ClW512);
                if (m1 == 1024) DP_CL_CASE(ClW1024);
                if (m1 == 2048) DP_CL_CASE(ClW2048);
            }
        }
    }
#undef DP_CL_CASE
    return DP_ERR_UNSUPPORTED;
}

}  // namespace

bool fit_cluster_enabled() { return getenv("DP_FIT_ONE_CTA") == nullptr; }

dp_status fit_cluster(dp_model *m, dp_nlist *nl, int mode, const float *T, double *E_atom, float *dT,
                      cudaStream_t st)
{
    switch (mode) {
    case 0: return run_cl<0>(m, nl, T, E_atom, dT, st, false);
    case 1: return run_cl<1>(m, nl, T, E_atom, dT, st, false);
    case 2: return run_cl<2>(m, nl, T, E_atom, dT, st, false);
    default: return DP_ERR_UNSUPPORTED;
    }
}

dp_status pack_fit_cluster_weights(dp_model *m)
{
    for (int mode = 0; mode < 3; ++mode) {
        if (!m->d_fitcl[mode]) continue;
        dp_status s = mode == 0   ? run_cl<0>(m, nullptr, nullptr, nullptr, nullptr, nullptr, true)
                      : mode == 1 ? run_cl<1>(m, nullptr, nullptr, nullptr, nullptr, nullptr, true)
                                  : run_cl<2>(m, nullptr, nullptr, nullptr, nullptr, nullptr, true);
        if (s != DP_OK) return s;
    }
    return DP_OK;
}

}  // namespace dp

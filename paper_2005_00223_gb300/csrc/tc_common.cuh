// Blackwell (sm_103a) tensor-core building blocks: tcgen05 MMA with operands in
// shared memory, accumulators in tensor memory (TMEM), bulk copies on the TMA
// engine, and mbarrier waits that give up after a bounded number of polls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dp {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: the operand is a grid of
// 8 x 16-byte core matrices.  K-major: lbo = byte stride between core
// matrices along K, sbo = byte stride between 8-row groups along M (or N).
// MN-major (with the transpose bit of the instruction descriptor): lbo =
// stride between groups of 8 K-rows, sbo = stride between groups of 8
// M (or N) elements.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the 5th-generation tensor core
    return d;                        // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both fp16
// (bf16 = 0) or both bf16 (bf16 = 1), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int bf16)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with fp16 A and B, both MN-major
// (transposed: bits 15 and 16), FP32 accumulator, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16_mn(int M, int N)
{
    return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with each operand K-major (0) or
// MN-major (1, the transpose bits 15 and 16), FP32 accumulator, fp16 (bf16
// = 0) or bf16 (bf16 = 1) operands, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16_major(int M, int N, int bf16, int a_mn, int b_mn)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (mn, k) of an MN-major no-swizzle tile with MN rows:
// core matrices of 8 K-rows x 16 bytes (8 consecutive MN elements); groups of
// 8 MN elements 128 bytes apart (the descriptor's sbo), groups of 8 K-rows
// MN/8 * 128 bytes apart (its lbo).
__host__ __device__ __forceinline__ uint32_t mnmaj_off(int mn, int k, int MN)
{
    return (uint32_t)((mn & 7) * 2 + (mn >> 3) * 128 + (k & 7) * 16 + (k >> 3) * (MN >> 3) * 128);
}

// Byte offset of element (r, k) of a K-major no-swizzle tile with K columns
// (lbo = 128, sbo = K/8 * 128).
__host__ __device__ __forceinline__ uint32_t kmaj_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// D[tmem] = A[smem] * B[smem]^T over K (multiple of 16), M = 128, or D += A B^T
// with accumulate; one thread issues.
__device__ __forceinline__ void mma_kloop(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, uint32_t idesc,
                                          bool accumulate = false)
{
    const uint32_t sbo = (uint32_t)(K >> 3) * 128;
    for (int ks = 0; ks < (K >> 4); ++ks) {
        uint64_t ad = smem_desc(a_saddr + ks * 256, 128, sbo);
        uint64_t bd = smem_desc(b_saddr + ks * 256, 128, sbo);
        uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

// D[tmem] (+)= A B^T with both operands MN-major (mnmaj_off layouts with
// MN extents MA and NB), K a multiple of 16 starting at K-row k0; M = 128.
__device__ __forceinline__ void mma_kloop_mn(uint32_t d_tmem, uint32_t a_saddr, int MA, uint32_t b_saddr, int NB,
                                             int k0, int K, uint32_t idesc, bool accumulate)
{
    const uint32_t lbo_a = (uint32_t)(MA >> 3) * 128, lbo_b = (uint32_t)(NB >> 3) * 128;
    for (int ks = 0; ks < (K >> 4); ++ks) {
        const int kg = (k0 >> 3) + 2 * ks;
        uint64_t ad = smem_desc(a_saddr + kg * lbo_a, lbo_a, 128);
        uint64_t bd = smem_desc(b_saddr + kg * lbo_b, lbo_b, 128);
        uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

// D[tmem] (+)= A B^T with A K-major ([128][K], kmaj_off layout) and B
// MN-major with MN extent NB (mnmaj_off layout), K a multiple of 16; M = 128.
// A K-major tile [R][C] (kmaj_off with K = C) is, byte for byte, the
// MN-major tile of its transpose (mnmaj_off with MN = C), so a weight tile
// stored for x W^T serves as B of the transposed product as well.
__device__ __forceinline__ void mma_kloop_bmn(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int NB, int K,
                                              uint32_t idesc, bool accumulate)
{
    const uint32_t sbo_a = (uint32_t)(K >> 3) * 128, lbo_b = (uint32_t)(NB >> 3) * 128;
    for (int ks = 0; ks < (K >> 4); ++ks) {
        uint64_t ad = smem_desc(a_saddr + ks * 256, 128, sbo_a);
        uint64_t bd = smem_desc(b_saddr + 2 * ks * lbo_b, lbo_b, 128);
        uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

// One arrival (release semantics at CTA scope) on a shared-memory mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Polls the mbarrier phase with the given parity at most `limit` times;
// returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long limit)
{
    uint32_t done = 0;
    for (long it = 0; it < limit; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

// Bulk copy global -> shared on the TMA engine, completing `bytes` on mbar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp w
// reads lanes 32w..32w+31; taddr carries the warp's base lane in bits 31:16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *out)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

// Stores 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 8 consecutive 32-bit columns of this thread's TMEM lane (raw bits).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *out)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace tc
}  // namespace dp

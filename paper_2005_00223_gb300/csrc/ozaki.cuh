// FP64 products on the tensor cores by error-free splitting into fp16
// digits (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)): the
// digit layout, the pipelined MMA kernel shared by the plain product
// (ozaki.cu) and the fused embedding kernels (oz_embed.cu), and the exact
// read-back of its accumulators.
//
// A row x of length K becomes a scale 2^e and S digit planes of BETA bits:
//   x_k = 2^e sum_{i=1..S} d_i(k) 2^(-BETA i),  d_i in [-2^(BETA-1), 2^(BETA-1)),
// with e = ilogb(max_k |x_k|) + 3, so that |x_k| < 2^(e-2) and the S balanced
// digits (covering about [-0.51, 0.49] 2^(BETA S) of the scaled value) keep
// one bit of headroom; the largest entry keeps BETA S - 3 bits and the row
// is rounded once, to 2^-52 of its maximum for BETA S >= 55.  Digits are
// small integers, exact in fp16; a product of two has at most 2 BETA - 2
// bits, and the (at most S) pairs (i, j) of one diagonal g = i + j, which
// share the weight 2^(-BETA g), are summed into one FP32 accumulator in
// tensor memory, exactly as long as S K 2^(2 BETA - 2) <= 2^24.  Pairs with
// i + j > S + 1 are dropped (weight below 2^(-BETA (S+2)) of the leading
// term).  The read-back combines the exact integer accumulators in two
// int64 sums and scales them with one FP64 rounding.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tc_common.cuh"

namespace dp {
namespace oz {

constexpr long kWait = 1L << 25;   // mbarrier polls (~1 s) before a kernel gives up

// Half offset of digit i (0-based) of element (r, k) in the tiled layout:
// tiles of TR rows, K chunks of KC columns (K_pad columns in all), the S
// digit planes of one (tile, chunk) one after the other, each a K-major
// core-matrix tile (tc::kmaj_off), so that one bulk copy stages a chunk.
__host__ __device__ inline int64_t tiled(int64_t r, int k, int i, int S, int TR, int KC, int K_pad)
{
    const int64_t t = r / TR;
    const int rr = (int)(r - t * TR), c = k / KC, kk = k - c * KC;
    return (((t * (K_pad / KC) + c) * S + i) * (int64_t)TR * KC) + tc::kmaj_off(rr, kk, KC) / 2;
}

// Row scale e of a row whose largest magnitude is mx (0 for a zero row).
__device__ __forceinline__ int row_exp(double mx) { return mx > 0.0 ? ilogb(mx) + 3 : 0; }

// 2^e as a double, built from its bits with integer instructions only (subnormal for
// -1074 <= e < -1022, 0 below, infinity above 1023): no FP64-pipe work.
__device__ __forceinline__ double pow2i(int e)
{
    long long bits;
    if (e > 1023) bits = 0x7ffLL << 52;
    else if (e >= -1022) bits = (long long)(e + 1023) << 52;
    else if (e >= -1074) bits = 1LL << (e + 1074);
    else bits = 0;
    return __longlong_as_double(bits);
}

// The S balanced digits of x for row scale e, most significant first.  The
// scaled significand m = round(x 2^(BETA S - e)) (ties away from zero) is
// formed from the bits of x with integer instructions: x = mant 2^(ex - 1075)
// and |x| < 2^(e-2) give a shift of at most BETA S - 55 bits to the left.
template <int S, int BETA>
__device__ __forceinline__ void digits(double x, int e, int (&d)[S])
{
    constexpr long long H = 1LL << (BETA - 1), MASK = (1LL << BETA) - 1;
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = (unsigned long long)bits & ((1ULL << 52) - 1);
    if (ex) mant |= 1ULL << 52;
    const int sh = (ex ? ex : 1) - 1075 + BETA * S - e;
    long long m;
    if (sh >= 0) m = (long long)(mant << sh);
    else if (sh > -64) m = (long long)((mant + (1ULL << (-sh - 1))) >> (-sh));
    else m = 0;
    if (bits < 0) m = -m;                           // |m| <= 2^(BETA S - 2)
#pragma unroll
    for (int i = S - 1; i >= 0; --i) {
        const long long v = ((m + H) & MASK) - H;
        m = (m - v) >> BETA;                           // exact: m - v is a multiple of 2^BETA
        d[i] = (int)v;
    }
}

// max(m, |v|) for m >= 0 by an integer comparison of the bit patterns (monotone for non-negative doubles).
__device__ __forceinline__ double amax(double m, double v)
{
    const unsigned long long a = (unsigned long long)__double_as_longlong(m);
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
    return __longlong_as_double((long long)(a > b ? a : b));
}

// Packs 8 digits (small integers) as 8 fp16 values.
__device__ __forceinline__ uint4 pack8(const int *v)
{
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __half2 h = __halves2half2(__int2half_rn(v[2 * q]), __int2half_rn(v[2 * q + 1]));
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Shared memory and tensor memory of a work unit of 128 rows of A x NC rows
// of B: NST stages, each the S digit planes of A (128 x KC) followed by
// those of B (NC x KC); the B planes stacked form one K-major tile of S NC
// rows.  Tensor memory: one FP32 accumulator of NC columns per diagonal
// g = 2 .. S+1 at column (g - 2) NC, so the products of A plane i with B
// planes 1 .. S+1-i land on contiguous columns from (i - 1) NC: one MMA
// (split at 256 columns) per A plane and K step.  EPI bytes of shared memory
// after the stages belong to the epilogue; at most MAXST stages.
template <int S_, int BETA_, int NC_, int KC_, int EPI_ = 0, int MAXST_ = 8>
struct Shape {
    static constexpr int S = S_, BETA = BETA_, NC = NC_, KC = KC_, EPI = EPI_;
    static constexpr uint32_t A_PLANE = 128 * KC * 2, B_PLANE = NC * KC * 2;
    static constexpr uint32_t A_BYTES = S * A_PLANE, B_BYTES = S * B_PLANE;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr int NST0 = (int)((220u * 1024u - (uint32_t)EPI) / STAGE);
    static constexpr int NST = NST0 < MAXST_ ? NST0 : MAXST_;   // fewer stages leave more L1 to the epilogue
    static constexpr uint32_t SMEM = NST * STAGE + EPI;
    static constexpr uint32_t SBO = (KC / 8) * 128;   // 8-row groups of a K-major tile
    // diagonals 2 .. GH+1 are combined in one int64 (shifts <= 27 bits), the rest in another
    static constexpr int GH = (27 / BETA + 1) < S ? (27 / BETA + 1) : S;
    static_assert(KC % 16 == 0 && NC % 16 == 0 && NC >= 16, "MMA shape");
    static_assert(S * NC <= 512, "one accumulator per diagonal in tensor memory");
    static_assert(NST >= 2, "shared memory");
    static_assert((S - GH - 1) * BETA <= 27, "two groups of diagonals");
    static_assert(EPI % 1024 == 0, "epilogue shared memory alignment");
};

__device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}" : "=r"(pred));
    return pred != 0;
}

// All 32 lanes of the calling warp poll; the outcome is made warp-uniform.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, int64_t use, int nst)
{
    const bool ok = tc::mbar_wait(bar, (uint32_t)((use / nst) & 1), kWait);
    return __all_sync(0xffffffffu, ok);
}

// Exact read-back of 16 columns (c0 .. c0+15 of a unit) of the accumulators
// of the calling thread's row: H = sum_{g <= GH+1} acc_g 2^(BETA (GH+1-g)),
// L = sum_{g > GH+1} acc_g 2^(BETA (S+1-g)).  The value is
// 2^E (H 2^(-BETA (GH+1)) + L 2^(-BETA (S+1))) for E = e_A + e_B (value()).
template <class Sh>
__device__ __forceinline__ void acc_load16(uint32_t trow, int c0, long long (&H)[16], long long (&L)[16])
{
#pragma unroll
    for (int c = 0; c < 16; ++c) H[c] = L[c] = 0;
#pragma unroll
    for (int g = 2; g <= Sh::S + 1; ++g) {
        float v[16];
        tc::tmem_ld16(trow + (uint32_t)((g - 2) * Sh::NC + c0), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const long long iv = (long long)__float2int_rn(v[c]);   // |acc| < 2^24: an exact integer
            if (g <= Sh::GH + 1)
                H[c] += iv << (Sh::BETA * (Sh::GH + 1 - g));
            else
                L[c] += iv << (Sh::BETA * (Sh::S + 1 - g));
        }
    }
}

// The accumulator bits as an integer: F2I in general; with SMALL (every
// |acc| < 2^22, i.e. S K 2^(2 BETA - 2) <= 2^22) by adding 1.5 2^23, which
// puts the integer in the low mantissa bits (an FP32 add instead of a
// conversion).
template <bool SMALL>
__device__ __forceinline__ long long acc_int(uint32_t bits)
{
    if (SMALL) return (long long)(__float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000);
    return (long long)__float2int_rn(__uint_as_float(bits));
}

// The same for 8 columns, the loads of all diagonals issued before one wait.
template <class Sh, bool SMALL = false>
__device__ __forceinline__ void acc_load8(uint32_t trow, int c0, long long (&H)[8], long long (&L)[8])
{
    uint32_t v[Sh::S][8];
#pragma unroll
    for (int g = 2; g <= Sh::S + 1; ++g) tc::tmem_ld8(trow + (uint32_t)((g - 2) * Sh::NC + c0), v[g - 2]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < 8; ++c) H[c] = L[c] = 0;
#pragma unroll
    for (int g = 2; g <= Sh::S + 1; ++g)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const long long iv = acc_int<SMALL>(v[g - 2][c]);
            if (g <= Sh::GH + 1)
                H[c] += iv << (Sh::BETA * (Sh::GH + 1 - g));
            else
                L[c] += iv << (Sh::BETA * (Sh::S + 1 - g));
        }
}

static __device__ __noinline__ double i2d_scaled_slow(long long v, int a) { return scalbn((double)v, a); }

// v 2^a as a double, exactly, for |v| < 2^53, built with integer instructions
// only (the FP64 pipe is the scarce unit); results outside the normal range
// take a library path.
__device__ __forceinline__ double i2d_scaled(long long v, int a)
{
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ULL << 63) : 0ULL;
    const unsigned long long u = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    const int be = 63 - lz + a + 1023;                       // biased exponent of u 2^a
    if (be <= 0 || be >= 2047) return i2d_scaled_slow(v, a);
    const unsigned long long mant = ((u << lz) << 1) >> 12;  // the 52 bits after the leading one
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | mant));
}

// The read-back value: H 2^(E - BETA (GH+1)) + L 2^(E - BETA (S+1)); both
// terms are exact doubles, so the one FP64 add is the only rounding (as for
// a fused multiply-add of the two).
template <class Sh>
__device__ __forceinline__ double acc_value(long long H, long long L, int E)
{
    return i2d_scaled(H, E - Sh::BETA * (Sh::GH + 1)) + i2d_scaled(L, E - Sh::BETA * (Sh::S + 1));
}

// C-unit pipeline.  Units u = tile * nn + nchunk (tile of 128 rows of A,
// chunk of NC rows of B) are spread over persistent CTAs; A digits of tile t
// and K chunk kc start at dA + ((t nk + kc) S) 128 KC, those of B at
// epi.b_unit(t, nchunk) + kc S NC KC.  Warp 0 (uniform control flow, one
// elected lane per instruction) streams the K chunks through a ring of NST
// stages with bulk copies and issues the MMAs; then all NT threads (4 or 8
// warps) run epi(tile, nchunk, trow, tid, esmem), trow = the tensor-memory
// address of the row quarter of the thread's warp (warp w reads lanes
// 32 (w % 4) ..; the thread's row is 32 (w % 4) + lane).  The first 16
// bytes of the epilogue's shared memory start zeroed.  The tile count is read from ntiles_dev
// when given (a device-built work list), else M_pad / 128.  Every wait is
// bounded; on expiry the kernel flags *err, stops and frees tensor memory.
template <class Sh, class Epi, int NT = 128>
__global__ void __launch_bounds__(NT, 1) k_gemm(int64_t M_pad, const int *ntiles_dev, int N, int K,
                                               const __half *__restrict__ dA, Epi epi, int *err)
{
    constexpr int S = Sh::S, NC = Sh::NC, KC = Sh::KC, NST = Sh::NST;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_t[NST], bar_m[NST];
    __shared__ uint32_t tmem_base;
    __shared__ int s_dead;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *esmem = smem + NST * Sh::STAGE;
    if (Sh::EPI >= 16 && tid < 4) reinterpret_cast<int *>(esmem)[tid] = 0;   // the epilogue's first 16 bytes start zeroed
    if (tid == 0) {
        s_dead = 0;
        for (int q = 0; q < NST; ++q) {
            tc::mbar_init(&bar_t[q], 1);
            tc::mbar_init(&bar_m[q], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    const uint32_t trow = tm + ((uint32_t)((warp & 3) * 32) << 16);
    const int nk = K / KC, nn = N / NC;
    const int64_t ntiles = ntiles_dev ? (int64_t)*ntiles_dev : M_pad / 128;
    const int64_t units = ntiles * nn;
    // the chunks of this CTA in order: unit blockIdx.x + q gridDim.x, K chunk kc -> c = q nk + kc,
    // staged in stage c % NST
    const int64_t my_units = units > blockIdx.x ? (units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int64_t total = my_units * nk;
    const uint32_t sbase = tc::smem_u32(smem);
    int64_t issued = 0, mma_done = 0;   // chunks copied; chunks whose MMAs were waited for
    bool ok = true;
    auto copy_chunk = [&](int64_t c) {
        const int s = (int)(c % NST);
        for (; ok && mma_done <= c - NST; ++mma_done)   // stage s is free once chunk c - NST's MMAs are done
            ok = warp_wait(&bar_m[mma_done % NST], mma_done, NST);
        if (!ok) return;
        const int64_t u = blockIdx.x + (c / nk) * gridDim.x, tile = u / nn;
        const int kc = (int)(c % nk), nchunk = (int)(u % nn);
        if (elect_one()) {
            unsigned char *st = smem + s * Sh::STAGE;
            tc::mbar_expect_tx(&bar_t[s], Sh::STAGE);
            tc::bulk_g2s(st, dA + ((tile * nk + kc) * S) * (int64_t)(128 * KC), Sh::A_BYTES, &bar_t[s]);
            tc::bulk_g2s(st + Sh::A_BYTES, epi.b_unit(tile, nchunk) + (int64_t)kc * S * NC * KC, Sh::B_BYTES,
                         &bar_t[s]);
        }
        __syncwarp();
    };
    if (warp == 0)
        for (; ok && issued < NST - 1 && issued < total; ++issued) copy_chunk(issued);
    for (int64_t q = 0; q < my_units; ++q) {
        const int64_t u = blockIdx.x + q * gridDim.x, tile = u / nn;
        const int nchunk = (int)(u % nn);
        if (warp == 0) {
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int64_t c = q * nk + kc;
                const int s = (int)(c % NST);
                ok = warp_wait(&bar_t[s], c, NST);
                if (!ok) break;
                tc::fence_after_sync();
                const uint32_t a0 = sbase + s * Sh::STAGE, b0 = a0 + Sh::A_BYTES;
                if (elect_one()) {
#pragma unroll
                    for (int i = 1; i <= S; ++i) {
#pragma unroll
                        for (int p = 0; p < ((S + 1 - i) * NC + 255) / 256; ++p) {
                            const int rows = (S + 1 - i) * NC - 256 * p;
                            const uint32_t idesc = tc::idesc_f16(128, rows < 256 ? rows : 256, 0);
                            const uint32_t d = tm + (uint32_t)((i - 1) * NC + 256 * p);
#pragma unroll
                            for (int ks = 0; ks < KC / 16; ++ks) {
                                const uint64_t ad =
                                    tc::smem_desc(a0 + (uint32_t)((i - 1) * Sh::A_PLANE + 256 * ks), 128, Sh::SBO);
                                const uint64_t bd =
                                    tc::smem_desc(b0 + (uint32_t)(32 * p * Sh::SBO + 256 * ks), 128, Sh::SBO);
                                // the first MMAs of a unit (plane 1 covers every diagonal) overwrite
                                const uint32_t accum = (kc > 0 || i > 1 || ks > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                            }
                        }
                    }
                    tc::mma_commit(&bar_m[s]);
                }
                __syncwarp();
                if (issued < total) copy_chunk(issued++);   // NST - 1 chunks ahead, possibly of the next unit
            }
            // every MMA of this unit done before the accumulators are read
            for (; ok && mma_done < (q + 1) * nk; ++mma_done) ok = warp_wait(&bar_m[mma_done % NST], mma_done, NST);
            if (!ok && elect_one()) s_dead = 1;
            __syncwarp();
        }
        tc::fence_before_sync();
        __syncthreads();
        if (s_dead) break;
        tc::fence_after_sync();
        epi(tile, nchunk, trow, tid, esmem);
        tc::fence_before_sync();
        __syncthreads();
    }
    if (s_dead && tid == 0) atomicOr(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

}  // namespace oz
}  // namespace dp

// FP64 matrix products on the 5th-generation tensor cores by error-free
// splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)).
//
// C = A B^T with A [M][K] and B [N][K] in FP64.  Every row of A and every
// row of B is written as a power-of-two scale times S signed digits of BETA
// bits:  x_k = 2^e sum_{i=1..S} d_i(k) 2^(-BETA i),  d_i in [-2^(BETA-1), 2^(BETA-1)),
// with |x_k| < 2^(e-2) (S balanced digits represent about
// [-0.51, 0.49] 2^(BETA S) of the scaled value, so one bit of headroom is
// kept) and the largest entry of the row carried to BETA S - 3 >= 51 bits,
// its last bits rounded, an error of at most 2^-52 of the row's maximum.  A
// digit is an integer of at most 2^(BETA-1) in magnitude, hence an exact
// fp16 value; a product of two digits has at most 2 BETA - 2 bits.  Pairs
// (i, j) with i + j = g share the weight 2^(-BETA g); the (at most S) pairs
// of one diagonal g are summed into one FP32 accumulator in tensor memory
// by kind::f16 MMAs, exact as long as S K 2^(2 BETA - 2) <= 2^24.  Pairs
// with i + j > S + 1 are dropped (their weight is below 2^(-BETA (S+2)) of
// the leading term).  The epilogue combines the accumulators, exact
// integers, in two int64 sums and scales them by 2^(e_A + e_B) with one
// FP64 rounding.  The error is that of a dot product of the digit-truncated
// rows, of the order of K 2^(-BETA S) |a|_max |b|_max per entry, the size
// of FP64 rounding.
//
// Kernels: k_oz_split writes the digits of the rows of an FP64 matrix (one
// warp per row), pre-tiled in the shared-memory layout of the MMAs;
// k_oz_gemm computes C for work units (128 rows of A) x (NC rows of B): one
// warp streams the K chunks of both digit sets through a ring of
// shared-memory stages with bulk copies on the TMA engine and issues the
// MMAs (one per A digit plane and K step, against the stacked B planes),
// then all four warps combine the accumulators.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "dp_internal.cuh"
#include "tc_common.cuh"

namespace dp {
namespace {

constexpr long kOzWait = 1L << 25;   // mbarrier polls (~1 s) before the kernel gives up

// Digits are stored pre-tiled in the layout the tensor cores read from
// shared memory, so that one bulk copy stages a K chunk: for a tile of TR
// rows (128 for A, NC for B) and a chunk of KC columns, the S digit planes
// follow each other, each a K-major core-matrix tile (kmaj_off).  Half
// offset of digit i (0-based) of element (r, k):
__host__ __device__ inline int64_t oz_tiled(int64_t r, int k, int i, int S, int TR, int KC, int K)
{
    const int64_t t = r / TR;
    const int rr = (int)(r - t * TR), c = k / KC, kk = k - c * KC;
    return (((t * (K / KC) + c) * S + i) * (int64_t)TR * KC) + tc::kmaj_off(rr, kk, KC) / 2;
}

template <int S, int BETA>
__global__ void k_oz_split(const double *__restrict__ X, int64_t ldx, int64_t rows, int64_t rows_pad, int K,
                           int TR, int KC, __half *__restrict__ dig, int *__restrict__ ex)
{
    constexpr long long H = 1LL << (BETA - 1), MASK = (1LL << BETA) - 1;
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows_pad) return;
    const bool live = r < rows;
    const double *x = X + r * ldx;
    double mx = 0.0;
    if (live)
        for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(x[k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = mx > 0.0 ? ilogb(mx) + 3 : 0;      // every |x_k| < 2^(e-2)
    if (lane == 0) ex[r] = e;
    for (int k = lane; k < K; k += 32) {
        long long m = live ? llrint(scalbn(x[k], BETA * S - e)) : 0LL;   // |m| <= 2^(BETA S - 2)
#pragma unroll
        for (int i = S; i >= 1; --i) {
            const long long d = ((m + H) & MASK) - H;                    // balanced digit
            m = (m - d) >> BETA;                                         // exact: m - d is a multiple of 2^BETA
            dig[oz_tiled(r, k, i - 1, S, TR, KC, K)] = __int2half_rn((int)d);
        }
    }
}

// Work unit: 128 rows of A x NC rows of B.  Shared memory holds NST
// stages, each the S digit planes of A (128 x KC) followed by those of B
// (NC x KC), K-major core-matrix tiles: the B planes stacked one after the
// other form one K-major tile of S NC rows.  Tensor memory holds one FP32
// accumulator of NC columns per diagonal g = i + j (g = 2 .. S+1) at column
// (g - 2) NC, so the products of A plane i with B planes 1 .. S+1-i land on
// diagonals i+1 .. S+1, columns (i - 1) NC onwards, contiguous: one MMA
// (split at 256 columns) per A plane and K step.
template <int S, int BETA, int NC, int KC>
struct OzShape {
    static constexpr uint32_t A_PLANE = 128 * KC * 2, B_PLANE = NC * KC * 2;
    static constexpr uint32_t A_BYTES = S * A_PLANE, B_BYTES = S * B_PLANE;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr int NST = (220 * 1024) / STAGE < 8 ? (220 * 1024) / STAGE : 8;
    static constexpr uint32_t SMEM = NST * STAGE;
    static constexpr uint32_t SBO = (KC / 8) * 128;   // 8-row groups of a K-major tile
    // diagonals 2 .. GH+1 are combined in one int64 (shifts <= 27 bits), the rest in another
    static constexpr int GH = (27 / BETA + 1) < S ? (27 / BETA + 1) : S;
    static_assert(KC % 16 == 0 && NC % 16 == 0 && NC >= 16, "MMA shape");
    static_assert(S * NC <= 512, "one accumulator per diagonal in tensor memory");
    static_assert(NST >= 2, "shared memory");
    static_assert((S - GH - 1) * BETA <= 27, "two groups of diagonals");
};

__device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}" : "=r"(pred));
    return pred != 0;
}

// 2^e as a double (built from its bits in the normal range).
__device__ __forceinline__ double pow2i(int e)
{
    return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : scalbn(1.0, e);
}

// All 32 lanes of the calling warp poll; the outcome is made warp-uniform.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, int64_t use, int nst)
{
    const bool ok = tc::mbar_wait(bar, (uint32_t)((use / nst) & 1), kOzWait);
    return __all_sync(0xffffffffu, ok);
}

template <int S, int BETA, int NC, int KC>
__global__ void __launch_bounds__(128, 1) k_oz_gemm(int64_t M, int N, int K, const __half *__restrict__ dA,
                                                   const int *__restrict__ eA, int64_t M_pad,
                                                   const __half *__restrict__ dB, const int *__restrict__ eB,
                                                   const double *__restrict__ bias, double *__restrict__ C,
                                                   int64_t ldc, int *err)
{
    using Sh = OzShape<S, BETA, NC, KC>;
    constexpr int NST = Sh::NST;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_t[NST], bar_m[NST];
    __shared__ uint32_t tmem_base;
    __shared__ int s_dead;
    const int tid = threadIdx.x, warp = tid >> 5;
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
    const uint32_t trow = tm + ((uint32_t)(warp * 32) << 16);
    const int nk = K / KC, nn = N / NC;
    const int64_t units = (M_pad / 128) * nn;
    // the chunks of this CTA in order: unit blockIdx.x + q gridDim.x, K chunk kc -> c = q nk + kc,
    // staged in stage c % NST
    const int64_t my_units = units > blockIdx.x ? (units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int64_t total = my_units * nk;
    const uint32_t sbase = tc::smem_u32(smem);
    int64_t issued = 0, mma_done = 0;   // chunks copied; chunks whose MMAs were waited for
    bool ok = true;
    // warp 0 copies and issues the MMAs (uniform control flow, one elected lane per instruction)
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
            tc::bulk_g2s(st + Sh::A_BYTES, dB + (((int64_t)nchunk * nk + kc) * S) * (int64_t)(NC * KC),
                         Sh::B_BYTES, &bar_t[s]);
        }
        __syncwarp();
    };
    if (warp == 0)
        for (; ok && issued < NST - 1 && issued < total; ++issued) copy_chunk(issued);
    for (int64_t q = 0; q < my_units; ++q) {
        const int64_t u = blockIdx.x + q * gridDim.x, tile = u / nn;
        const int n0 = (int)(u % nn) * NC;
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
        // epilogue: the accumulators are exact integers (|acc| < 2^24).  Diagonals
        // 2 .. GH+1 and GH+2 .. S+1 are summed exactly in int64 with their
        // relative weights (H, L), then
        // C = 2^(eA + eB) (H 2^(-BETA (GH+1)) + L 2^(-BETA (S+1))), one rounding.
        const int64_t r = tile * 128 + tid;
        const int er = eA[r];
#pragma unroll 1
        for (int c0 = 0; c0 < NC; c0 += 16) {
            long long H[16], L[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) H[c] = L[c] = 0;
#pragma unroll
            for (int g = 2; g <= S + 1; ++g) {
                float v[16];
                tc::tmem_ld16(trow + (uint32_t)((g - 2) * NC + c0), v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const long long iv = (long long)__float2int_rn(v[c]);
                    if (g <= Sh::GH + 1)
                        H[c] += iv << (BETA * (Sh::GH + 1 - g));
                    else
                        L[c] += iv << (BETA * (S + 1 - g));
                }
            }
            if (r < M) {
                double *out = C + r * ldc + n0 + c0;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int E = er + eB[n0 + c0 + c];
                    const double lo = (double)L[c] * pow2i(E - BETA * (S + 1));
                    const double y = fma((double)H[c], pow2i(E - BETA * (Sh::GH + 1)), lo);
                    out[c] = bias ? y + bias[n0 + c0 + c] : y;
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (s_dead && tid == 0) atomicOr(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

}  // namespace

// Digits of the rows of X [rows][K] (leading dimension ldx) into dig, tiled
// for tiles of TR rows and K chunks of KC (oz_tiled; rows >= rows are zero),
// and their scales ex [rows_pad].
template <int S, int BETA>
dp_status oz_split(const double *X, int64_t ldx, int64_t rows, int64_t rows_pad, int K, int TR, int KC, __half *dig,
                   int *ex, cudaStream_t st)
{
    if (rows_pad == 0) return DP_OK;
    if (rows_pad % TR || K % KC) {
        set_error("ozaki split: %lld rows / %d columns do not tile", (long long)rows_pad, K);
        return DP_ERR_ARG;
    }
    const unsigned blocks = (unsigned)((rows_pad * 32 + 255) / 256);
    k_oz_split<S, BETA><<<blocks, 256, 0, st>>>(X, ldx, rows, rows_pad, K, TR, KC, dig, ex);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// C [M][N] (leading dimension ldc) = A B^T (+ bias [N]) from the digits of A
// (tiled for 128 rows and KC columns, scales eA [M_pad]) and of B (tiled
// for NC rows and KC columns, scales eB [N]).
template <int S, int BETA, int NC, int KC>
dp_status oz_gemm(const dp_model *m, int64_t M, int N, int K, const __half *dA, const int *eA, int64_t M_pad,
                  const __half *dB, const int *eB, const double *bias, double *C, int64_t ldc, cudaStream_t st)
{
    using Sh = OzShape<S, BETA, NC, KC>;
    if (M == 0) return DP_OK;
    if (N % NC || K % KC || M_pad % 128 || M_pad < M) {
        set_error("ozaki GEMM: shape %lld x %d x %d does not fit the tiles", (long long)M, N, K);
        return DP_ERR_ARG;
    }
    if ((long long)S * K << (2 * BETA - 2) > (1LL << 24)) {
        set_error("ozaki GEMM: K = %d too large for exact FP32 sums of %d-bit digit products", K, BETA);
        return DP_ERR_ARG;
    }
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    const int64_t units = (M_pad / 128) * (N / NC);
    const unsigned grid = (unsigned)(units < nsm ? units : nsm);
    DP_CUDA(cudaFuncSetAttribute(k_oz_gemm<S, BETA, NC, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Sh::SMEM));
    k_oz_gemm<S, BETA, NC, KC><<<grid, 128, Sh::SMEM, st>>>(M, N, K, dA, eA, M_pad, dB, eB, bias, C, ldc, m->d_err);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// The two shapes of the fitting net's first layer: K = 1600 (z1 = D W1) with
// 6-bit digits (9 of them), and K = 240 (dD = dz1 W1^T) with 7-bit digits (8).
template dp_status oz_split<9, 6>(const double *, int64_t, int64_t, int64_t, int, int, int, __half *, int *,
                                  cudaStream_t);
template dp_status oz_split<8, 7>(const double *, int64_t, int64_t, int64_t, int, int, int, __half *, int *,
                                  cudaStream_t);
template dp_status oz_gemm<9, 6, 48, 16>(const dp_model *, int64_t, int, int, const __half *, const int *, int64_t,
                                         const __half *, const int *, const double *, double *, int64_t,
                                         cudaStream_t);
template dp_status oz_gemm<8, 7, 64, 16>(const dp_model *, int64_t, int, int, const __half *, const int *, int64_t,
                                         const __half *, const int *, const double *, double *, int64_t,
                                         cudaStream_t);

}  // namespace dp

using namespace dp;

extern "C" dp_status dp_ozaki_dgemm_dev(dp_model *m, int64_t M, int32_t N, int32_t K, const double *d_A,
                                        const double *d_Bt, double *d_C, void *stream)
{
    if (!m || M < 0 || N <= 0 || K <= 0 || (M > 0 && (!d_A || !d_Bt || !d_C))) {
        set_error("dp_ozaki_dgemm_dev: bad argument");
        return DP_ERR_ARG;
    }
    if (M == 0) return DP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t Mp = (M + 127) / 128 * 128;
    const bool small = K <= 256;   // 8 digits of 7 bits, else 9 of 6 bits
    const int S = small ? 8 : 9;
    if (K % 16 || (small ? N % 64 : N % 48) || K > 1808) {
        set_error("dp_ozaki_dgemm_dev: needs K %% 16 == 0, K <= 1808 and N %% 64 == 0 (K <= 256) or N %% 48 == 0");
        return DP_ERR_ARG;
    }
    __half *dA = nullptr, *dB = nullptr;
    int *eA = nullptr, *eB = nullptr;
    cudaError_t e = cudaMalloc((void **)&dA, sizeof(__half) * S * Mp * K);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dB, sizeof(__half) * S * (size_t)N * K);
    if (e == cudaSuccess) e = cudaMalloc((void **)&eA, sizeof(int) * Mp);
    if (e == cudaSuccess) e = cudaMalloc((void **)&eB, sizeof(int) * N);
    dp_status s = e == cudaSuccess ? DP_OK : DP_ERR_OOM;
    if (s == DP_OK) {
        if (small) {
            s = oz_split<8, 7>(d_A, K, M, Mp, K, 128, 16, dA, eA, st);
            if (s == DP_OK) s = oz_split<8, 7>(d_Bt, K, N, N, K, 64, 16, dB, eB, st);
            if (s == DP_OK) s = oz_gemm<8, 7, 64, 16>(m, M, N, K, dA, eA, Mp, dB, eB, nullptr, d_C, N, st);
        } else {
            s = oz_split<9, 6>(d_A, K, M, Mp, K, 128, 16, dA, eA, st);
            if (s == DP_OK) s = oz_split<9, 6>(d_Bt, K, N, N, K, 48, 16, dB, eB, st);
            if (s == DP_OK) s = oz_gemm<9, 6, 48, 16>(m, M, N, K, dA, eA, Mp, dB, eB, nullptr, d_C, N, st);
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && s == DP_OK) s = DP_ERR_CUDA;
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(eA);
    cudaFree(eB);
    if (s == DP_OK) {
        int32_t derr = 0;
        cudaMemcpy(&derr, m->d_err, sizeof(derr), cudaMemcpyDeviceToHost);
        if (derr) {
            cudaMemset(m->d_err, 0, sizeof(int32_t));
            set_error("a bounded device wait gave up");
            return DP_ERR_TIMEOUT;
        }
    }
    return s;
}

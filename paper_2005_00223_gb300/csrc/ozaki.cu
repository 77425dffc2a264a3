// FP64 matrix products on the 5th-generation tensor cores by error-free
// splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)); the
// digit representation, its error and the MMA pipeline are described in
// ozaki.cuh.
//
// C = A B^T with A [M][K] and B [N][K] in FP64: k_oz_split writes the
// digits of the rows of each operand (one warp per row), pre-tiled in the
// shared-memory layout of the MMAs; oz::k_gemm with the plain epilogue
// below (C = value + bias) computes C.  The error is that of a dot product
// of the digit-truncated rows, of the order of K 2^-52 |a|_max |b|_max per
// entry, the size of FP64 rounding.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"
#include "ozaki.cuh"

namespace dp {
namespace {

template <int S, int BETA>
__global__ void k_oz_split(const double *__restrict__ X, int64_t ldx, int64_t rows, int64_t rows_pad, int K,
                           int K_pad, int TR, int KC, __half *__restrict__ dig, int *__restrict__ ex)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows_pad) return;
    const bool live = r < rows;
    const double *x = X + r * ldx;
    double mx = 0.0;
    if (live)
        for (int k = lane; k < K; k += 32) mx = oz::amax(mx, x[k]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = oz::row_exp(mx);
    if (lane == 0) ex[r] = e;
    for (int k = lane; k < K_pad; k += 32) {
        int d[S];
        oz::digits<S, BETA>(live && k < K ? x[k] : 0.0, e, d);
#pragma unroll
        for (int i = 0; i < S; ++i) dig[oz::tiled(r, k, i, S, TR, KC, K_pad)] = __int2half_rn(d[i]);
    }
}

// C [M][N] (leading dimension ldc) = value (+ bias [N]), or C += value.
template <class Sh>
struct PlainEpi {
    const __half *dB;
    int nk;
    const int *eA, *eB;
    const double *bias;
    double *C;
    int64_t ldc, M;
    bool acc;
    __device__ const __half *b_unit(int64_t, int nchunk) const
    {
        return dB + (int64_t)nchunk * nk * Sh::S * Sh::NC * Sh::KC;
    }
    __device__ void operator()(int64_t tile, int nchunk, uint32_t trow, int tid, unsigned char *) const
    {
        const int64_t r = tile * 128 + tid;
        const int er = eA[r], n0 = nchunk * Sh::NC;
#pragma unroll 1
        for (int c0 = 0; c0 < Sh::NC; c0 += 16) {
            long long H[16], L[16];
            oz::acc_load16<Sh>(trow, c0, H, L);
            if (r < M) {
                double *out = C + r * ldc + n0 + c0;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const double y = oz::acc_value<Sh>(H[c], L[c], er + eB[n0 + c0 + c]);
                    out[c] = acc ? out[c] + y : (bias ? y + bias[n0 + c0 + c] : y);
                }
            }
        }
    }
};

}  // namespace

// Digits of the rows of X [rows][K] (leading dimension ldx; columns K ..
// K_pad-1 and rows >= rows are zero) into dig, tiled for tiles of TR rows
// and K chunks of KC (oz::tiled), and their scales ex [rows_pad].
template <int S, int BETA>
dp_status oz_split(const double *X, int64_t ldx, int64_t rows, int64_t rows_pad, int K, int K_pad, int TR, int KC,
                   __half *dig, int *ex, cudaStream_t st)
{
    if (rows_pad == 0) return DP_OK;
    if (rows_pad % TR || K_pad % KC || K > K_pad) {
        set_error("ozaki split: %lld rows / %d columns do not tile", (long long)rows_pad, K_pad);
        return DP_ERR_ARG;
    }
    const unsigned blocks = (unsigned)((rows_pad * 32 + 255) / 256);
    k_oz_split<S, BETA><<<blocks, 256, 0, st>>>(X, ldx, rows, rows_pad, K, K_pad, TR, KC, dig, ex);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// C [M][N] (leading dimension ldc) = A B^T (+ bias [N]) from the digits of A
// (tiled for 128 rows and KC columns, scales eA [M_pad]) and of B (tiled
// for NC rows and KC columns, scales eB [N]).
template <int S, int BETA, int NC, int KC>
dp_status oz_gemm(const dp_model *m, int64_t M, int N, int K, const __half *dA, const int *eA, int64_t M_pad,
                  const __half *dB, const int *eB, const double *bias, double *C, int64_t ldc, cudaStream_t st,
                  bool accumulate)
{
    using Sh = oz::Shape<S, BETA, NC, KC>;
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
    PlainEpi<Sh> epi{dB, K / KC, eA, eB, bias, C, ldc, M, accumulate};
    auto kern = oz::k_gemm<Sh, PlainEpi<Sh>>;
    static bool attrs_set = false;   // per instantiation: once per process
    if (!attrs_set) {
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
        // the smallest shared-memory carveout that holds the stages: the rest of the SM's 256 KB stays L1
        DP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)((Sh::SMEM + 2048) * 100 / (228 * 1024)) + 1));
        attrs_set = true;
    }
    kern<<<grid, 128, Sh::SMEM, st>>>(M_pad, nullptr, N, K, dA, epi, m->d_err);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// The two shapes of the fitting net's first layer: K = 1600 (z1 = D W1) with
// 6-bit digits (9 of them), and K = 240 (dD = dz1 W1^T) with 7-bit digits (8).
template dp_status oz_split<9, 6>(const double *, int64_t, int64_t, int64_t, int, int, int, int, __half *, int *,
                                  cudaStream_t);
template dp_status oz_split<8, 7>(const double *, int64_t, int64_t, int64_t, int, int, int, int, __half *, int *,
                                  cudaStream_t);
template dp_status oz_gemm<9, 6, 48, 16>(const dp_model *, int64_t, int, int, const __half *, const int *, int64_t,
                                         const __half *, const int *, const double *, double *, int64_t,
                                         cudaStream_t, bool);
template dp_status oz_gemm<8, 7, 64, 16>(const dp_model *, int64_t, int, int, const __half *, const int *, int64_t,
                                         const __half *, const int *, const double *, double *, int64_t,
                                         cudaStream_t, bool);

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
            s = oz_split<8, 7>(d_A, K, M, Mp, K, K, 128, 16, dA, eA, st);
            if (s == DP_OK) s = oz_split<8, 7>(d_Bt, K, N, N, K, K, 64, 16, dB, eB, st);
            if (s == DP_OK) s = oz_gemm<8, 7, 64, 16>(m, M, N, K, dA, eA, Mp, dB, eB, nullptr, d_C, N, st);
        } else {
            s = oz_split<9, 6>(d_A, K, M, Mp, K, K, 128, 16, dA, eA, st);
            if (s == DP_OK) s = oz_split<9, 6>(d_Bt, K, N, N, K, K, 48, 16, dB, eB, st);
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

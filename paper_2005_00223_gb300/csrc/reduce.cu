// Deterministic reductions: E = sum_i E_i and W = sum_i W_i in a fixed order
// (kRedParts blocks over contiguous atom ranges, strided partial sums and a
// fixed tree in each, then the last block to finish over the partial sums in
// block order), plus a scan of
// the forces for NaN / Inf.  E is summed in FP64 as Sec. 4.1.3 prescribes
// for the mixed schemes too.
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"

namespace dp {
namespace {

constexpr int kRedThreads = 256;

// Fixed-shape tree over the block's kRedThreads values of 10 sums.
__device__ __forceinline__ void block_tree(double (*s)[kRedThreads], double acc[10])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q][t] = acc[q];
    __syncthreads();
    for (int h = kRedThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
#pragma unroll
            for (int q = 0; q < 10; ++q) s[q][t] += s[q][t + h];
        }
        __syncthreads();
    }
}

// One launch: kRedParts blocks form the partial sums over contiguous atom
// ranges; the last block to finish (arrival counter after the partials)
// sums them in block order with the same fixed tree and resets the counter.
__global__ void __launch_bounds__(kRedThreads) k_reduce(const double *__restrict__ Ei, const double *__restrict__ Wi,
                                                       int64_t n, double *__restrict__ part,
                                                       unsigned int *__restrict__ counter, double *__restrict__ E,
                                                       double *__restrict__ W)
{
    __shared__ double s[10][kRedThreads];
    __shared__ bool last;
    const int t = threadIdx.x;
    const int64_t per = (n + kRedParts - 1) / kRedParts;
    const int64_t b0 = blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
    double acc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (int64_t i = b0 + t; i < b1; i += kRedThreads) {
        acc[0] += Ei[i];
        if (Wi) {
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[1 + q] += Wi[9 * i + q];
        }
    }
    block_tree(s, acc);
    if (t < 10) part[blockIdx.x * 10 + t] = s[t][0];
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(counter, 1u) == (unsigned)(kRedParts - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (int b = t; b < kRedParts; b += kRedThreads) {
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] += __ldcg(part + b * 10 + q);
    }
    block_tree(s, acc);
    if (t == 0) {
        E[0] = s[0][0];
        if (W && Wi)
            for (int q = 0; q < 9; ++q) W[q] = s[1 + q][0];
        *counter = 0u;
    }
}

__global__ void k_nonfinite(const double *__restrict__ x, int64_t n, int32_t *flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicOr(flag, 1);
}

}  // namespace

dp_status reduce_energy_virial(const double *d_atom_energy, const double *d_atom_virial, int64_t n,
                               double *d_energy, double *d_virial, double *d_scratch, cudaStream_t st)
{
    k_reduce<<<kRedParts, kRedThreads, 0, st>>>(d_atom_energy, d_atom_virial, n, d_scratch,
                                                reinterpret_cast<unsigned int *>(d_scratch + kRedParts * 10),
                                                d_energy, d_virial);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

dp_status check_nonfinite(const double *d_x, int64_t n, int32_t *d_flag, cudaStream_t st)
{
    if (n == 0) return DP_OK;
    k_nonfinite<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_x, n, d_flag);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace dp

// Deterministic reductions: E = sum_i E_i and W = sum_i W_i in a fixed order
// (one block, strided partial sums, then a fixed tree), plus a scan of the
// forces for NaN / Inf.  E is summed in FP64 as Sec. 4.1.3 prescribes for
// the mixed schemes too.
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"

namespace dp {
namespace {

constexpr int kRedThreads = 512;

__global__ void __launch_bounds__(kRedThreads) k_reduce(const double *__restrict__ Ei, const double *__restrict__ Wi,
                                                       int64_t n, double *__restrict__ E, double *__restrict__ W)
{
    __shared__ double s[10][kRedThreads];
    const int t = threadIdx.x;
    double acc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (int64_t i = t; i < n; i += kRedThreads) {
        acc[0] += Ei[i];
        if (Wi) {
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[1 + q] += Wi[9 * i + q];
        }
    }
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
    if (t == 0) {
        E[0] = s[0][0];
        if (W && Wi)
            for (int q = 0; q < 9; ++q) W[q] = s[1 + q][0];
    }
}

__global__ void k_nonfinite(const double *__restrict__ x, int64_t n, int32_t *flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicOr(flag, 1);
}

}  // namespace

dp_status reduce_energy_virial(const double *d_atom_energy, const double *d_atom_virial, int64_t n,
                               double *d_energy, double *d_virial, cudaStream_t st)
{
    k_reduce<<<1, kRedThreads, 0, st>>>(d_atom_energy, d_atom_virial, n, d_energy, d_virial);
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

// Deterministic reductions: E = sum_i E_i and W = sum_i W_i in a fixed order
// (up to 152 blocks over contiguous atom ranges, strided partial sums and a
// fixed warp butterfly in each, then the last block to finish over the partial
// sums in block order), plus a scan of
// the forces for NaN / Inf.  E is summed in FP64 as Sec. 4.1.3 prescribes
// for the mixed schemes too.
#include <cuda_runtime.h>
#include <math.h>

#include "dp_internal.cuh"

namespace dp {
namespace {

constexpr int kRedThreads = 256;

// Fixed-order sum over the block's threads of 10 values each, returned to
// threads 0..9 (sum q at thread q).  Within a warp a butterfly
// reduce-scatter over 16 slots (10 used): at each of 4 levels a lane keeps
// half of its slots and adds the partner's copy of them, so after the last
// exchange lanes 2q and 2q+1 hold the warp total of slot q; 16 FP64 adds per
// lane instead of 50 for ten separate shuffle trees, and far fewer than a
// shared-memory tree (GB300 runs FP64 at 1/64 of the FP32 rate).  The 8 warp
// totals are then added in warp order.
__device__ __forceinline__ double block_sum10(double v[16], double (*s)[10])
{
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
#pragma unroll
    for (int lv = 0; lv < 4; ++lv) {
        const int half = 8 >> lv, off = 16 >> lv;
        const bool up = lane & off;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double keep = up ? v[i + half] : v[i];
            const double give = up ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, off);
        }
    }
    const double tot = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int q = (lane >> 1) & 15;
    __syncthreads();   // s free from any earlier use
    if (!(lane & 1) && q < 10) s[warp][q] = tot;
    __syncthreads();
    double x = 0.0;
    if (t < 10) {
        x = s[0][t];
#pragma unroll
        for (int w = 1; w < kRedThreads / 32; ++w) x += s[w][t];
    }
    return x;
}

// One launch: gridDim.x (<= kRedParts, a function of n) blocks form the
// partial sums over contiguous atom ranges; the last block to finish
// (arrival counter after the partials) sums them in block order the same
// way and resets the counter.
__global__ void __launch_bounds__(kRedThreads) k_reduce(const double *__restrict__ Ei, const double *__restrict__ Wi,
                                                       int64_t n, double *__restrict__ part,
                                                       unsigned int *__restrict__ counter, double *__restrict__ E,
                                                       double *__restrict__ W)
{
    __shared__ double s[kRedThreads / 32][10];
    __shared__ bool last;
    const int t = threadIdx.x;
    const int parts = gridDim.x;
    const int64_t per = (n + parts - 1) / parts;
    const int64_t b0 = blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int64_t i = b0 + t; i < b1; i += kRedThreads) {
        acc[0] += Ei[i];
        if (Wi) {
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[1 + q] += Wi[9 * i + q];
        }
    }
    double x = block_sum10(acc, s);
    if (t < 10) part[blockIdx.x * 10 + t] = x;
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(counter, 1u) == (unsigned)(parts - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int b = t; b < parts; b += kRedThreads) {
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] += __ldcg(part + b * 10 + q);
    }
    x = block_sum10(acc, s);
    if (t == 0) E[0] = x;
    if (t >= 1 && t < 10 && W && Wi) W[t - 1] = x;
    if (t == 0) *counter = 0u;
}

__global__ void k_nonfinite(const double *__restrict__ x, int64_t n, int32_t *flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicOr(flag, 1);
}

// The FP64 value of each fixed-point accumulator (fx_add): integer part plus the two fraction limbs
// scaled by 2^-32 and 2^-64, summed in that order (each limb sum is exact; the conversions and the
// two additions round the same way every time).
__global__ void k_fx_finish(int64_t count, const unsigned long long *__restrict__ l, double *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const unsigned long long *v = l + 3 * i;
    out[i] = (double)(long long)v[0] + (double)v[1] * 0x1p-32 + (double)v[2] * 0x1p-64;
}

}  // namespace

dp_status reduce_energy_virial(const double *d_atom_energy, const double *d_atom_virial, int64_t n,
                               double *d_energy, double *d_virial, double *d_scratch, cudaStream_t st)
{
    // about 64 atoms per block up to one block per SM (152): the block sums dominate, not the loads
    const int64_t want = (n + 63) / 64;
    const unsigned parts = (unsigned)(want < 1 ? 1 : (want > 152 ? 152 : want));
    k_reduce<<<parts, kRedThreads, 0, st>>>(d_atom_energy, d_atom_virial, n, d_scratch,
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

dp_status fx_finish(int64_t count, const unsigned long long *l, double *out, cudaStream_t st)
{
    if (count <= 0) return DP_OK;
    k_fx_finish<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, l, out);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace dp

// Spatial decomposition support (Sec. 4.3, "Reducing MPI communication
// bottlenecks"): the paper runs DP inside LAMMPS's spatial partitioning, where
// each rank evaluates the atoms of its sub-domain with the ghost atoms of a
// halo around it and the forces on ghosts go back to their owners.  This
// file holds the device side of that scheme for one rank:
//  - ghost atoms in a neighbor list (dp_nlist_set_centers): atoms
//    [n_centers, n) are neighbors of the centers but not centers themselves;
//    their list rows are cleared after every format, so they carry no
//    energy, no virial and no forces of their own, only the reactions
//    F_j -= g_ij of the centers' pairs;
//  - the halo selection (dp_halo_select_dev): the atoms of a slab of x,
//    packed with their coordinates shifted into the receiver's frame, in
//    index order (a deterministic compaction);
//  - the reverse halo (dp_halo_accumulate_dev): forces of returned ghosts
//    added into their owners' forces.
// The exchanges themselves (positions out, ghost forces back, the energy and
// virial sums) are collectives of the caller (torch.distributed over NCCL or
// gloo in the Python package).
#include <cuda_runtime.h>

#include "dp_internal.cuh"

namespace dp {

namespace {

constexpr int kSelThreads = 1024;

// Rows of atoms [c0, n): every slot -1, no neighbor of any type.
__global__ void k_clear_ghost_rows(int64_t c0, int64_t n, int nsel, int ntypes, int32_t *__restrict__ nlist,
                                   int32_t *__restrict__ nnei)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t rows = n - c0;
    if (q < rows * nsel) nlist[c0 * nsel + q] = -1;
    if (q < rows * ntypes) nnei[c0 * ntypes + q] = 0;
}

// One block walks the atoms in chunks of kSelThreads: in-slab flags, a block
// scan of each chunk, and the packed outputs in index order.
__global__ void __launch_bounds__(kSelThreads) k_halo_select(int64_t n, const double *__restrict__ coord,
                                                            const int32_t *__restrict__ type, double lo, double hi,
                                                            double shift_x, int64_t cap, int32_t *__restrict__ idx,
                                                            double *__restrict__ out_coord,
                                                            int32_t *__restrict__ out_type, int64_t *count)
{
    __shared__ int warp_sums[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t base_out = 0;
    for (int64_t c = 0; c < n; c += kSelThreads) {
        const int64_t i = c + t;
        const double x = i < n ? coord[3 * i] : 0.0;
        const int in = (i < n && x >= lo && x < hi) ? 1 : 0;
        // exclusive scan of `in` over the block
        int v = in;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) warp_sums[w] = v;
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
        const int excl = v - in + (w > 0 ? warp_sums[w - 1] : 0);
        const int total = warp_sums[31];
        const int64_t p = base_out + excl;
        if (in && p < cap) {
            idx[p] = (int32_t)i;
            out_coord[3 * p] = x + shift_x;
            out_coord[3 * p + 1] = coord[3 * i + 1];
            out_coord[3 * p + 2] = coord[3 * i + 2];
            out_type[p] = type[i];
        }
        base_out += total;
        __syncthreads();
    }
    if (t == 0) *count = base_out;
}

__global__ void k_halo_accumulate(int64_t m, const int32_t *__restrict__ idx, const double *__restrict__ f_ghost,
                                  double *__restrict__ force)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int64_t i = idx[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) force[3 * i + c] += f_ghost[3 * k + c];
}

}  // namespace

void nlist_graph_drop(dp_nlist *nl)
{
    if (nl->cgraph_exec) cudaGraphExecDestroy(nl->cgraph_exec);
    if (nl->cgraph) cudaGraphDestroy(nl->cgraph);
    nl->cgraph_exec = nullptr;
    nl->cgraph = nullptr;
}

dp_status clear_ghost_rows(const dp_model *m, dp_nlist *nl, cudaStream_t st)
{
    const int64_t c0 = centers_of(nl), rows = nl->n - c0;
    if (rows <= 0) return DP_OK;
    const int64_t work = rows * (m->dev.nsel > m->dev.ntypes ? m->dev.nsel : m->dev.ntypes);
    k_clear_ghost_rows<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(c0, nl->n, m->dev.nsel, m->dev.ntypes,
                                                                      nl->d_nlist, nl->d_nnei);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace dp

using namespace dp;

extern "C" {

dp_status dp_nlist_set_centers(dp_nlist *nl, int64_t n_centers)
{
    if (!nl || n_centers < 0 || n_centers > nl->n) {
        set_error("dp_nlist_set_centers: NULL list or n_centers outside 0..n");
        return DP_ERR_ARG;
    }
    nl->n_centers = n_centers;
    nlist_graph_drop(nl);   // a captured evaluation holds the old launches
    return DP_OK;
}

dp_status dp_halo_select_dev(int64_t n, const double *d_coord, const int32_t *d_type, double lo, double hi,
                             double shift_x, int64_t cap, int32_t *d_idx, double *d_out_coord, int32_t *d_out_type,
                             int64_t *d_count, void *stream)
{
    if (n < 0 || cap < 0 || !d_count || (n > 0 && (!d_coord || !d_type)) ||
        (cap > 0 && (!d_idx || !d_out_coord || !d_out_type)) || n > (int64_t)INT32_MAX) {
        set_error("dp_halo_select_dev: invalid arguments");
        return DP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_halo_select<<<1, kSelThreads, 0, st>>>(n, d_coord, d_type, lo, hi, shift_x, cap, d_idx, d_out_coord, d_out_type,
                                             d_count);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

dp_status dp_halo_accumulate_dev(int64_t m, const int32_t *d_idx, const double *d_f_ghost, double *d_force,
                                 void *stream)
{
    if (m < 0 || (m > 0 && (!d_idx || !d_f_ghost || !d_force))) {
        set_error("dp_halo_accumulate_dev: invalid arguments");
        return DP_ERR_ARG;
    }
    if (m == 0) return DP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    k_halo_accumulate<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, d_idx, d_f_ghost, d_force);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // extern "C"

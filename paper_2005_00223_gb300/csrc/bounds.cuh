// Bounds-checked debug build of libdp (the stand-in for a memory checker).
//
// Built with -DDP_BOUNDS_CHECK (paper_2005_00223_gb300.build(bounds_check=True), a library of its
// own under _build_bounds/), every index that a kernel reads from memory or derives from
// coordinates is checked against the size of the buffer it addresses before it is used: neighbor
// indexes of the formatted and candidate lists, atoms of the cell lists and of the tensor-core work
// lists, cell indexes computed from positions, type ids read back from packed keys.  A bad index is
// not used (the neighbor is treated as padding or the access is skipped) and the first one is
// recorded.  Loop bounds that the host derives from validated sizes are not re-checked, nor are the
// halo kernels (their indexes come from the selection kernel's own count) and the allocation-free
// list (its own limits are checked on the host and flagged on the device).
//
// Each translation unit keeps its own record, a file-scope device array {count of bad indexes,
// site, index, limit}; dp_bounds_read() (prof.cu) collects and clears them.  In the default build
// every check is the constant `true` and the records hold zeros.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dp {

// Where a bad index was found (the record's site field).
enum BoundsSite {
    BS_NONE = 0,
    BS_TYPE = 1,            // type id read back from a packed key or a work-list chunk: [0, ntypes)
    BS_CELL = 2,            // cell index from a position (cell grid): [0, ncell)
    BS_CELL_SLOT = 3,       // slot of an atom in the cell list: [0, n)
    BS_CAND_J = 4,          // atom of a candidate list entry or of a cell list: [0, n)
    BS_NLIST_J = 5,         // neighbor index of the formatted list: [0, n)
    BS_CHUNK_ATOM = 6,      // center atom of a tensor-core work-list chunk: [0, n)
};

#ifdef DP_BOUNDS_CHECK
static __device__ unsigned long long g_bounds[4];

__device__ __forceinline__ bool bounds_ok(long long idx, long long limit, int site)
{
    if (idx >= 0 && idx < limit) return true;
    if (atomicAdd(&g_bounds[0], 1ull) == 0ull) {
        g_bounds[1] = (unsigned long long)site;
        g_bounds[2] = (unsigned long long)idx;
        g_bounds[3] = (unsigned long long)limit;
    }
    return false;
}
#define DP_IDX_OK(idx, limit, site) ::dp::bounds_ok((long long)(idx), (long long)(limit), (int)(site))

// Host accessor of this translation unit's record: copies it to out[4], then zeroes it if clear.
#define DP_BOUNDS_ACCESSOR(NAME)                                                              \
    cudaError_t NAME(unsigned long long *out, bool clear)                                     \
    {                                                                                         \
        cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds, sizeof(g_bounds));                \
        if (e == cudaSuccess && clear) {                                                      \
            const unsigned long long z[4] = {0ull, 0ull, 0ull, 0ull};                         \
            e = cudaMemcpyToSymbol(g_bounds, z, sizeof(z));                                   \
        }                                                                                     \
        return e;                                                                             \
    }
#else
#define DP_IDX_OK(idx, limit, site) true
#define DP_BOUNDS_ACCESSOR(NAME)                                                              \
    cudaError_t NAME(unsigned long long *out, bool)                                           \
    {                                                                                         \
        out[0] = out[1] = out[2] = out[3] = 0ull;                                             \
        return cudaSuccess;                                                                   \
    }
#endif

// One accessor per translation unit that checks indexes.
cudaError_t bounds_read_nlist(unsigned long long *out, bool clear);
cudaError_t bounds_read_simt(unsigned long long *out, bool clear);
cudaError_t bounds_read_oz_embed(unsigned long long *out, bool clear);
cudaError_t bounds_read_tc(unsigned long long *out, bool clear);
cudaError_t bounds_read_tc_x3(unsigned long long *out, bool clear);
cudaError_t bounds_read_wide(unsigned long long *out, bool clear);
cudaError_t bounds_read_grad(unsigned long long *out, bool clear);

}  // namespace dp

// Formatted neighbor list without device allocation (dp_nlist_format_noalloc).
//
// For callers that cannot allocate device memory: code that runs inside a
// host application whose device memory is owned by another allocator (an MD
// engine's pool, a framework's caching allocator) or that must not let
// cudaMalloc / cudaFree synchronise the device in the middle of its own
// work.  The caller passes the coordinates, types and the output buffers;
// the only scratch memory (the cell grid) is a file-scope static device
// array of fixed size, so this entry point never allocates.
//
// The list is the same canonical list as dp_nlist_build + dp_nlist_get
// produce (same explicitly rounded FP64 distances, same packed key order),
// built in one pass from the cell grid with no candidate list.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "dp_internal.cuh"

namespace dp {
namespace {

constexpr int64_t kNaMaxAtoms = 131072;        // atoms per call
constexpr int64_t kNaMaxCells = 65536;         // cells of the grid (larger cells are used above this)
constexpr int kNaMaxKeys = 1024;               // neighbors within r_c per atom
constexpr int kNaWarps = 4;

// cell_of [max atoms], cell_atoms [max atoms], cell_cnt [max cells + 1], cell_start [max cells + 1]
constexpr size_t kNaScratchBytes =
    sizeof(int32_t) * (2 * (size_t)kNaMaxAtoms + 2 * ((size_t)kNaMaxCells + 1));

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

struct NaBox {
    double L[3], invL[3];
    int nc[3];
};

__device__ __forceinline__ double na_dist(const double *__restrict__ coord, int64_t i, int64_t j, const NaBox &bx)
{
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double dk = __dsub_rn(coord[3 * j + k], coord[3 * i + k]);
        double nk = rint(__dmul_rn(dk, bx.invL[k]));
        d[k] = __dsub_rn(dk, __dmul_rn(bx.L[k], nk));
    }
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    return __dsqrt_rn(r2);
}

__device__ __forceinline__ int na_cell(double x, double invL, int nc)
{
    double f = x * invL;
    f -= floor(f);
    int c = (int)(f * nc);
    return c >= nc ? nc - 1 : (c < 0 ? 0 : c);
}

__global__ void k_na_zero(int64_t ncell, int32_t *cnt)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c <= ncell) cnt[c] = 0;
}

__global__ void k_na_assign(int64_t n, const double *__restrict__ coord, NaBox bx, int32_t *cell_of, int32_t *cnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (na_cell(coord[3 * i], bx.invL[0], bx.nc[0]) * bx.nc[1] + na_cell(coord[3 * i + 1], bx.invL[1], bx.nc[1])) *
                      bx.nc[2] +
                  na_cell(coord[3 * i + 2], bx.invL[2], bx.nc[2]);
    cell_of[i] = c;
    atomicAdd(&cnt[c], 1);
}

__global__ void __launch_bounds__(1024) k_na_scan(int64_t ncell, int32_t *cnt, int32_t *start)
{
    __shared__ int32_t part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int64_t per = (ncell + nt - 1) / nt;
    const int64_t b = t * per, e = b + per < ncell ? b + per : ncell;
    int32_t s = 0;
    for (int64_t c = b; c < e; ++c) s += cnt[c];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {
        int32_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = part[t] - s;
    for (int64_t c = b; c < e; ++c) {
        const int32_t v = cnt[c];
        start[c] = run;
        run += v;
        cnt[c] = 0;
    }
    if (t == nt - 1) start[ncell] = part[t];
}

__global__ void k_na_fill(int64_t n, const int32_t *cell_of, const int32_t *start, int32_t *cursor, int32_t *atoms)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    atoms[start[c] + atomicAdd(&cursor[c], 1)] = (int32_t)i;
}

struct NaSel {
    int ntypes, nsel;
    int sel[kMaxTypes], off[kMaxTypes];
};

// One warp per atom: keys (type:8 | floor(r 1e8):30 | j:26) of every j in
// the surrounding cells with r < r_c, ranked by counting, written in
// type blocks of sel_t slots, padded with -1.
__global__ void __launch_bounds__(32 * kNaWarps) k_na_format(int64_t n, const double *__restrict__ coord,
                                                            const int32_t *__restrict__ type, NaBox bx, double rcut,
                                                            NaSel ns, const int32_t *__restrict__ cell_of,
                                                            const int32_t *__restrict__ start,
                                                            const int32_t *__restrict__ atoms,
                                                            int32_t *__restrict__ nlist,
                                                            unsigned long long *__restrict__ ntrunc,
                                                            int32_t *__restrict__ status)
{
    __shared__ unsigned long long keys_all[kNaWarps][kNaMaxKeys];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)kNaWarps + warp;
    if (i >= n) return;
    unsigned long long *keys = keys_all[warp];
    const int c = cell_of[i];
    const int c3[3] = {c / (bx.nc[1] * bx.nc[2]), (c / bx.nc[2]) % bx.nc[1], c % bx.nc[2]};
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (bx.nc[k] >= 3) { lo[k] = -1; hi[k] = 1; }
        else { lo[k] = -c3[k]; hi[k] = bx.nc[k] - 1 - c3[k]; }
    }
    int nk = 0;
    bool over = false;
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int e = lo[2]; e <= hi[2]; ++e) {
                const int x = (c3[0] + a + bx.nc[0]) % bx.nc[0];
                const int y = (c3[1] + b + bx.nc[1]) % bx.nc[1];
                const int z = (c3[2] + e + bx.nc[2]) % bx.nc[2];
                const int cell = (x * bx.nc[1] + y) * bx.nc[2] + z;
                const int s0 = start[cell], s1 = start[cell + 1];
                for (int base = s0; base < s1; base += 32) {
                    const int p = base + lane;
                    bool ok = false, bad = false;
                    unsigned long long key = 0;
                    if (p < s1) {
                        const int32_t j = atoms[p];
                        const int tj = type[j];
                        bad = tj < 0 || tj >= ns.ntypes;
                        if (j != i && !bad) {
                            const double r = na_dist(coord, i, j, bx);
                            if (r < rcut) {
                                ok = true;
                                const unsigned long long q = (unsigned long long)floor(__dmul_rn(r, 1e8));
                                key = ((unsigned long long)tj << 56) | (q << 26) | (unsigned long long)j;
                            }
                        }
                    }
                    if (bad) over = true;   // reported below; such neighbors are left out
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    const int off = __popc(m & ((1u << lane) - 1u));
                    if (ok && nk + off < kNaMaxKeys) keys[nk + off] = key;
                    nk += __popc(m);
                }
            }
    over = __any_sync(0xffffffffu, over);
    if (nk > kNaMaxKeys) {
        over = true;
        nk = kNaMaxKeys;
    }
    __syncwarp();
    int tcount[kMaxTypes];
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t) tcount[t] = 0;
    for (int p = lane; p < nk; p += 32) {
        const int t = (int)(keys[p] >> 56);
#pragma unroll
        for (int u = 0; u < kMaxTypes; ++u) tcount[u] += (t == u);
    }
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t)
        for (int o = 16; o > 0; o >>= 1) tcount[t] += __shfl_xor_sync(0xffffffffu, tcount[t], o);
    int tstart[kMaxTypes], acc = 0;
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t) { tstart[t] = acc; acc += tcount[t]; }
    int32_t *out = nlist + i * (int64_t)ns.nsel;
    for (int p = lane; p < nk; p += 32) {
        const unsigned long long k = keys[p];
        int rank = 0;
        for (int q = 0; q < nk; ++q) rank += keys[q] < k;
        const int t = (int)(k >> 56);
        const int local = rank - tstart[t];
        if (local < ns.sel[t]) out[ns.off[t] + local] = (int32_t)(k & ((1ull << 26) - 1));
    }
    unsigned long long dropped = 0;
    for (int t = 0; t < ns.ntypes; ++t) {
        const int kept = tcount[t] < ns.sel[t] ? tcount[t] : ns.sel[t];
        for (int s = kept + lane; s < ns.sel[t]; s += 32) out[ns.off[t] + s] = -1;
        if (tcount[t] > ns.sel[t]) dropped += (unsigned long long)(tcount[t] - ns.sel[t]);
    }
    if (lane == 0) {
        if (dropped) atomicAdd(ntrunc, dropped);
        if (over) atomicOr(status, 1);
    }
}

// Device address of the static scratch, looked up once per device.
std::mutex g_na_lock;
void *g_na_addr[64] = {nullptr};

dp_status na_scratch(int dev, void **out)
{
    std::lock_guard<std::mutex> g(g_na_lock);
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return DP_ERR_ARG;
    }
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static neighbor-list scratch)");
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return DP_OK;
}

}  // namespace
}  // namespace dp

using namespace dp;

extern "C" {

dp_status dp_nlist_format_noalloc(int64_t n, const double *d_coord, const int32_t *d_type, const double box[9],
                                  double rcut, int32_t ntypes, const int32_t *sel, int32_t *d_nlist,
                                  unsigned long long *d_ntrunc, int32_t *d_status, void *stream)
{
    if (!box || !sel || !d_ntrunc || !d_status || (n > 0 && (!d_coord || !d_type || !d_nlist))) {
        set_error("dp_nlist_format_noalloc: NULL argument");
        return DP_ERR_ARG;
    }
    if (n < 0 || n > kNaMaxAtoms) {
        set_error("dp_nlist_format_noalloc: %lld atoms exceed the static scratch limit of %lld", (long long)n,
                  (long long)kNaMaxAtoms);
        return DP_ERR_ARG;
    }
    if (ntypes < 1 || ntypes > kMaxTypes || !(rcut > 0) || !(rcut * 1e8 < (double)(1 << 30))) {
        set_error("dp_nlist_format_noalloc: ntypes must be 1..%d and 0 < rcut < 10.7 A", kMaxTypes);
        return DP_ERR_ARG;
    }
    NaSel ns{};
    ns.ntypes = ntypes;
    for (int t = 0; t < ntypes; ++t) {
        if (sel[t] < 1) { set_error("dp_nlist_format_noalloc: sel[%d] < 1", t); return DP_ERR_ARG; }
        ns.sel[t] = sel[t];
        ns.off[t] = ns.nsel;
        ns.nsel += sel[t];
    }
    double L[3];
    DP_TRY(check_box(box, rcut, L));
    NaBox bx;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        bx.L[k] = L[k];
        bx.invL[k] = 1.0 / L[k];
        // cells wider than r_c by a relative margin far above the rounding of the binning
        // (x * invL * nc), so two atoms closer than r_c are never binned two cells apart
        const int c = (int)floor(L[k] / (rcut * (1.0 + 1e-9)));
        bx.nc[k] = c < 1 ? 1 : c;
        ncell *= bx.nc[k];
    }
    while (ncell > kNaMaxCells) {   // coarser grid: cells stay at least r_c wide
        int kmax = 0;
        for (int k = 1; k < 3; ++k) if (bx.nc[k] > bx.nc[kmax]) kmax = k;
        bx.nc[kmax] = bx.nc[kmax] / 2 > 0 ? bx.nc[kmax] / 2 : 1;
        ncell = (int64_t)bx.nc[0] * bx.nc[1] * bx.nc[2];
    }
    int dev = 0;
    DP_CUDA(cudaGetDevice(&dev));
    void *scratch = nullptr;
    DP_TRY(na_scratch(dev, &scratch));
    int32_t *cell_of = static_cast<int32_t *>(scratch);
    int32_t *cell_atoms = cell_of + kNaMaxAtoms;
    int32_t *cell_cnt = cell_atoms + kNaMaxAtoms;
    int32_t *cell_start = cell_cnt + kNaMaxCells + 1;
    cudaStream_t st = (cudaStream_t)stream;
    DP_CUDA(cudaMemsetAsync(d_ntrunc, 0, sizeof(unsigned long long), st));
    DP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
    if (n == 0) return DP_OK;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_na_zero<<<(unsigned)((ncell + 1 + 255) / 256), 256, 0, st>>>(ncell, cell_cnt);
    k_na_assign<<<nb, 256, 0, st>>>(n, d_coord, bx, cell_of, cell_cnt);
    k_na_scan<<<1, 1024, 0, st>>>(ncell, cell_cnt, cell_start);
    k_na_fill<<<nb, 256, 0, st>>>(n, cell_of, cell_start, cell_cnt, cell_atoms);
    k_na_format<<<(unsigned)((n + kNaWarps - 1) / kNaWarps), 32 * kNaWarps, 0, st>>>(
        n, d_coord, d_type, bx, rcut, ns, cell_of, cell_start, cell_atoms, d_nlist, d_ntrunc, d_status);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // extern "C"

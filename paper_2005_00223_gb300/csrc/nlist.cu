// Neighbor list on the device: cell-grid skin candidates (Sec. 5.1, a buffer
// region around r_c) and the per-step formatting of Sec. 4.1.1-4.1.2: keep
// r < r_c, order by neighbor type, then by floor(r * 1e8), then by index,
// keep the first sel_t of each type block and pad with -1.
//
// The paper packs (type, distance, index) into one decimal 64-bit key
// (type * 1e16 + floor(r * 1e8) * 1e6 + j) and sorts with a CUB block sort.
// Here the key is packed in binary, type:8 | floor(r * 1e8):30 | j:26, which
// orders exactly like the decimal key wherever both fit and holds indices up
// to 2^26 (the decimal key stops at 10^6, below the 1.57M-atom water box).
// Each warp owns one atom; its keys sit in shared memory and every key finds
// its slot by counting the smaller keys (keys are distinct because j is),
// which needs no sort network and no padding to a power of two.
//
// Distances use explicitly rounded FP64 operations (no contraction) in the
// order d_k = (r_j - r_i) - L_k rint((r_j - r_i) / L_k),
// r = sqrt((dx dx + dy dy) + dz dz), so the list is bit-identical to any
// IEEE implementation that uses the same order.
#include <cuda_runtime.h>

#include "dp_internal.cuh"
#include "geom.cuh"

namespace dp {
namespace {

__device__ __forceinline__ int cell_coord(double x, double invL, int nc)
{
    double f = x * invL;
    f -= floor(f);
    int c = (int)(f * nc);
    return c >= nc ? nc - 1 : (c < 0 ? 0 : c);
}

__global__ void k_pack(int64_t n, const double *__restrict__ coord, const int32_t *__restrict__ type, BoxDev bx,
                       Pos4 *__restrict__ pos, float4 *__restrict__ posf)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    pos[i] = Pos4{coord[3 * i], coord[3 * i + 1], coord[3 * i + 2], (double)type[i]};
    posf[i] = wrapped_f32(coord + 3 * i, type[i], bx);
}

// flags[1] gates the conditional (MD) rebuild: kernels return at once when
// it is zero.
__device__ __forceinline__ bool skip(const int32_t *flags, int cond) { return cond && flags[1] == 0; }

// Cell of every atom and the cell counts (atomics); the last block to finish
// (arrival counter flags[3]) turns the counts into cell starts and zeroes
// them for use as the fill cursor.  The counts are zero on entry: the
// candidate kernel of the previous build (or the allocation) leaves them so.
__global__ void __launch_bounds__(1024) k_cell_assign_scan(int64_t n, int64_t ncell, const Pos4 *__restrict__ pos,
                                                          BoxDev bx, int32_t *cell_of, int32_t *cnt,
                                                          int32_t *start, int32_t *flags, int cond)
{
    if (skip(flags, cond)) return;
    __shared__ int32_t part[1024];
    __shared__ bool last;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t i = blockIdx.x * (int64_t)nt + tid;
    if (i < n) {
        Pos4 p = pos[i];
        int cx = cell_coord(p.x, bx.invL[0], bx.nc[0]);
        int cy = cell_coord(p.y, bx.invL[1], bx.nc[1]);
        int cz = cell_coord(p.z, bx.invL[2], bx.nc[2]);
        // each frame has its own block of cells, so no candidate crosses frames
        int c = (int)(i / bx.frame_n) * bx.ncell_f + (cx * bx.nc[1] + cy) * bx.nc[2] + cz;
        if (!DP_IDX_OK(c, ncell, BS_CELL)) c = -1;
        cell_of[i] = c;
        if (c >= 0) atomicAdd(&cnt[c], 1);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(reinterpret_cast<unsigned *>(flags + 3), 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int64_t per = (ncell + nt - 1) / nt;
    const int64_t b = tid * per, e = b + per < ncell ? b + per : ncell;
    int32_t sum = 0;
    for (int64_t c = b; c < e; ++c) sum += __ldcg(cnt + c);
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int32_t v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int32_t run = part[tid] - sum;
    for (int64_t c = b; c < e; ++c) {
        int32_t v = __ldcg(cnt + c);
        start[c] = run;
        run += v;
        cnt[c] = 0;
    }
    if (tid == nt - 1) start[ncell] = part[tid];
    if (tid == 0) flags[3] = 0;
}
__global__ void k_cell_fill(int64_t n, int64_t ncell, const int32_t *cell_of, const int32_t *start, int32_t *cursor,
                            int32_t *atoms, const int32_t *flags, int cond)
{
    if (skip(flags, cond)) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    if (!DP_IDX_OK(c, ncell, BS_CELL)) return;
    const int64_t slot = start[c] + atomicAdd(&cursor[c], 1);
    if (DP_IDX_OK(slot, n, BS_CELL_SLOT)) atoms[slot] = (int32_t)i;
}

// One warp per atom: every j != i in the surrounding cells whose
// minimum-image distance, in FP32 on the wrapped FP32 coordinates, is below
// rlist + 2e-3 A.  The FP32 distance is within about 1e-4 A of the exact
// one for boxes up to 400 A (coordinates rounded to 2^-24 L), so the list
// holds every atom within
// rlist (the skin criterion needs no more) plus a few just outside, which
// the exact FP64 test of the formatting drops.
__global__ void k_candidates(int64_t n, const Pos4 *__restrict__ pos, const float4 *__restrict__ posf, BoxDev bx,
                             double rlist,
                             const int32_t *__restrict__ cell_of, const int32_t *__restrict__ start,
                             const int32_t *__restrict__ atoms, int32_t cap, int32_t *__restrict__ cand,
                             int32_t *__restrict__ cand_cnt, Pos4 *__restrict__ ref, int32_t *cell_cnt,
                             int64_t ncell, int32_t *flags, int cond)
{
    if (skip(flags, cond)) return;
    // the cell counts (the fill cursor, now complete) back to zero for the next build
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ncell; c += (int64_t)gridDim.x * blockDim.x)
        cell_cnt[c] = 0;
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const Pos4 pi = pos[i];
    const float4 pf = posf[i];
    const float Lf[3] = {(float)bx.L[0], (float)bx.L[1], (float)bx.L[2]};
    const float iLf[3] = {bx.invLf[0], bx.invLf[1], bx.invLf[2]};
    const float rpre = (float)rlist + 2e-3f;
    const int cf = cell_of[i];
    if (!DP_IDX_OK(cf, ncell, BS_CELL)) {
        if (lane == 0) cand_cnt[i] = 0;
        return;
    }
    const int fbase = (cf / bx.ncell_f) * bx.ncell_f;      // first cell of this atom's frame
    const int c = cf - fbase;
    const int c3[3] = {c / (bx.nc[1] * bx.nc[2]), (c / bx.nc[2]) % bx.nc[1], c % bx.nc[2]};
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (bx.nc[k] >= 3) { lo[k] = -1; hi[k] = 1; }
        else { lo[k] = -c3[k]; hi[k] = bx.nc[k] - 1 - c3[k]; }
    }
    int32_t count = 0;
    int32_t *row = cand + i * (int64_t)cap;
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int e = lo[2]; e <= hi[2]; ++e) {
                int x = (c3[0] + a + bx.nc[0]) % bx.nc[0];
                int y = (c3[1] + b + bx.nc[1]) % bx.nc[1];
                int z = (c3[2] + e + bx.nc[2]) % bx.nc[2];
                int cell = fbase + (x * bx.nc[1] + y) * bx.nc[2] + z;
                int s0 = start[cell], s1 = start[cell + 1];
                for (int base = s0; base < s1; base += 32) {
                    int p = base + lane;
                    bool ok = false;
                    int32_t j = -1;
                    if (p < s1) {
                        j = atoms[p];
                        if (j != i && DP_IDX_OK(j, n, BS_CAND_J)) {
                            const float4 qf = posf[j];
                            float df[3] = {qf.x - pf.x, qf.y - pf.y, qf.z - pf.z};
#pragma unroll
                            for (int k = 0; k < 3; ++k) df[k] -= Lf[k] * rintf(df[k] * iLf[k]);
                            ok = df[0] * df[0] + df[1] * df[1] + df[2] * df[2] < rpre * rpre;
                        }
                    }
                    unsigned m = __ballot_sync(0xffffffffu, ok);
                    int off = __popc(m & ((1u << lane) - 1u));
                    if (ok && count + off < cap) row[count + off] = j;
                    count += __popc(m);
                }
            }
    if (lane == 0) {
        cand_cnt[i] = count < cap ? count : cap;
        if (count > cap) atomicOr(&flags[0], kErrCapacity);
        ref[i] = pi;
    }
    if (i == 0 && lane == 0) atomicAdd(&flags[2], 1);
}

// FP32 value of a double rounded to nearest (ties away from zero) with
// integer instructions; magnitudes below 2^-126 give 0.
__device__ __forceinline__ float d2f_rn(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) + (1ull << 28);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (ex <= 0) return 0.0f;
    return __uint_as_float((unsigned)(b >> 32 & 0x80000000u) | ((unsigned)ex << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// Geometry record of a kept neighbor for the tensor-core path, from the
// exact FP64 difference d and distance r: the switching function s(r), its
// derivative ds/dr and d/r evaluated in FP64 and stored rounded to FP32 as
// (s, d/r) and (ds/dr, r).  1/r is the Newton-Raphson reciprocal in FP64
// (recip_nr: two steps from the FP32 estimate, the relative error squaring
// at each step to below the FP64 rounding), instead of the general FP64
// division; the quintic is evaluated in the factored
// form 1 - 10u^3 + 15u^4 - 6u^5 = (1 - u)^3 (1 + 3u + 6u^2), with u and
// 1 - u both taken from r directly, so neither end of the switching region
// loses precision to cancellation.  The FP32 roundings use integer
// instructions (d2f_rn), not the FP64 pipe.
__device__ __forceinline__ void env_record(const double d[3], double r, const ModelDev &md, float4 &ra, float2 &rb)
{
    const double ir = recip_nr(r);
    double s, ds;
    if (r < md.rcs) {
        s = ir;
        ds = -ir * ir;
    } else {
        const double u = (r - md.rcs) * md.inv_sw;
        const double um = (md.rcut - r) * md.inv_sw;   // 1 - u
        const double um2 = um * um;
        const double poly = um2 * um * fma(fma(6.0, u, 3.0), u, 1.0);
        const double dpoly = (-30.0 * md.inv_sw) * (u * u) * um2;
        s = poly * ir;
        ds = (dpoly - s) * ir;
    }
    ra = make_float4(d2f_rn(s), d2f_rn(d[0] * ir), d2f_rn(d[1] * ir), d2f_rn(d[2] * ir));
    rb = make_float2(d2f_rn(ds), d2f_rn(r));
}

constexpr int kRecStage = 192;   // kept neighbors per atom whose records are staged in shared memory

// One warp per atom, three stages.  (A) FP32 prefilter on wrapped FP32
// coordinates: candidates within r_c plus a margin far above its error are
// compacted into a list of (type << 26 | j).  (B) The exact FP64
// minimum-image distance on the compacted list (dense warps); keys of the
// atoms within r_c are staged in shared memory.  (C) Slot of a key = number
// of smaller keys minus the keys of lower types.  With env != NULL stage B
// also computes the geometry record of each kept neighbor for the
// tensor-core path (env_record; planes (s, d/r) at env[slot] and
// (ds/dr, r) at env + 4 n nsel); the first kRecStage are staged beside the
// keys, any later one is computed again in stage C by the same function.
// Shared memory per warp (cap2 = cap rounded up to even): keys [cap2] u64
// with the list [nc] u32 in its tail (stage B reads entry p of its
// iteration before writing key q <= p, and key q ends below every later
// entry p': 8 (q + 1) <= 4 (2 cap2 - nc + p')), then the records recA
// [kRecStage] float4 and recB [kRecStage] float2.
__global__ void k_format(int64_t n, const Pos4 *__restrict__ pos, const float4 *__restrict__ posf, BoxDev bx,
                         ModelDev md, const int32_t *__restrict__ cand, const int32_t *__restrict__ cand_cnt,
                         int32_t cap, int32_t *__restrict__ nlist, int32_t *__restrict__ nnei,
                         unsigned long long *ntrunc, float *__restrict__ env)
{
    extern __shared__ unsigned long long keys_all[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int cap2 = (cap + 1) & ~1;
    const int per_warp = cap2 + (env ? 3 * kRecStage : 0);   // 8-byte words
    unsigned long long *keys = keys_all + (int64_t)warp * per_warp;
    float4 *recA = reinterpret_cast<float4 *>(keys + cap2);
    float2 *recB = reinterpret_cast<float2 *>(keys + cap2 + 2 * kRecStage);
    const Pos4 pi = pos[i];
    const float4 pf = posf[i];
    const int32_t nc = cand_cnt[i];
    const int32_t *row = cand + i * (int64_t)cap;
    uint32_t *list = reinterpret_cast<uint32_t *>(keys) + 2 * cap2 - nc;
    const unsigned lt = (1u << lane) - 1u;
    // (A) prefilter
    int nf = 0;
    {
        const float Lf[3] = {(float)bx.L[0], (float)bx.L[1], (float)bx.L[2]};
        const float iLf[3] = {bx.invLf[0], bx.invLf[1], bx.invLf[2]};
        const float rpre = (float)md.rcut + 2e-3f;
        for (int base = 0; base < nc; base += 32) {
            const int c = base + lane;
            bool pass = false;
            uint32_t e = 0;
            if (c < nc && DP_IDX_OK(row[c], n, BS_CAND_J)) {
                const int32_t j = row[c];
                const float4 qf = posf[j];
                float df[3] = {qf.x - pf.x, qf.y - pf.y, qf.z - pf.z};
#pragma unroll
                for (int k = 0; k < 3; ++k) df[k] -= Lf[k] * rintf(df[k] * iLf[k]);
                const float r2f = df[0] * df[0] + df[1] * df[1] + df[2] * df[2];
                pass = j != i && r2f < rpre * rpre;
                e = ((uint32_t)__float_as_int(qf.w) << 26) | (uint32_t)j;
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (pass) list[nf + __popc(m & lt)] = e;
            nf += __popc(m);
        }
    }
    __syncwarp();
    // (B) exact distances on the dense list
    int nk = 0;
    for (int base = 0; base < nf; base += 32) {
        const int p = base + lane;
        const uint32_t e = p < nf ? list[p] : 0u;
        __syncwarp();
        const int32_t j = (int32_t)(e & ((1u << 26) - 1u));
        bool ok = false;
        double d[3], r = 0.0;
        if (p < nf) {
            r = min_image_r(pi, pos[j], bx, d);
            ok = r < md.rcut;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int q = nk + __popc(m & lt);
            // r >= 0: the conversion's truncation is the floor
            const unsigned long long qr = (unsigned long long)__dmul_rn(r, 1e8);
            keys[q] = ((unsigned long long)(e >> 26) << 56) | (qr << 26) | (unsigned long long)j;
            if (env && q < kRecStage) env_record(d, r, md, recA[q], recB[q]);
        }
        nk += __popc(m);
    }
    __syncwarp();
    // per-type counts
    int tcount[kMaxTypes];
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t) tcount[t] = 0;
    for (int p = lane; p < nk; p += 32) {
        int t = (int)(keys[p] >> 56);
#pragma unroll
        for (int u = 0; u < kMaxTypes; ++u) tcount[u] += (t == u);
    }
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t)
        for (int o = 16; o > 0; o >>= 1) tcount[t] += __shfl_xor_sync(0xffffffffu, tcount[t], o);
    int tstart[kMaxTypes];
    int acc = 0;
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t) { tstart[t] = acc; acc += tcount[t]; }
    int32_t *out = nlist + i * (int64_t)md.nsel;
    const int64_t plane = n * (int64_t)md.nsel;
    for (int p = lane; p < nk; p += 32) {
        unsigned long long k = keys[p];
        int rank = 0;
        for (int q = 0; q < nk; ++q) rank += keys[q] < k;
        int t = (int)(k >> 56);
        if (!DP_IDX_OK(t, md.ntypes, BS_TYPE)) continue;
        int local = rank - tstart[t];
        if (local < md.sel[t]) {
            const int slot = md.sel_off[t] + local;
            out[slot] = (int32_t)(k & ((1ull << 26) - 1));
            if (env) {
                const int64_t q = (int64_t)i * md.nsel + slot;
                float4 ra;
                float2 rb;
                if (p < kRecStage) {
                    ra = recA[p];
                    rb = recB[p];
                } else {
                    double d[3];
                    const int32_t j = (int32_t)(k & ((1ull << 26) - 1));
                    env_record(d, min_image_r(pi, pos[j], bx, d), md, ra, rb);
                }
                reinterpret_cast<float4 *>(env)[q] = ra;
                reinterpret_cast<float2 *>(env + 4 * plane)[q] = rb;
            }
        }
    }
    unsigned long long dropped = 0;
    for (int t = 0; t < md.ntypes; ++t) {
        int kept = tcount[t] < md.sel[t] ? tcount[t] : md.sel[t];
        for (int s = kept + lane; s < md.sel[t]; s += 32) out[md.sel_off[t] + s] = -1;
        if (lane == 0) nnei[i * md.ntypes + t] = kept;
        if (tcount[t] > md.sel[t]) dropped += (unsigned long long)(tcount[t] - md.sel[t]);
    }
    if (lane == 0 && dropped) atomicAdd(ntrunc, dropped);
}

inline unsigned blocks_for(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

}  // namespace

DP_BOUNDS_ACCESSOR(bounds_read_nlist)

dp_status pack_positions(dp_nlist *nl, const double *d_coord, cudaStream_t st)
{
    if (nl->n == 0) return DP_OK;
    ProfScope ps(nl->m->prof, PG_PACK, 1, st);
    k_pack<<<blocks_for(nl->n, 256), 256, 0, st>>>(nl->n, d_coord, nl->d_type, make_box(nl), (Pos4 *)nl->d_pos,
                                                   (float4 *)nl->d_posf);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

// Builds the candidate lists from d_pos.  With conditional = true every
// kernel first reads flags[1] and does nothing when no rebuild is needed.
dp_status nlist_build_device(dp_nlist *nl, cudaStream_t st, bool conditional)
{
    if (nl->n == 0) return DP_OK;
    BoxDev bx = make_box(nl);
    int cond = conditional ? 1 : 0;
    const Pos4 *pos = (const Pos4 *)nl->d_pos;
    ProfScope ps(nl->m->prof, PG_BUILD, 3, st);
    k_cell_assign_scan<<<blocks_for(nl->n, 1024), 1024, 0, st>>>(nl->n, nl->ncell, pos, bx, nl->d_cell_of,
                                                              nl->d_cell_cnt, nl->d_cell_start, nl->d_flags, cond);
    k_cell_fill<<<blocks_for(nl->n, 256), 256, 0, st>>>(nl->n, nl->ncell, nl->d_cell_of, nl->d_cell_start, nl->d_cell_cnt,
                                                       nl->d_cell_atoms, nl->d_flags, cond);
    k_candidates<<<blocks_for(nl->n * 32, 256), 256, 0, st>>>(nl->n, pos, (const float4 *)nl->d_posf, bx, nl->rlist,
                                                             nl->d_cell_of,
                                                             nl->d_cell_start, nl->d_cell_atoms, nl->cap,
                                                             nl->d_cand, nl->d_cand_cnt, (Pos4 *)nl->d_ref,
                                                             nl->d_cell_cnt, nl->ncell, nl->d_flags, cond);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

dp_status nlist_format_device(const dp_model *m, dp_nlist *nl, const double *d_coord, cudaStream_t st,
                              bool with_env)
{
    if (nl->n == 0) return DP_OK;
    if (d_coord) DP_TRY(pack_positions(nl, d_coord, st));
    if (with_env && !nl->d_env) {
        DP_CUDA(cudaStreamSynchronize(st));
        DP_CUDA(cudaMalloc((void **)&nl->d_env, sizeof(float) * 6 * (size_t)nl->n * m->dev.nsel));
    }
    BoxDev bx = make_box(nl);
    DP_CUDA(cudaMemsetAsync(nl->d_ntrunc, 0, sizeof(unsigned long long), st));
    const size_t cap2 = (size_t)((nl->cap + 1) & ~1);
    const size_t per_warp = (cap2 + (with_env ? 3 * kRecStage : 0)) * sizeof(unsigned long long);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(200 * 1024) / per_warp));
    size_t smem = (size_t)warps * per_warp;
    if (smem > 48 * 1024)
        DP_CUDA(cudaFuncSetAttribute(k_format, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(m->prof, PG_FORMAT, 1, st);
    k_format<<<blocks_for(nl->n, warps), warps * 32, smem, st>>>(
        nl->n, (const Pos4 *)nl->d_pos, (const float4 *)nl->d_posf, bx, m->dev, nl->d_cand, nl->d_cand_cnt, nl->cap,
        nl->d_nlist, nl->d_nnei, nl->d_ntrunc, with_env ? nl->d_env : nullptr);
    DP_CUDA(cudaGetLastError());
    if (centers_of(nl) < nl->n) DP_TRY(clear_ghost_rows(m, nl, st));
    return DP_OK;
}

}  // namespace dp

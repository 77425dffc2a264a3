// Wide embedding nets on the tensor cores, layer by layer (Sec. 6, "Network size": the paper sweeps
// the embedding net up to a 1024 x 2048 last-layer matrix, where its MIX-16 throughput kept rising).
//
// Nets (w, 2w, 4w) with w = 64 .. 512 (last layers 128 x 256 .. 1024 x 2048) in MIX-16 with bf16
// operands.  At these widths the activations of a 128-row tile (up to 3.5 K values per row) no longer
// fit beside the weights in shared and tensor memory, so the fused per-tile kernels of tc.cu give way
// to one tensor-core GEMM per layer with the activations in HBM; the products are large enough
// (up to 2 M multiply-adds per row for the last layer) that the GEMMs, not the activation traffic,
// bound the step.  The rows are the tiles of the MIX-16 work list (128 rows of one net, 4 chunks of
// up to 32 neighbors of one atom).  Per evaluation:
//   k_wide_l1   t1 = tanh(s W1 + b1) -> Y1 (bf16)                                   CUDA cores
//   GEMM FWD2   z2 = Y1 W2;  t2 = tanh(z2 + b2) -> T2, y2 = (y1, y1) + t2 -> Y2           tcgen05
//   GEMM FWD3   z3 = Y2 W3;  t3 -> T3, G = (y2, y2) + t3; T_q += G^T R per chunk         tcgen05
//   fitting net (tc.cu), dE/dT
//   k_wide_b1   dG = dT R, dR = dT^T G, dz3 = dG (1 - t3^2) -> DZ3                        CUDA cores
//   GEMM BWD3   dy2 = dz3 W3^T + skip(dG) -> DY2 (FP32), dz2 = dy2 (1 - t2^2) -> DZ2        tcgen05
//   GEMM BWD2   dy1 = dz2 W2^T + skip(dy2); ds += sum_k dy1 (1 - t1^2) W1_k                 tcgen05
//   k_wide_force g_ij from ds and dR, FP64 force and virial atomics                        CUDA cores
// The GEMM kernel: persistent CTAs over (tile, 256-column block) units; all 128 threads stream the
// K chunks (64 wide) of A (the tile's 128 rows) and B (the block's rows of the net's weight matrix)
// into a three-stage ring with cp.async (16-byte copies placed straight into the core-matrix layout
// of the MMA operands); one thread issues the M = 128, N = 256 MMAs into a tensor-memory accumulator;
// every thread then runs the layer's epilogue for its row.
//
// FP8 (precision DP_MIX_FP8, beyond the paper's MIX-16): the same GEMMs with e4m3 operands
// (tcgen05 kind::f8f6f4, FP32 accumulation).  The producing epilogues write an e4m3 copy of each GEMM
// input beside the bf16 values that the skips and derivatives read; the weights are quantised once per
// parameter upload with a power-of-two scale per row (its largest entry in (224, 448]), undone in the
// consuming epilogue; the backward inputs carry dE/dT scaled by a power of two 2^(3-e), e the exponent
// of its largest entry, undone (exactly) on g before the force and virial sums.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "dp_internal.cuh"
#include "tc_common.cuh"

namespace dp {

namespace {

constexpr long kWaitW = 1L << 25;   // mbarrier polls (~1 s) before a kernel gives up
constexpr int kWChunkB = 128;       // bytes of K per row in one chunk (64 bf16 or 128 e4m3)
constexpr int kWNB = 256;           // columns per unit
constexpr uint32_t kWA = 128 * kWChunkB, kWB = kWNB * kWChunkB, kWStage = kWA + kWB;
constexpr uint32_t kWGT = kWNB * 128 * 2, kWRT = 16 * 128 * 2;   // contraction operands (FWD3)

enum WideKind { WK_FWD2 = 0, WK_FWD3 = 1, WK_BWD3 = 2, WK_BWD2 = 3 };

// Stages of the copy / MMA ring and shared memory of a GEMM kind (FWD3 also holds the contraction's
// G^T and R^T).
template <int KIND>
constexpr int wide_stages() { return KIND == WK_FWD3 ? 3 : 4; }
template <int KIND>
constexpr uint32_t wide_smem() { return wide_stages<KIND>() * kWStage + (KIND == WK_FWD3 ? kWGT + kWRT : 0u); }
static_assert(wide_smem<WK_FWD3>() <= 227 * 1024 && wide_smem<WK_FWD2>() <= 227 * 1024, "shared memory");

// Byte offset of element (row, k) of a [rows][K] GEMM operand with es-byte elements stored pre-tiled:
// blocks of rows_blk rows x 128 bytes of K, block (row / rows_blk, K chunk) at
// ((row / rows_blk) nk + chunk) rows_blk 128, each block in the K-major core-matrix layout of the MMA
// operands (8 rows x 16 bytes), so that one bulk copy moves a chunk of a tile.
__host__ __device__ __forceinline__ size_t wtile_off(int64_t row, int rows_blk, int k, int K, int es)
{
    const int ke = kWChunkB / es, nk = K / ke;
    const int64_t rb = row / rows_blk;
    const int r = (int)(row - rb * rows_blk);
    const int kc = k / ke, kb = (k - kc * ke) * es;
    return ((size_t)rb * nk + kc) * (size_t)rows_blk * kWChunkB +
           (size_t)((r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

struct WideArgs {
    int E0, E1, E2;
    uint32_t img;                       // bytes of one net's weight image
    uint32_t oW2T, oW3T, oW3, oW2, oVec;   // offsets in the image
    // FP8: one net's e4m3 image (the same four matrices, then their row scales 1/s as FP32)
    uint32_t qimg, qW2T, qW3T, qW3, qW2, qS2T, qS3T, qS3, qS2;
    const unsigned char *wq;
    unsigned char *Y1q, *Y2q, *DZ3q, *DZ2q;   // e4m3 copies of the GEMM inputs
    const unsigned *gbits;              // bits of max |dE/dT| (FP8: backward scaling), or null
    const int4 *chunks;
    const int *ntiles;
    const int32_t *nnei, *nlist;
    const float4 *envA;
    const float2 *envB;
    const unsigned char *wimg;
    __nv_bfloat16 *Y1, *T2, *Y2, *T3, *DZ3, *DZ2;
    float *DY2, *DR, *DS;
    float *T;                           // [n][E2][4], accumulated (times 1, scaled by 1/sum(sel) later)
    const float *dT;                    // [n][E2][4], already scaled by 1/sum(sel)
    double *force, *atom_virial;
    int *err;
};

// The row `r` (0..127) of tile `tile`: its chunk entry, validity, geometry and neighbor.
struct WRow {
    int atom, net, j;
    bool valid;
    float4 a;   // s, u
    float2 b;   // ds/dr, r
};

__device__ __forceinline__ WRow wide_row(const ModelDev &md, const WideArgs &w, int64_t tile, int r)
{
    WRow o;
    const int4 c4 = w.chunks[tile * 4 + (r >> 5)];
    o.net = w.chunks[tile * 4].w;
    o.atom = c4.x;
    o.valid = false;
    o.j = -1;
    o.a = make_float4(0.f, 0.f, 0.f, 0.f);
    o.b = make_float2(0.f, 0.f);
    if (c4.x >= 0 && !(DP_IDX_OK(c4.x, md.n_list, BS_CHUNK_ATOM) && DP_IDX_OK(c4.y, md.ntypes, BS_TYPE)))
        o.atom = -1;   // bounds-checked build: a bad chunk is treated as padding
    if (o.atom >= 0) {
        const int k = c4.z + (r & 31);
        if (k < w.nnei[(int64_t)c4.x * md.ntypes + c4.y]) {
            const int64_t slot = (int64_t)c4.x * md.nsel + md.sel_off[c4.y] + k;
            o.j = w.nlist[slot];
            o.valid = DP_IDX_OK(o.j, md.n_list, BS_NLIST_J);
            if (o.valid) {
                o.a = w.envA[slot];
                o.b = w.envB[slot];
            }
        }
    }
    return o;
}


__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unbf2(uint32_t v) { return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&v)); }

// 16 bf16 values as floats: 8 at p and 8 at p + step (step = 8: contiguous; 64: the next 16-byte
// segment of a pre-tiled operand).
__device__ __forceinline__ void ld16(const __nv_bfloat16 *p, float *v, int step = 8)
{
    const uint4 a = *reinterpret_cast<const uint4 *>(p), b = *reinterpret_cast<const uint4 *>(p + step);
    const uint32_t q[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 f = unbf2(q[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void st16(__nv_bfloat16 *p, const float *v, int step = 8)
{
    *reinterpret_cast<uint4 *>(p) = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(p + step) =
        make_uint4(bf2(v[8], v[9]), bf2(v[10], v[11]), bf2(v[12], v[13]), bf2(v[14], v[15]));
}

// Element (row, k) of a pre-tiled activation (128-row blocks) of width K.
__device__ __forceinline__ __nv_bfloat16 *tb16(__nv_bfloat16 *base, int64_t row, int k, int K)
{
    return reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(base) + wtile_off(row, 128, k, K, 2));
}
__device__ __forceinline__ unsigned char *tq8(unsigned char *base, int64_t row, int k, int K)
{
    return base + wtile_off(row, 128, k, K, 1);
}

// 2^(3-e) and its inverse for e the exponent of max |dE/dT| (bits of a non-negative float); 1, 1 when
// there is nothing to scale.
__device__ __forceinline__ void grad_scale(const unsigned *bits, float &s, float &inv)
{
    s = inv = 1.f;
    if (bits == nullptr) return;
    const unsigned b = *bits;
    const int e = (int)((b >> 23) & 0xffu) - 127 - 3;
    if (b != 0u && e > -120 && e < 120) {
        s = __int_as_float((127 - e) << 23);
        inv = __int_as_float((127 + e) << 23);
    }
}

// 16 floats as e4m3 (saturating) at p (16-byte aligned).
__device__ __forceinline__ void st16q(unsigned char *p, const float *v)
{
    uint32_t q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i], v[4 * i + 1]), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t b = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i + 2], v[4 * i + 3]), __NV_SATFINITE, __NV_E4M3);
        q[i] = (uint32_t)a | ((uint32_t)b << 16);
    }
    *reinterpret_cast<uint4 *>(p) = make_uint4(q[0], q[1], q[2], q[3]);
}

__device__ __forceinline__ uint16_t q2(float a, float b)
{
    return (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
}

template <int KIND, int Q>
__global__ void __launch_bounds__(128, 1) k_wide_gemm(ModelDev md, WideArgs w)
{
    constexpr int S = wide_stages<KIND>();
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_done, bar_c;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // A [rows][K] (the layer input, pre-tiled in 128-row blocks) and B [N][K] (the net's weight matrix,
    // pre-tiled in blocks of min(N, 256) rows)
    const int K = KIND == WK_FWD2 ? w.E0 : KIND == WK_FWD3 ? w.E1 : KIND == WK_BWD3 ? w.E2 : w.E1;
    const int N = KIND == WK_FWD2 ? w.E1 : KIND == WK_FWD3 ? w.E2 : KIND == WK_BWD3 ? w.E1 : w.E0;
    constexpr int ES = Q ? 1 : 2;          // bytes per operand element
    const unsigned char *A = Q ? (KIND == WK_FWD2 ? w.Y1q : KIND == WK_FWD3 ? w.Y2q : KIND == WK_BWD3 ? w.DZ3q : w.DZ2q)
                               : reinterpret_cast<const unsigned char *>(
                                     KIND == WK_FWD2 ? w.Y1 : KIND == WK_FWD3 ? w.Y2 : KIND == WK_BWD3 ? w.DZ3 : w.DZ2);
    const uint32_t oB = Q ? (KIND == WK_FWD2 ? w.qW2T : KIND == WK_FWD3 ? w.qW3T : KIND == WK_BWD3 ? w.qW3 : w.qW2)
                          : (KIND == WK_FWD2 ? w.oW2T : KIND == WK_FWD3 ? w.oW3T : KIND == WK_BWD3 ? w.oW3 : w.oW2);
    const uint32_t oS = KIND == WK_FWD2 ? w.qS2T : KIND == WK_FWD3 ? w.qS3T : KIND == WK_BWD3 ? w.qS3 : w.qS2;
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&bar_full[q], 1);
            tc::mbar_init(&bar_empty[q], 1);
        }
        tc::mbar_init(&bar_done, 1);
        tc::mbar_init(&bar_c, 1);
        tc::mbar_init_fence();
        s_fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    // copy / MMA ring state, kept by thread 0: phases, and which stages hold a copy or an MMA whose
    // completion has not been waited for
    uint32_t ph_f[S], ph_e[S], ph_d = 0, ph_c = 0;
    bool loaded[S], busy[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
        ph_f[q] = ph_e[q] = 0;
        loaded[q] = busy[q] = false;
    }
    const int nk = K * ES / kWChunkB, nbr = N < kWNB ? N : kWNB, nblk = N / nbr;
    const int64_t ntiles = *w.ntiles, units = ntiles * nblk;
    bool dead = false;
    auto wait_all = [&](uint64_t *bar, uint32_t &ph) {
        const bool ok = tc::mbar_wait(bar, ph, kWaitW);
        ph ^= 1;
        return __syncthreads_and(ok) != 0;
    };
    // kind::f16 bf16 x bf16, or kind::f8f6f4 e4m3 x e4m3 (format codes 0), FP32 accumulator
    const uint32_t id = Q ? ((1u << 4) | ((uint32_t)(nbr >> 3) << 17) | ((uint32_t)(128 >> 4) << 24))
                          : tc::idesc_f16(128, nbr, 1);
    const uint32_t bbytes = (uint32_t)nbr * kWChunkB;
    for (int64_t u = blockIdx.x; u < units && !dead; u += gridDim.x) {
        const int64_t tile = u / nblk;
        const int nb = (int)(u - tile * nblk);
        const int nbc = nbr;
        const int net = w.chunks[tile * 4].w;
        const unsigned char *Ab = A + (size_t)tile * nk * kWA;
        const unsigned char *Bb = (Q ? w.wq + (size_t)net * w.qimg : w.wimg + (size_t)net * w.img) + oB +
                                  (size_t)nb * nk * bbytes;
        if (tid == 0) {
            // producer and MMA issuer: chunk c's A and B blocks by two bulk copies into stage c % S;
            // the copies run S - 1 chunks ahead of the MMAs
            bool ok = true;
            auto stage_free = [&](int q) {
                if (busy[q]) {
                    busy[q] = false;
                    if (!tc::mbar_wait(&bar_empty[q], ph_e[q], kWaitW)) return false;
                    ph_e[q] ^= 1;
                }
                return true;
            };
            auto issue = [&](int c) {
                const int q = c % S;
                unsigned char *sa = smem + q * kWStage;
                tc::mbar_expect_tx(&bar_full[q], kWA + bbytes);
                tc::bulk_g2s(sa, Ab + (size_t)c * kWA, kWA, &bar_full[q]);
                tc::bulk_g2s(sa + kWA, Bb + (size_t)c * bbytes, bbytes, &bar_full[q]);
                loaded[q] = true;
            };
            for (int c = 0; c < S - 1 && c < nk && ok; ++c) {
                ok = stage_free(c % S);
                if (ok) issue(c);
            }
            for (int c = 0; c < nk && ok; ++c) {
                const int q = c % S;
                loaded[q] = false;
                if (!tc::mbar_wait(&bar_full[q], ph_f[q], kWaitW)) { ok = false; break; }
                ph_f[q] ^= 1;
                tc::fence_after_sync();
                const uint32_t sa = tc::smem_u32(smem + q * kWStage), sb = sa + kWA;
                // one MMA step covers 32 bytes of K (16 bf16 or 32 e4m3): two core matrices
                for (int ks = 0; ks < kWChunkB / 32; ++ks) {
                    const uint64_t ad = tc::smem_desc(sa + ks * 256, 128, 1024);
                    const uint64_t bd = tc::smem_desc(sb + ks * 256, 128, 1024);
                    const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                    if (Q)
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(id), "r"(acc));
                    else
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(id), "r"(acc));
                }
                tc::mma_commit(&bar_empty[q]);
                busy[q] = true;
                const int cn = c + S - 1;   // its stage held chunk c - 1, whose MMAs were issued before
                if (cn < nk) {
                    if (!stage_free(cn % S)) { ok = false; break; }
                    issue(cn);
                }
            }
            if (ok) tc::mma_commit(&bar_done);   // arrives once every MMA of the unit has completed
            else s_fail = 1;
        }
        // every thread: the accumulator is complete (or thread 0 gave up: then no arrival comes)
        const bool done_ok = tc::mbar_wait(&bar_done, ph_d, s_fail ? 1 : kWaitW);
        ph_d ^= 1;
        if (!__syncthreads_and(done_ok && !s_fail)) { dead = true; break; }
        tc::fence_after_sync();
        // ---------------------------------------------------------------- epilogues (thread = row)
        const WRow row = wide_row(md, w, tile, tid);
        const int64_t gr = tile * 128 + tid;
        const float *vec = reinterpret_cast<const float *>(w.wimg + (size_t)net * w.img + w.oVec);
        const float *W1 = vec, *b1 = vec + w.E0, *b2 = vec + 2 * w.E0, *b3 = b2 + w.E1;
        // FP8: the accumulator of column n carries the weight row's scale s_n; inv_s[n] = 1 / s_n
        const float *inv_s = Q ? reinterpret_cast<const float *>(w.wq + (size_t)net * w.qimg + oS) + nb * kWNB : nullptr;
        auto acc16 = [&](int c0, float *z) {
            tc::tmem_ld16(taddr + c0, z);
            tc::tmem_ld_wait();
            if (Q) {
#pragma unroll
                for (int i = 0; i < 16; ++i) z[i] *= inv_s[c0 + i];
            }
        };
        float gs = 1.f, gi = 1.f;   // FP8: the backward scaling of dE/dT (DZ3, DY2, DZ2 carry it)
        if (Q) grad_scale(w.gbits, gs, gi);
        if constexpr (KIND == WK_FWD2) {
            for (int c0 = 0; c0 < nbc; c0 += 16) {
                const int k0 = nb * kWNB + c0;
                float z[16], y1[16], t[16], y[16];
                acc16(c0, z);
                ld16(tb16(w.Y1, gr, k0 % w.E0, w.E0), y1, 64);   // skip: y2 = (y1, y1) + t2
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    t[i] = tc::tanh_fast(z[i] + b2[k0 + i]);
                    y[i] = y1[i] + t[i];
                }
                st16(w.T2 + gr * w.E1 + k0, t);
                st16(tb16(w.Y2, gr, k0, w.E1), y, 64);
                if (Q) st16q(tq8(w.Y2q, gr, k0, w.E1), y);
            }
        } else if constexpr (KIND == WK_FWD3) {
            unsigned char *GT = smem + S * kWStage, *RT = GT + kWGT;
            {
                const float s = row.valid ? row.a.x : 0.f;
                float r8[8] = {s, s * row.a.y, s * row.a.z, s * row.a.w, 0.f, 0.f, 0.f, 0.f};
                if (!row.valid) r8[1] = r8[2] = r8[3] = 0.f;
                *reinterpret_cast<uint4 *>(RT + tc::mnmaj_off(0, tid, 16)) =
                    make_uint4(bf2(r8[0], r8[1]), bf2(r8[2], r8[3]), 0u, 0u);
                *reinterpret_cast<uint4 *>(RT + tc::mnmaj_off(8, tid, 16)) = make_uint4(0u, 0u, 0u, 0u);
            }
            for (int c0 = 0; c0 < nbc; c0 += 16) {
                const int m0 = nb * kWNB + c0;
                float z[16], y2[16], t[16], g[16];
                acc16(c0, z);
                ld16(tb16(w.Y2, gr, m0 % w.E1, w.E1), y2, 64);   // skip: G = (y2, y2) + t3
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    t[i] = tc::tanh_fast(z[i] + b3[m0 + i]);
                    g[i] = y2[i] + t[i];
                }
                st16(w.T3 + gr * w.E2 + m0, t);
                *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0, tid, kWNB)) =
                    make_uint4(bf2(g[0], g[1]), bf2(g[2], g[3]), bf2(g[4], g[5]), bf2(g[6], g[7]));
                *reinterpret_cast<uint4 *>(GT + tc::mnmaj_off(c0 + 8, tid, kWNB)) =
                    make_uint4(bf2(g[8], g[9]), bf2(g[10], g[11]), bf2(g[12], g[13]), bf2(g[14], g[15]));
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            // T_q[m][c] = sum over chunk q's 32 rows of G[row][m] R[row][c], for the block's channels in
            // halves of 128 (tensor-memory columns 256 + 16 (4 h + q))
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t idT = tc::idesc_f16_major(128, 16, 1, 1, 1);
                for (int h = 0; h < nbc / 128; ++h)
                    for (int q = 0; q < 4; ++q)
                        tc::mma_kloop_mn(tmem + 256 + 16 * (4 * h + q), tc::smem_u32(GT) + 2048 * h, kWNB,
                                         tc::smem_u32(RT), 16, 32 * q, 32, idT, false);
                tc::mma_commit(&bar_c);
            }
            if (!wait_all(&bar_c, ph_c)) { dead = true; break; }
            tc::fence_after_sync();
            for (int h = 0; h < nbc / 128; ++h) {
                const int m = nb * kWNB + 128 * h + warp * 32 + lane;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[4];
                    tc::tmem_ld4(taddr + 256 + 16 * (4 * h + q), v);
                    tc::tmem_ld_wait();
                    const int atom = w.chunks[tile * 4 + q].x;
                    if (atom >= 0) {
                        float *Tm = w.T + ((int64_t)atom * w.E2 + m) * 4;
#pragma unroll
                        for (int c = 0; c < 4; ++c) atomicAdd(Tm + c, v[c]);
                    }
                }
            }
        } else if constexpr (KIND == WK_BWD3) {
            const float s = row.valid ? row.a.x : 0.f;
            const float R[4] = {s, s * row.a.y, s * row.a.z, s * row.a.w};
            const float4 *dTa = reinterpret_cast<const float4 *>(w.dT + (int64_t)(row.atom >= 0 ? row.atom : 0) * w.E2 * 4);
            for (int c0 = 0; c0 < nbc; c0 += 16) {
                const int k0 = nb * kWNB + c0;
                float z[16], t2[16], dz[16];
                acc16(c0, z);
                ld16(w.T2 + gr * w.E1 + k0, t2);
                float dy[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    // skip of layer 3: dG[k] + dG[k + E1], dG[m] = dT[m] . R
                    float sk = 0.f;
                    if (row.valid) {
                        const float4 a = dTa[k0 + i], b = dTa[k0 + i + w.E1];
                        sk = a.x * R[0] + a.y * R[1] + a.z * R[2] + a.w * R[3] + b.x * R[0] + b.y * R[1] +
                             b.z * R[2] + b.w * R[3];
                    }
                    dy[i] = z[i] + sk * gs;
                    dz[i] = dy[i] * (1.f - t2[i] * t2[i]);
                }
                if (Q) st16q(tq8(w.DZ2q, gr, k0, w.E1), dz);
                else st16(tb16(w.DZ2, gr, k0, w.E1), dz, 64);
                float4 *d4 = reinterpret_cast<float4 *>(w.DY2 + gr * w.E1 + k0);
#pragma unroll
                for (int i = 0; i < 4; ++i) d4[i] = make_float4(dy[4 * i], dy[4 * i + 1], dy[4 * i + 2], dy[4 * i + 3]);
            }
        } else {   // WK_BWD2
            const float s = row.valid ? row.a.x : 0.f;
            float ds = 0.f;
            for (int c0 = 0; c0 < nbc; c0 += 16) {
                const int k0 = nb * kWNB + c0;
                float z[16];
                acc16(c0, z);
                const float4 *a4 = reinterpret_cast<const float4 *>(w.DY2 + gr * w.E1 + k0);
                const float4 *b4 = reinterpret_cast<const float4 *>(w.DY2 + gr * w.E1 + k0 + w.E0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 a = a4[i], b = b4[i];
                    const float sk[4] = {a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};   // skip of layer 2
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k = k0 + 4 * i + e;
                        const float t1 = tc::tanh_fast(fmaf(s, W1[k], b1[k]));
                        ds = fmaf((z[4 * i + e] + sk[e]) * (1.f - t1 * t1), W1[k], ds);
                    }
                }
            }
            if (row.valid) atomicAdd(w.DS + gr, ds);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (dead && tid == 0) {
        // a wait gave up: flag it, then wait (bounded again) for this CTA's copies and products in
        // flight before the tensor memory is freed
        atomicOr(w.err, 1);
        for (int q = 0; q < S; ++q) {
            if (loaded[q]) tc::mbar_wait(&bar_full[q], ph_f[q], kWaitW);
            if (busy[q]) tc::mbar_wait(&bar_empty[q], ph_e[q], kWaitW);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Layer 1 (1 -> E0, plain since E0 >= 64): one warp per row, lanes over the outputs.
template <int Q>
__global__ void k_wide_l1(ModelDev md, WideArgs w, int64_t max_rows)
{
    const int64_t gr = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gr >= max_rows || gr >= (int64_t)(*w.ntiles) * 128) return;
    const WRow row = wide_row(md, w, gr >> 7, (int)(gr & 127));
    const float *vec = reinterpret_cast<const float *>(w.wimg + (size_t)row.net * w.img + w.oVec);
    const float s = row.valid ? row.a.x : 0.f;
    for (int k = 2 * lane; k < w.E0; k += 64) {
        const float t0 = tc::tanh_fast(fmaf(s, vec[k], vec[w.E0 + k]));
        const float t1 = tc::tanh_fast(fmaf(s, vec[k + 1], vec[w.E0 + k + 1]));
        *reinterpret_cast<uint32_t *>(tb16(w.Y1, gr, k, w.E0)) = bf2(t0, t1);
        if (Q) *reinterpret_cast<uint16_t *>(tq8(w.Y1q, gr, k, w.E0)) = q2(t0, t1);
    }
}

// Start of the backward pass per row (one warp, lanes over the channels m):
//   dG = dT R, G = (y2, y2) + t3, dR = dT^T G (warp sum), dz3 = dG (1 - t3^2) -> DZ3.
template <int Q>
__global__ void k_wide_b1(ModelDev md, WideArgs w, int64_t max_rows)
{
    const int64_t gr = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gr >= max_rows || gr >= (int64_t)(*w.ntiles) * 128) return;
    const WRow row = wide_row(md, w, gr >> 7, (int)(gr & 127));
    float dR[4] = {0.f, 0.f, 0.f, 0.f};
    const float s = row.valid ? row.a.x : 0.f;
    const float R[4] = {s, s * row.a.y, s * row.a.z, s * row.a.w};
    const float4 *dTa = reinterpret_cast<const float4 *>(w.dT + (int64_t)(row.atom >= 0 ? row.atom : 0) * w.E2 * 4);
    float gs = 1.f, gi = 1.f;
    if (Q) grad_scale(w.gbits, gs, gi);
    for (int m = 2 * lane; m < w.E2; m += 64) {
        const float2 t3 = unbf2(*reinterpret_cast<const uint32_t *>(w.T3 + gr * w.E2 + m));
        const float2 y2 = unbf2(*reinterpret_cast<const uint32_t *>(tb16(w.Y2, gr, m % w.E1, w.E1)));
        float dz[2] = {0.f, 0.f};
        if (row.valid) {
            const float tt[2] = {t3.x, t3.y}, yy[2] = {y2.x, y2.y};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float4 d = dTa[m + e];
                const float G = yy[e] + tt[e];
                dR[0] = fmaf(d.x, G, dR[0]);
                dR[1] = fmaf(d.y, G, dR[1]);
                dR[2] = fmaf(d.z, G, dR[2]);
                dR[3] = fmaf(d.w, G, dR[3]);
                const float dG = d.x * R[0] + d.y * R[1] + d.z * R[2] + d.w * R[3];
                dz[e] = dG * (1.f - tt[e] * tt[e]) * gs;
            }
        }
        if (Q) *reinterpret_cast<uint16_t *>(tq8(w.DZ3q, gr, m, w.E2)) = q2(dz[0], dz[1]);
        else *reinterpret_cast<uint32_t *>(tb16(w.DZ3, gr, m, w.E2)) = bf2(dz[0], dz[1]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        for (int o = 16; o > 0; o >>= 1) dR[c] += __shfl_xor_sync(0xffffffffu, dR[c], o);
        dR[c] *= gs;
    }
    if (lane == 0) *reinterpret_cast<float4 *>(w.DR + 4 * gr) = make_float4(dR[0], dR[1], dR[2], dR[3]);
}

// g_ij = (dR/dr_ij)^T dE/dR from ds and dR (R = (s, s u), u = d/r):
//   g = u (dR0 s' + (s' - s/r) u.dR') + (s/r) dR'; F_j -= g, F_i += g, W_i -= d (x) g (FP64 atomics);
// one block per tile, a warp per chunk (one atom).
template <int Q>
__global__ void __launch_bounds__(128) k_wide_force(ModelDev md, WideArgs w)
{
    const int64_t tile = blockIdx.x;
    if (tile >= *w.ntiles) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const WRow row = wide_row(md, w, tile, tid);
    const int64_t gr = tile * 128 + tid;
    float gv[3] = {0.f, 0.f, 0.f}, vir[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) vir[q] = 0.f;
    if (row.valid) {
        const float4 dr = *reinterpret_cast<const float4 *>(w.DR + 4 * gr);
        const float u[3] = {row.a.y, row.a.z, row.a.w}, dsdr = row.b.x, r = row.b.y, s = row.a.x;
        const float sr = s / r;
        const float dR0 = dr.x + w.DS[gr];
        const float ud = u[0] * dr.y + u[1] * dr.z + u[2] * dr.w;
        const float cu = fmaf(dsdr - sr, ud, dR0 * dsdr);
        const float dRp[3] = {dr.y, dr.z, dr.w};
        float gs = 1.f, gi = 1.f;
        if (Q) grad_scale(w.gbits, gs, gi);
#pragma unroll
        for (int k = 0; k < 3; ++k) gv[k] = fmaf(cu, u[k], sr * dRp[k]) * gi;
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(&w.force[3 * (int64_t)row.j + k], -(double)gv[k]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) vir[3 * a + b] = -(r * u[a]) * gv[b];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) gv[k] += __shfl_xor_sync(0xffffffffu, gv[k], o);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        for (int o = 16; o > 0; o >>= 1) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], o);
    const int atom = row.atom;
    if (atom >= 0) {
        if (lane < 3) {
            const float v = lane == 0 ? gv[0] : (lane == 1 ? gv[1] : gv[2]);
            atomicAdd(&w.force[3 * (int64_t)atom + lane], (double)v);
        }
        if (lane < 9) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) v = (q == lane) ? vir[q] : v;
            atomicAdd(&w.atom_virial[9 * (int64_t)atom + lane], (double)v);
        }
    }
}

// *out = bits of max |x| over x [n] (non-negative floats order like their bits); *out zeroed first.
__global__ void k_wide_absmax(int64_t n, const float *__restrict__ x, unsigned *out)
{
    unsigned m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned b = __float_as_uint(fabsf(x[i]));
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

struct WideLayout {
    int E0, E1, E2;
    uint32_t oW2T, oW3T, oW3, oW2, oVec, img;
    uint32_t qW2T, qW3T, qW3, qW2, qS2T, qS3T, qS3, qS2, qimg;   // FP8 image: e4m3 matrices, then 1 / row scale
};

WideLayout wide_layout(const ModelDev &md)
{
    WideLayout L;
    L.E0 = md.emb.wout[0];
    L.E1 = md.emb.wout[1];
    L.E2 = md.emb.wout[2];
    L.oW2T = 0;
    L.oW3T = L.oW2T + (uint32_t)L.E1 * L.E0 * 2;
    L.oW3 = L.oW3T + (uint32_t)L.E2 * L.E1 * 2;
    L.oW2 = L.oW3 + (uint32_t)L.E1 * L.E2 * 2;
    L.oVec = L.oW2 + (uint32_t)L.E0 * L.E1 * 2;
    L.img = L.oVec + (uint32_t)(2 * L.E0 + L.E1 + L.E2) * 4;
    L.qW2T = 0;
    L.qW3T = L.qW2T + (uint32_t)L.E1 * L.E0;
    L.qW3 = L.qW3T + (uint32_t)L.E2 * L.E1;
    L.qW2 = L.qW3 + (uint32_t)L.E1 * L.E2;
    L.qS2T = L.qW2 + (uint32_t)L.E0 * L.E1;
    L.qS3T = L.qS2T + (uint32_t)L.E1 * 4;
    L.qS3 = L.qS3T + (uint32_t)L.E2 * 4;
    L.qS2 = L.qS3 + (uint32_t)L.E1 * 4;
    L.qimg = L.qS2 + (uint32_t)L.E0 * 4;
    return L;
}

// rows x cols FP64 matrix M (element (r, c) = M[r * rs + c * cs]) as e4m3 rows scaled by a power of
// two s_r (largest |entry| of the row times s_r in (224, 448]), pre-tiled like the bf16 matrices;
// inv[r] = 1 / s_r.
void quant_rows(const double *M, int rows, int cols, int64_t rs, int64_t cs, unsigned char *q, float *inv)
{
    const int rb = rows < kWNB ? rows : kWNB;
    for (int r = 0; r < rows; ++r) {
        double mx = 0.0;
        for (int c = 0; c < cols; ++c) mx = fmax(mx, fabs(M[r * rs + c * cs]));
        const int e = mx > 0.0 ? (int)floor(log2(448.0 / mx)) : 0;
        const double s = ldexp(1.0, e);
        inv[r] = (float)ldexp(1.0, -e);
        for (int c = 0; c < cols; ++c) {
            const __nv_fp8_e4m3 v((float)(M[r * rs + c * cs] * s));
            q[wtile_off(r, rb, c, cols, 1)] = (unsigned char)v.__x;
        }
    }
}

}  // namespace

// Nets (w, 2w, 4w), w = 64, 128, 256, 512: the wide path of this file.
bool embed_is_wide(int n_embed, const int *e)
{
    if (n_embed != 3) return false;
    const int b = e[0];
    return (b == 64 || b == 128 || b == 256 || b == 512) && e[1] == 2 * b && e[2] == 4 * b;
}

dp_status pack_wide_weights(dp_model *m)
{
    const ModelDev &md = m->dev;
    const WideLayout L = wide_layout(md);
    const int nn = m->ntypes * m->ntypes;
    std::vector<unsigned char> img((size_t)nn * L.img, 0);
    auto bf = [](double v) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        uint16_t u;
        memcpy(&u, &h, 2);
        return u;
    };
    for (int q = 0; q < nn; ++q) {
        const double *p = m->h_params.data() + md.emb_base + q * md.emb.size;
        unsigned char *o = img.data() + (size_t)q * L.img;
        // element (r, c) of a rows x cols matrix at its pre-tiled place (blocks of min(rows, 256) rows)
        auto put = [&](uint32_t off, int rows, int cols, int r, int c, double v) {
            const uint16_t b = bf(v);
            memcpy(o + off + wtile_off(r, rows < kWNB ? rows : kWNB, c, cols, 2), &b, 2);
        };
        const double *W1 = p + md.emb.W[0], *b1 = p + md.emb.b[0], *W2 = p + md.emb.W[1], *b2 = p + md.emb.b[1];
        const double *W3 = p + md.emb.W[2], *b3 = p + md.emb.b[2];
        for (int a = 0; a < L.E0; ++a)
            for (int b = 0; b < L.E1; ++b) {
                put(L.oW2, L.E0, L.E1, a, b, W2[(size_t)a * L.E1 + b]);    // W2 [E0][E1]
                put(L.oW2T, L.E1, L.E0, b, a, W2[(size_t)a * L.E1 + b]);   // W2^T [E1][E0]
            }
        for (int a = 0; a < L.E1; ++a)
            for (int b = 0; b < L.E2; ++b) {
                put(L.oW3, L.E1, L.E2, a, b, W3[(size_t)a * L.E2 + b]);
                put(L.oW3T, L.E2, L.E1, b, a, W3[(size_t)a * L.E2 + b]);
            }
        float *vec = reinterpret_cast<float *>(o + L.oVec);
        for (int k = 0; k < L.E0; ++k) {
            vec[k] = (float)W1[k];
            vec[L.E0 + k] = (float)b1[k];
        }
        for (int k = 0; k < L.E1; ++k) vec[2 * L.E0 + k] = (float)b2[k];
        for (int k = 0; k < L.E2; ++k) vec[2 * L.E0 + L.E1 + k] = (float)b3[k];
    }
    if (!m->d_wide) DP_CUDA(cudaMalloc((void **)&m->d_wide, img.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_wide, img.data(), img.size(), cudaMemcpyHostToDevice, m->stream));
    // the e4m3 image of the same matrices (rows of W2^T, W3^T, W3, W2)
    std::vector<unsigned char> qi((size_t)nn * L.qimg, 0);
    for (int q = 0; q < nn; ++q) {
        const double *p = m->h_params.data() + md.emb_base + q * md.emb.size;
        unsigned char *o = qi.data() + (size_t)q * L.qimg;
        const double *W2 = p + md.emb.W[1], *W3 = p + md.emb.W[2];
        quant_rows(W2, L.E1, L.E0, 1, L.E1, o + L.qW2T, reinterpret_cast<float *>(o + L.qS2T));   // W2^T
        quant_rows(W3, L.E2, L.E1, 1, L.E2, o + L.qW3T, reinterpret_cast<float *>(o + L.qS3T));   // W3^T
        quant_rows(W3, L.E1, L.E2, L.E2, 1, o + L.qW3, reinterpret_cast<float *>(o + L.qS3));     // W3
        quant_rows(W2, L.E0, L.E1, L.E1, 1, o + L.qW2, reinterpret_cast<float *>(o + L.qS2));     // W2
    }
    if (!m->d_wide_q) DP_CUDA(cudaMalloc((void **)&m->d_wide_q, qi.size()));
    DP_CUDA(cudaMemcpyAsync(m->d_wide_q, qi.data(), qi.size(), cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return DP_OK;
}

namespace {

template <int Q>
dp_status run_wide(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                   double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    const ModelDev &md = m->dev;
    const WideLayout L = wide_layout(md);
    if (Q && L.E0 % 128 != 0) {   // e4m3 K chunks are 128 wide
        set_error("DP_MIX_FP8 needs embedding nets (w, 2w, 4w) with w >= 128");
        return DP_ERR_UNSUPPORTED;
    }
    const int64_t n = nl->n;
    const int nn = md.ntypes * md.ntypes;
    const int64_t max_chunks = n * md.chunks_per_atom + 4 * nn + 4;
    const int64_t max_rows = max_chunks * 32;   // 4 chunks of 32 rows per tile
    if (!nl->d_env) {
        set_error("wide embedding path needs the neighbor geometry of the formatting kernel");
        return DP_ERR_ARG;
    }
    if (!m->d_wide) DP_TRY(pack_wide_weights(m));
    size_t need = 0;
    auto sz = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    sz(sizeof(float) * 4 * md.m1 * n);
    sz(sizeof(float) * 4 * md.m1 * n);
    sz(sizeof(int4) * max_chunks);
    sz(sizeof(int) * 4);
    sz(sizeof(unsigned) * 4);
    sz(chunks_batch_scratch(md, n));
    sz(2 * (size_t)max_rows * L.E0);        // Y1
    sz(2 * (size_t)max_rows * L.E1 * 3);    // T2, Y2, DZ2
    sz(2 * (size_t)max_rows * L.E2 * 2);    // T3, DZ3
    sz(4 * (size_t)max_rows * L.E1);        // DY2
    sz(4 * (size_t)max_rows * 5);           // DR, DS
    if (Q) {
        sz((size_t)max_rows * L.E0);        // e4m3 Y1, Y2, DZ3, DZ2
        sz((size_t)max_rows * L.E1 * 2);
        sz((size_t)max_rows * L.E2);
    }
    DP_TRY(ensure_workspace(m, need));
    char *wp = m->ws;
    auto carve = [&](size_t bytes) {
        char *p = wp;
        wp += (bytes + 255) & ~(size_t)255;
        return p;
    };
    WideArgs a{};
    a.E0 = L.E0;
    a.E1 = L.E1;
    a.E2 = L.E2;
    a.img = L.img;
    a.oW2T = L.oW2T;
    a.oW3T = L.oW3T;
    a.oW3 = L.oW3;
    a.oW2 = L.oW2;
    a.oVec = L.oVec;
    a.qimg = L.qimg;
    a.qW2T = L.qW2T;
    a.qW3T = L.qW3T;
    a.qW3 = L.qW3;
    a.qW2 = L.qW2;
    a.qS2T = L.qS2T;
    a.qS3T = L.qS3T;
    a.qS3 = L.qS3;
    a.qS2 = L.qS2;
    a.wq = m->d_wide_q;
    a.T = (float *)carve(sizeof(float) * 4 * md.m1 * n);
    float *dT = (float *)carve(sizeof(float) * 4 * md.m1 * n);
    a.dT = dT;
    int4 *chunks = (int4 *)carve(sizeof(int4) * max_chunks);
    int *cnt = (int *)carve(sizeof(int) * 4);
    unsigned *gbits = (unsigned *)carve(sizeof(unsigned) * 4);
    a.gbits = Q ? gbits : nullptr;
    char *scratch = carve(chunks_batch_scratch(md, n));
    a.Y1 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E0);
    a.T2 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E1);
    a.Y2 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E1);
    a.DZ2 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E1);
    a.T3 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E2);
    a.DZ3 = (__nv_bfloat16 *)carve(2 * (size_t)max_rows * L.E2);
    a.DY2 = (float *)carve(4 * (size_t)max_rows * L.E1);
    a.DR = (float *)carve(4 * (size_t)max_rows * 4);
    a.DS = (float *)carve(4 * (size_t)max_rows);
    if (Q) {
        a.Y1q = (unsigned char *)carve((size_t)max_rows * L.E0);
        a.Y2q = (unsigned char *)carve((size_t)max_rows * L.E1);
        a.DZ2q = (unsigned char *)carve((size_t)max_rows * L.E1);
        a.DZ3q = (unsigned char *)carve((size_t)max_rows * L.E2);
    }
    a.chunks = chunks;
    a.ntiles = cnt;
    a.nnei = nl->d_nnei;
    a.nlist = nl->d_nlist;
    a.envA = reinterpret_cast<const float4 *>(nl->d_env);
    a.envB = reinterpret_cast<const float2 *>(nl->d_env + 4 * (size_t)n * md.nsel);
    a.wimg = m->d_wide;
    a.force = d_force;
    a.atom_virial = d_atom_virial;
    a.err = m->d_err;
    int nsm = 0;
    DP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    DP_CUDA(cudaMemsetAsync(a.T, 0, sizeof(float) * 4 * md.m1 * n, st));
    DP_CUDA(cudaMemsetAsync(a.DS, 0, 4 * (size_t)max_rows, st));
    DP_CUDA(cudaMemsetAsync(d_force, 0, sizeof(double) * 3 * n, st));
    DP_CUDA(cudaMemsetAsync(d_atom_virial, 0, sizeof(double) * 9 * n, st));
    {
        ProfScope ps(m->prof, PG_CHUNKS, 3, st);
        DP_TRY(build_chunks_batch(m, nl, 0, n, chunks, nullptr, cnt, scratch, st));
    }
    DP_CUDA(cudaFuncSetAttribute(k_wide_gemm<WK_FWD2, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<WK_FWD2>()));
    DP_CUDA(cudaFuncSetAttribute(k_wide_gemm<WK_FWD3, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<WK_FWD3>()));
    DP_CUDA(cudaFuncSetAttribute(k_wide_gemm<WK_BWD3, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<WK_BWD3>()));
    DP_CUDA(cudaFuncSetAttribute(k_wide_gemm<WK_BWD2, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wide_smem<WK_BWD2>()));
    const unsigned rb = (unsigned)((max_rows * 32 + 255) / 256);
    {
        ProfScope ps(m->prof, PG_EMBED_FWD, 3, st);
        k_wide_l1<Q><<<rb, 256, 0, st>>>(md, a, max_rows);
        k_wide_gemm<WK_FWD2, Q><<<nsm, 128, wide_smem<WK_FWD2>(), st>>>(md, a);
        k_wide_gemm<WK_FWD3, Q><<<nsm, 128, wide_smem<WK_FWD3>(), st>>>(md, a);
    }
    DP_CUDA(cudaGetLastError());
    DP_TRY(fit_mix16_bf16(m, nl, a.T, d_atom_energy, dT, st));
    if (Q) {   // the scale of dE/dT for the e4m3 backward operands
        ProfScope ps(m->prof, PG_DESC, 1, st);
        DP_CUDA(cudaMemsetAsync(gbits, 0, sizeof(unsigned), st));
        k_wide_absmax<<<(unsigned)(2 * nsm), 256, 0, st>>>((int64_t)4 * md.m1 * n, dT, gbits);
        DP_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(m->prof, PG_EMBED_BWD, 4, st);
        k_wide_b1<Q><<<rb, 256, 0, st>>>(md, a, max_rows);
        k_wide_gemm<WK_BWD3, Q><<<nsm, 128, wide_smem<WK_BWD3>(), st>>>(md, a);
        k_wide_gemm<WK_BWD2, Q><<<nsm, 128, wide_smem<WK_BWD2>(), st>>>(md, a);
        k_wide_force<Q><<<(unsigned)(max_chunks / 4 + 1), 128, 0, st>>>(md, a);
    }
    DP_CUDA(cudaGetLastError());
    ProfScope ps(m->prof, PG_REDUCE, 1, st);
    return reduce_energy_virial(d_atom_energy, d_atom_virial, centers_of(nl), d_energy, d_virial, m->d_red, st);
}

}  // namespace

DP_BOUNDS_ACCESSOR(bounds_read_wide)

dp_status compute_wide(dp_model *m, dp_nlist *nl, int fp8, double *d_energy, double *d_atom_energy, double *d_force,
                       double *d_virial, double *d_atom_virial, cudaStream_t st)
{
    return fp8 ? run_wide<1>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st)
               : run_wide<0>(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
}

}  // namespace dp

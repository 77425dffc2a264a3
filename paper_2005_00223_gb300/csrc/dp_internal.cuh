// Internal declarations of libdp: handle structs, device-side model view,
// kernel launchers.  Not part of the public C-ABI (include/dp.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dp.h"
#include "bounds.cuh"

namespace dp {

constexpr int kMaxTypes = 8;
constexpr int kMaxEmbed = 4;
constexpr int kMaxFit = 4;
constexpr int kMaxM1 = 128;
constexpr int kMaxFitWidth = 256;
constexpr int kChunk = 32;          // neighbors per chunk (one per lane)

// Device-side error word bits (ModelDev::err / NlistDev::flags).
constexpr int kErrCapacity = 1;

void set_error(const char *fmt, ...);
dp_status cuda_fail(cudaError_t e, const char *what);

#define DP_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return dp::cuda_fail(e_, #call); \
    } while (0)

#define DP_TRY(call)                        \
    do {                                    \
        dp_status s_ = (call);              \
        if (s_ != DP_OK) return s_;         \
    } while (0)

// Offsets of one net's layers inside the flat parameter vector, relative to
// the start of the net.  The transposed copy (pT) uses the same offsets with
// each W (fan_in x fan_out) stored as W^T (fan_out x fan_in).
struct NetLayout {
    int n_layers;
    int win[kMaxFit + 1];
    int wout[kMaxFit + 1];
    int64_t W[kMaxFit + 1];
    int64_t b[kMaxFit + 1];
    int64_t size;
};

// Everything a kernel needs to know about the model (passed by value).
struct ModelDev {
    int ntypes, nsel, m1, m2, n_embed, n_fit, desc_dim;
    int sel[kMaxTypes], sel_off[kMaxTypes + 1];
    int chunk_off[kMaxTypes + 1];   // chunk index where each type block starts
    int chunks_per_atom;            // sum_t ceil(sel_t / 32)
    double rcut, rcs;
    double inv_sw;                  // 1 / (rcut - rcs)
    double inv_nsel;
    NetLayout emb;                  // layout of every embedding net (all alike)
    NetLayout fit;                  // layout of every fitting net, incl. the output layer
    int64_t emb_base;               // 0
    int64_t fit_base;               // ntypes^2 * emb.size
    const double *p;                // FP64 parameters (flat order)
    const double *pT;               // FP64 parameters with every W transposed
    const float *p32;               // FP32 copy (flat order)
    const float *pT32;              // FP32 transposed copy
    int act_stride;                 // doubles stored per neighbor for the backward pass
    // Test of the bounded waits (dp_test_starve_wait): which wait is starved (0 = none) and the
    // polls after which that one wait gives up.  Every other wait keeps its default limit.
    int wait_test;
    long long wait_short;
    // Deterministic mode (dp_model_set_deterministic): the force and per-atom virial scatters add
    // into these fixed-point limb arrays (3 limbs per value) instead of FP64 atomics; null: FP64
    // atomics.  Set for the duration of one evaluation.
    unsigned long long *fx, *fxv;
    // Atoms of the list being evaluated (centers and ghosts), set at the start of each evaluation:
    // the limit of the neighbor indexes that the bounds-checked build checks.
    int64_t n_list;
};

// Order-independent accumulation of v: an exact fixed-point number with 64 fractional bits, its
// integer part and two 32-bit fraction limbs each summed by an integer atomic (integer sums
// commute, so the total does not depend on the order of the additions); bits of v below 2^-64 are
// dropped (truncated towards minus infinity).  |v| must stay below 2^62.
__device__ __forceinline__ void fx_add(unsigned long long *l, double v)
{
    const double ip = floor(v);
    const double r = (v - ip) * 4294967296.0;   // the fraction times 2^32: exact
    const double hi = floor(r);
    const double lo = floor((r - hi) * 4294967296.0);
    atomicAdd(l, (unsigned long long)(long long)ip);
    atomicAdd(l + 1, (unsigned long long)hi);
    atomicAdd(l + 2, (unsigned long long)lo);
}

// acc[idx] += v: into the limbs lx (deterministic mode) or by an FP64 atomic.
__device__ __forceinline__ void acc_add(unsigned long long *lx, double *acc, int64_t idx, double v)
{
    if (lx) fx_add(lx + 3 * idx, v);
    else atomicAdd(acc + idx, v);
}

// Waits that dp_test_starve_wait can starve.
enum WaitTest { WT_NONE = 0, WT_EMBED_FWD_WEIGHTS = 1 };

// Kernel launch groups timed by the tracing calls (dp_profile_*).
enum ProfGroup {
    PG_BUILD = 0,     // cell grid and skin candidates (3 kernels)
    PG_FORMAT,        // neighbor-list formatting
    PG_PACK,          // coordinate packing
    PG_EMBED_FWD,     // environment rows + embedding net + descriptor
    PG_FIT,           // fitting net forward + input gradient
    PG_EMBED_BWD,     // embedding backward + force / virial scatter
    PG_REDUCE,        // energy / virial reduction
    PG_MD,            // integrator kernels (kick, drift, displacement check)
    PG_THERMO,        // thermo rows
    PG_CHECK,         // non-finite scans
    PG_CHUNKS,        // tensor-core work list
    PG_DESC,          // descriptor D and dE/dT between the embedding passes
    PG_GRAD,          // parameter-gradient kernels
    PG_OPT,           // optimizer step
    PG_EMBED_FWD_L2,  // FP64 split-product route: the widest embedding layer (forward, with its epilogue)
    PG_EMBED_BWD_L2,  // FP64 split-product route: its input gradient (with its epilogue)
    PG_COUNT
};

struct Prof {
    struct Rec {
        int g, n;
        cudaEvent_t a, b;
    };
    bool on = false;
    uint32_t mask = ~0u;          // groups that are timed while on
    bool capturing = false;       // scopes record graph event nodes into captured
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    std::vector<Rec> captured;
    int64_t launches[PG_COUNT] = {0};
    double ms[PG_COUNT] = {0};
    cudaEvent_t get();
    void drain();
    void clear();
    ~Prof();
};

// Brackets a group of n kernel launches on stream st with events when on.
struct ProfScope {
    Prof *p;
    int g, n;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(Prof *p_, int g_, int n_, cudaStream_t st_);
    ~ProfScope();
};

}  // namespace dp

struct dp_model {
    int device = 0;
    int32_t ntypes = 0;
    double rcut = 0, rcs = 0;
    int32_t sel[dp::kMaxTypes] = {0};
    int32_t n_embed = 0, embed[dp::kMaxEmbed] = {0}, m2 = 0, n_fit = 0, fit[dp::kMaxFit] = {0};
    int64_t nparams = 0;
    std::vector<double> h_params;
    double *d_params = nullptr, *d_paramsT = nullptr;
    float *d_params32 = nullptr, *d_paramsT32 = nullptr;
    dp::ModelDev dev{};
    cudaStream_t stream = nullptr;      // stream in use (own_stream unless the caller set one)
    cudaStream_t own_stream = nullptr;
    dp::Prof *prof = nullptr;
    // device workspace (grown on demand, freed at destroy)
    char *ws = nullptr;
    size_t ws_bytes = 0;
    double *d_scalar = nullptr;       // [16] pinned-reduction target on device
    int64_t batch_atoms = 0;          // atoms per batch (0 = derived from the workspace budget)
    // per-atom scratch for the host-pointer calls: E_i [n], W_i [9n], F [3n], coord [3n], scalars [16]
    double *d_aux = nullptr;
    int64_t aux_n = -1;
    int32_t *d_flag = nullptr;        // [4] non-finite flag and spare
    double *d_red = nullptr;          // [kRedParts][10] partial sums of the energy / virial reduction
    int32_t *d_err = nullptr;         // [4] device error word (bounded waits that gave up)
    unsigned char *d_tcw = nullptr;   // packed fp16 and bf16 embedding weights for the tensor cores
    unsigned char *d_tcfit = nullptr; // packed fp16 and bf16 fitting weights for the tensor cores
    unsigned char *d_tcw_x3 = nullptr; // packed split-bf16 (hi, lo) embedding weights (DP_MIX_BF16X3)
    unsigned char *d_tcfit_x3 = nullptr; // packed split-bf16 fitting weights (DP_MIX_BF16X3)
    unsigned char *d_fitcl[3] = {nullptr, nullptr, nullptr};   // cluster fitting kernel: fp16, bf16, split-bf16 images
    unsigned char *d_wide = nullptr;  // bf16 weights of the wide embedding nets (W2^T, W3^T, W3, W2, vectors)
    unsigned char *d_wide_q = nullptr;   // their e4m3 copies with row scales (DP_MIX_FP8)
    void *d_ozw = nullptr;            // fp16 digits of the first fitting layer's weights (FP64 products on the tensor cores)
    int *d_oze = nullptr;             // their row scales
    bool oz_stale = true;             // digits older than the parameters
    void *d_ozw_fit = nullptr;        // fp16 digits of the other fitting layers' weights, per type
    int *d_oze_fit = nullptr;         // their row scales
    bool oz_fit_stale = true;
    void *d_ozw_emb = nullptr;        // fp16 digits of the hidden embedding layers' weights, per net
    int *d_oze_emb = nullptr;         // their row scales
    bool oz_emb_stale = true;
    uint32_t tc_img_bytes = 0;
    double *d_train = nullptr;        // Adam moments m, v [n_params] each
    double *d_tscr = nullptr;         // scratch of the training calls
    int64_t tscr_n = -1;
    bool params_dirty = false;        // device parameters newer than the host copy
    uint64_t epoch = 0;               // bumped whenever a buffer or parameter that launches capture changes
    int32_t deterministic = 0;        // fixed-point force / virial scatters on the FP64 and MIX-32 routes
};

struct dp_nlist {
    const dp_model *m = nullptr;
    int64_t n = 0;
    int64_t n_centers = -1;           // atoms [0, n_centers) are centers; the rest are ghosts (-1: all)
    double rcut = 0, skin = 0, rlist = 0;
    int32_t cap = 0;
    double L[3] = {0, 0, 0};
    int nc[3] = {1, 1, 1};
    int64_t ncell = 0;                // cells of all frames: nframes x ncell_frame
    int64_t ncell_frame = 0;          // nc[0] nc[1] nc[2]
    int32_t nframes = 1;              // independent configurations of frame_n atoms each (atoms f*frame_n..)
    int64_t frame_n = 0;
    int32_t *d_type = nullptr;
    int32_t *d_cand = nullptr;        // [n][cap]
    int32_t *d_cand_cnt = nullptr;    // [n]
    double *d_ref = nullptr;          // [n][4] positions at the last build
    int32_t *d_cell_of = nullptr;     // [n]
    int32_t *d_cell_cnt = nullptr;    // [ncell + 1]
    int32_t *d_cell_start = nullptr;  // [ncell + 1]
    int32_t *d_cell_atoms = nullptr;  // [n]
    int32_t *d_nlist = nullptr;       // [n][nsel]
    int32_t *d_nnei = nullptr;        // [n][ntypes] real neighbors kept per type
    unsigned long long *d_ntrunc = nullptr;
    int32_t *d_flags = nullptr;       // [0] error bits, [1] rebuild needed, [2] rebuild count, [3] block arrivals of a build
    double *d_pos = nullptr;          // [n][4] packed current coordinates (x, y, z, type)
    float *d_posf = nullptr;          // [n][4] FP32 copy of the coordinates (prefilter of the formatting)
    float *d_env = nullptr;           // tensor-core geometry (lazy): [n][nsel] float4 (s, u), then [n][nsel] float2 (ds/dr, r)
    double *d_coord = nullptr;        // [n][3] staging for host-pointer calls
    int32_t *d_order = nullptr;       // [n] atom indices sorted by type (stable)
    std::vector<int64_t> type_count, type_off;
    // dp_compute with host arrays as one captured graph (H2D of the coordinates from pinned staging,
    // the evaluation, D2H of the results into it), replayed while its key holds
    cudaGraph_t cgraph = nullptr;
    cudaGraphExec_t cgraph_exec = nullptr;
    dp_precision cgraph_prec = DP_FP64;
    uint64_t cgraph_epoch = 0;
    std::string cgraph_env;
    int cgraph_direct = 0;            // direct calls with the current key (capture after the first)
    double *h_io = nullptr;           // pinned: coord [3n], F [3n], E_i [n], E and W [10], two int32 flags
    unsigned long long *d_fx = nullptr;   // deterministic mode: limbs of F [3n][3], then of W_i [9n][3]
    size_t fx_cap = 0;
};

struct dp_md_state {
    dp_model *m = nullptr;
    dp_nlist *nl = nullptr;
    int64_t n = 0;
    double *d_x = nullptr;            // [n][3]
    double *d_v = nullptr;            // [n][3]
    double *d_f = nullptr;            // [n][3]
    double *d_minv = nullptr;         // [ntypes] 9.648533212e-3 / m
    double *d_mass = nullptr;         // [ntypes]
    double *d_e = nullptr;            // [n] atom energies
    double *d_scal = nullptr;         // [16]: E, W[9], KE, ...
    double *d_thermo = nullptr;       // ring of thermo rows
    unsigned long long *d_steps = nullptr;   // steps since the fixed-interval rebuilds were switched on
    int32_t rebuild_every = 0;        // > 0: also rebuild the skin list every that many steps
    int64_t thermo_cap = 0;
    double box[9] = {0};
    int64_t step = 0;
    bool forces_valid = false;
    dp_precision forces_prec = DP_FP64;
    // one MD step captured as a CUDA graph, replayed while its key holds
    struct GraphScope {
        int g, n;
        cudaGraphNode_t na, nb;       // event-record nodes of the scope's two events
        cudaEvent_t ea, eb;           // the events recorded at capture
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<GraphScope> graph_scopes;
    dp_precision graph_prec = DP_FP64;
    double graph_dt = 0.0;
    uint64_t graph_epoch = 0;
    bool graph_prof = false;
    uint32_t graph_mask = 0;
    std::string graph_env;
};

namespace dp {

// Routing switches read from the environment (part of the key of a captured graph).
std::string route_env();

// Launchers (return DP_OK or an error after recording a message).
dp_status nlist_build_device(dp_nlist *nl, cudaStream_t st, bool conditional);
dp_status nlist_format_device(const dp_model *m, dp_nlist *nl, const double *d_coord, cudaStream_t st,
                              bool with_env = false);
dp_status pack_positions(dp_nlist *nl, const double *d_coord, cudaStream_t st);
dp_status compute_fp64(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                       double *d_virial, double *d_atom_virial, cudaStream_t st);
constexpr int kRedParts = 256;        // blocks of the first reduction stage
dp_status reduce_energy_virial(const double *d_atom_energy, const double *d_atom_virial, int64_t n,
                               double *d_energy, double *d_virial, double *d_scratch, cudaStream_t st);
dp_status ensure_workspace(dp_model *m, size_t bytes);
dp_status check_nonfinite(const double *d_x, int64_t n, int32_t *d_flag, cudaStream_t st);
bool embed_shape_supported(int n_embed, const int *e);
size_t fp64_bytes_per_atom(const ModelDev &md);
dp_status compute_mix32(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                        double *d_virial, double *d_atom_virial, cudaStream_t st);
// Full evaluation on device data: pack, format, compute in the requested precision.  reformat = false
// reuses the formatted list (and geometry records) of the evaluation just before it on the same
// coordinates; the caller guarantees it was formatted for the same r_c, types and sel (format_shared).
dp_status compute_device(dp_model *m, dp_nlist *nl, const double *d_coord, dp_precision prec, double *d_energy,
                         double *d_atom_energy, double *d_force, double *d_virial, double *d_atom_virial,
                         cudaStream_t st, bool reformat = true);
// True when a list formatted for model a in precision pa also serves model b in precision pb: the same
// r_c, r_cs, number of types and sel, and geometry records present if pb reads them.
bool format_shared(const dp_model *a, dp_precision pa, const dp_model *b, dp_precision pb);
dp_status check_box(const double box[9], double rcut, double L[3]);
dp_status pack_tc_weights(dp_model *m);
dp_status compute_mix16(dp_model *m, dp_nlist *nl, int bf16, double *d_energy, double *d_atom_energy,
                        double *d_force, double *d_virial, double *d_atom_virial, cudaStream_t st);
// FP32 fitting net over all atoms (type-sorted positions): D, dD [n][desc], E_i FP64.
dp_status fit_f32(dp_model *m, dp_nlist *nl, const float *D, float *dD, double *d_atom_energy, cudaStream_t st);
dp_status pack_x3_weights(dp_model *m);
// Marks an evaluation already dispatched (compute_device).
constexpr dp_precision DP_PRECISION_DONE = (dp_precision)1000;
// Wide embedding nets (w, 2w, 4w), w = 64 .. 512, layer by layer on the tensor cores (wide.cu).
bool embed_is_wide(int n_embed, const int *e);
dp_status pack_wide_weights(dp_model *m);
dp_status compute_wide(dp_model *m, dp_nlist *nl, int fp8, double *d_energy, double *d_atom_energy, double *d_force,
                       double *d_virial, double *d_atom_virial, cudaStream_t st);
// The MIX-16 fitting net (bf16 operands) of tc.cu, for the wide path.
dp_status fit_mix16_bf16(dp_model *m, dp_nlist *nl, const float *T, double *E_atom, float *dT, cudaStream_t st);
// Fitting net + descriptor adjoint on the tensor cores with a tile split over a thread-block cluster
// (fit_cluster.cu); mode 0 fp16, 1 bf16, 2 split bf16.  DP_ERR_UNSUPPORTED (no error text) for shapes
// it does not cover, which the single-CTA kernels then take.  DP_FIT_ONE_CTA selects those always.
bool fit_cluster_enabled();
dp_status fit_cluster(dp_model *m, dp_nlist *nl, int mode, const float *T, double *E_atom, float *dT,
                      cudaStream_t st);
dp_status pack_fit_cluster_weights(dp_model *m);   // repacks the images already in use
// out[i] = the value of limbs l[3i .. 3i + 2] (fx_add), i < count, in FP64.
dp_status fx_finish(int64_t count, const unsigned long long *l, double *out, cudaStream_t st);
// Ghost atoms of a spatial decomposition (dp_nlist_set_centers): their list rows are cleared after each
// format, so they appear only as neighbors.
dp_status clear_ghost_rows(const dp_model *m, dp_nlist *nl, cudaStream_t st);
void nlist_graph_drop(dp_nlist *nl);   // drops the captured host-array evaluation of a list
inline int64_t centers_of(const dp_nlist *nl) { return nl->n_centers >= 0 ? nl->n_centers : nl->n; }
dp_status compute_mix_x3(dp_model *m, dp_nlist *nl, double *d_energy, double *d_atom_energy, double *d_force,
                         double *d_virial, double *d_atom_virial, cudaStream_t st);
dp_status param_grad_device(dp_model *m, dp_nlist *nl, const double *d_v, const double *d_ab, dp_precision prec,
                            double *d_E_atom, double *d_Ed_atom, double *d_grad, cudaStream_t st);
// Per frame f of a list (frames of frame_n atoms): v = F - F_ref, the frame's
// energy from the per-atom energies d_Ei, d_ab = [beta, alpha_0 .. alpha_{F-1}],
// d_lf [F] scratch; d_loss += the loss summed over the frames in frame order.
dp_status loss_terms_device(int64_t n, int64_t frame_n, const double *d_F, const double *d_F_ref,
                            const double *d_Ei, const double *d_E_ref, double p_e, double p_f, double *d_v,
                            double *d_ab, double *d_lf, double *d_loss, cudaStream_t st);
dp_status refresh_params_device(dp_model *m, cudaStream_t st);
// FP64 products on the tensor cores (ozaki.cu): digits of the rows of an
// FP64 matrix, and C = A B^T (+ bias) from the digits of A and of B, or
// C += A B^T with accumulate (one more FP64 rounding: a product over a long
// K is taken as a sum of products over K ranges, each with its own scales).
template <int S, int BETA>
dp_status oz_split(const double *X, int64_t ldx, int64_t rows, int64_t rows_pad, int K, int K_pad, int TR, int KC,
                   __half *dig, int *ex, cudaStream_t st);
template <int S, int BETA, int NC, int KC>
dp_status oz_gemm(const dp_model *m, int64_t M, int N, int K, const __half *dA, const int *eA, int64_t M_pad,
                  const __half *dB, const int *eB, const double *bias, double *C, int64_t ldc, cudaStream_t st,
                  bool accumulate = false);
// Work list of the 32-neighbor chunks of positions [p0, p0 + nb) in tiles of
// 4 chunks of one net (tc.cu): entry {atom, batch position, first slot,
// net}, firstc [nb][ntypes], the tile count on the device.
size_t chunks_batch_scratch(const ModelDev &md, int64_t nb);
dp_status build_chunks_batch(dp_model *m, dp_nlist *nl, int64_t p0, int64_t nb, int4 *chunks, int *firstc,
                             int *ntiles, char *scratch, cudaStream_t st);
// FP64 embedding forward with its widest layer as a split product on the
// tensor cores (oz_embed.cu): shapes, scratch per batch, weight digits, and
// the forward of a batch (T, D, the stored activations).
struct BoxDev;
bool oz_emb_ok(const ModelDev &md);
size_t oz_emb_bytes(const ModelDev &md, int64_t nb);
dp_status oz_emb_refresh(dp_model *m, cudaStream_t st);
dp_status oz_emb_fwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t p0, int64_t nb, double *T, double *D,
                     double *act, char *scratch, cudaStream_t st);
// The backward of the batch whose forward ran last on the same scratch:
// forces (added) and per-atom virials (added; zeroed by the caller).
dp_status oz_emb_bwd(dp_model *m, dp_nlist *nl, const BoxDev &bx, int64_t nb, const double *T, const double *dD,
                     const double *act, double *force, double *atom_virial, char *scratch, cudaStream_t st);
// The fitting net's hidden layers after the first as split products
// (oz_fit.cu): shape check, weight digits, scratch for `count` atoms, and the
// chain from z1 to E_i and dz1.
bool oz_fit_chain_ok(const ModelDev &md);
dp_status oz_fit_chain_refresh(dp_model *m, cudaStream_t st);
size_t oz_fit_chain_bytes(const ModelDev &md, int64_t count);
dp_status oz_fit_chain(dp_model *m, int ti, const int32_t *order, int64_t pos_begin, int64_t count,
                       const double *z1, double *dz1, double *E_atom, char *scratch, cudaStream_t st);
// Per-atom scratch of the model: E_i [n] at d_aux, W_i [9n] right after it.
dp_status ensure_aux(dp_model *m, int64_t n);
dp_status nlist_create_internal(const dp_model *m, int64_t n, const int32_t *type, const double box[9], double rcut,
                                double skin, int32_t cand_cap, dp_nlist **out, int32_t nframes = 1);

}  // namespace dp

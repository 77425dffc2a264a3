/*
 * libdp — DeepPot-SE (se_a) energy, force and virial evaluation and
 * velocity-Verlet NVE on one NVIDIA GB300 (sm_103a).
 *
 * Paper: Jia et al., "Pushing the limit of molecular dynamics with ab initio
 * accuracy to 100 million atoms with machine learning", SC20.
 *
 * The method (Sec. 2, Fig. 1): the total energy is E = sum_i E_i; E_i is the
 * output of a per-type fitting net applied to a descriptor D_i built from the
 * environment matrix R_i of atom i's neighbors within r_c and from a
 * per-neighbor embedding net; forces are F = -dE/dr and the virial
 * W = -sum_ij d_ij (x) dE_i/dd_ij.  Sec. 4.1.1-4.1.2 fix the neighbor list
 * layout (sorted by type, then distance; padded per type to sel; nearest
 * kept on overflow); Sec. 4.1.3 the MIX-32 / MIX-16 precision schemes;
 * Sec. 5.1 the velocity-Verlet MD loop with a skin neighbor list.
 *
 * Conventions for every call
 *   - Units: A, eV, amu, fs; FP64 row-major arrays; type ids 0..ntypes-1.
 *   - The caller owns every array it passes.  The library owns the opaque
 *     handles and their device memory, which is allocated at create time or
 *     when a call needs more room than before (never in steady state).
 *   - Every call returns a dp_status and never aborts.  On error the output
 *     arrays are left untouched (the *_dev calls excepted: device outputs may
 *     be partly written) and dp_last_error() describes the failure.
 *   - Boxes: orthorhombic only in this version (off-diagonal entries must be
 *     zero) and r_c < L/2 along every axis, else DP_ERR_BOX.
 *   - Calls on one model (or on handles made from it) must not overlap: the
 *     model's device workspace is shared by them.
 *   - Host-pointer calls run on the library's own stream and return after
 *     their results are in host memory.  *_dev calls take device pointers
 *     and a cudaStream_t (passed as void*; NULL = the legacy default stream)
 *     and return after enqueueing; their outputs are valid once that stream
 *     reaches the work.
 */
#ifndef DP_H
#define DP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DP_OK = 0,
    DP_ERR_ARG = -1,         /* invalid argument (NULL pointer, bad size, ...) */
    DP_ERR_CUDA = -2,        /* a CUDA runtime call or kernel launch failed */
    DP_ERR_OOM = -3,         /* device or host allocation failed */
    DP_ERR_BOX = -4,         /* non-orthorhombic box, or r_c >= L/2 */
    DP_ERR_CAPACITY = -5,    /* a candidate list exceeded its capacity; build again with more room */
    DP_ERR_TIMEOUT = -6,     /* a bounded device wait expired */
    DP_ERR_NONFINITE = -7,   /* a NaN or Inf appeared in energies or forces */
    DP_ERR_UNSUPPORTED = -8  /* model shape or precision not supported by this build */
} dp_status;

/* Precision schemes (Sec. 4.1.3).  Coordinates, minimum-image differences,
 * the environment matrix, force/virial accumulation and the integrator are
 * FP64 in every scheme.
 *   DP_FP64      every step in FP64.
 *   DP_MIX32     nets in FP32 (MIX-32).
 *   DP_MIX_BF16  MIX-16 with bf16 operands on the tensor cores, FP32
 *                accumulation; first embedding layer, tanh and the last
 *                fitting layer in FP32.
 *   DP_MIX_FP16  the same with fp16 operands.
 *   DP_MIX_BF16X3  the embedding net's products on the tensor cores with
 *                FP32-class accuracy: every operand split into two bf16
 *                terms (hi = bf16(x), lo = bf16(x - hi)) and each product
 *                taken as hi hi + hi lo + lo hi (three MMAs, FP32
 *                accumulation), tanh in FP32 (tanhf); descriptor and
 *                fitting net in FP32 on the CUDA cores (as DP_MIX32).
 *   DP_MIX_FP8   the wide embedding nets (w, 2w, 4w), w = 128 .. 512, with
 *                the products of layers 2 and 3 and their input gradients
 *                on e4m3 operands (tcgen05 kind::f8f6f4, FP32 accumulation;
 *                weights quantised with a power-of-two scale per row, the
 *                backward operands with one power-of-two scale); all else as
 *                DP_MIX_BF16.  Other nets: DP_ERR_UNSUPPORTED. */
typedef enum { DP_FP64 = 0, DP_MIX32 = 1, DP_MIX_BF16 = 2, DP_MIX_FP16 = 3, DP_MIX_BF16X3 = 4,
               DP_MIX_FP8 = 5 } dp_precision;

/* Model hyper-parameters (Sec. 2, Sec. 5.1).
 *   ntypes       number of atom types (1..8)
 *   rcut         cut-off radius r_c (A)
 *   rcut_smth    start r_cs of the switching region (A), 0 < r_cs < r_c
 *   sel          [ntypes] neighbors kept per type (padding size per block)
 *   n_embed      number of embedding layers (1..4); embed[n_embed] widths
 *                after the 1-wide input; the last width is M1 (<= 128)
 *   axis_neuron  M2 <= M1, leading embedding channels used in D
 *   n_fit        number of hidden fitting layers (1..4); fit[n_fit] widths
 *                (<= 256); the output layer is linear, width 1
 * One embedding net per (center type, neighbor type) pair, one fitting net
 * per center type.  Each hidden layer is y = act(x W + b) with tanh and the
 * skip rule of Fig. 1(e)-(g): y = x + t when widths are equal, (x, x) + t
 * when the width doubles, t otherwise.  The switching function is 1/r below
 * r_cs and (1/r)(u^3(-6u^2 + 15u - 10) + 1), u = (r - r_cs)/(r_c - r_cs),
 * up to r_c: twice continuously differentiable as Sec. 2 requires. */
typedef struct {
    int32_t ntypes;
    double rcut;
    double rcut_smth;
    const int32_t *sel;
    int32_t n_embed;
    const int32_t *embed;
    int32_t axis_neuron;
    int32_t n_fit;
    const int32_t *fit;
} dp_model_config;

typedef struct dp_model dp_model;
typedef struct dp_nlist dp_nlist;
typedef struct dp_md_state dp_md_state;

/* Human-readable name of a status, and the calling thread's last error
 * message (empty string when none).  Both strings are owned by the library. */
const char *dp_status_string(dp_status st);
const char *dp_last_error(void);

/* ---------------------------------------------------------------- model */

/* Create a model on the current CUDA device with seeded weights: every
 * weight and bias entry is drawn N(0, 1/fan_in) from SplitMix64(seed)
 * uniforms (top 53 bits) through Box-Muller, cosine branch first, in the
 * flat parameter order of dp_model_get_params.  The config is copied.
 * Errors: DP_ERR_ARG (NULL / invalid shape), DP_ERR_UNSUPPORTED (shape
 * beyond the limits above), DP_ERR_CUDA, DP_ERR_OOM. */
dp_status dp_model_create(const dp_model_config *cfg, uint64_t seed, dp_model **out);

/* Number of parameters.  Flat order: embedding nets for (ti, tj) in
 * row-major pair order, then fitting nets per ti; inside a net every layer
 * as W (fan_in x fan_out, row-major) followed by b (fan_out). */
dp_status dp_model_n_params(const dp_model *m, int64_t *n);

/* Copy the FP64 parameters out (n must equal dp_model_n_params). */
dp_status dp_model_get_params(const dp_model *m, double *flat, int64_t n);

/* Replace the parameters (FP64 master copy; lower-precision copies are
 * re-derived).  n must equal dp_model_n_params, else DP_ERR_ARG. */
dp_status dp_model_set_params(dp_model *m, const double *flat, int64_t n);

void dp_model_destroy(dp_model *m);

/* Run this model's host-pointer calls and MD steps on `stream` (a
 * cudaStream_t passed as void*) instead of the library's own stream; NULL
 * switches back.  The caller keeps the stream alive while the model uses it. */
dp_status dp_model_set_stream(dp_model *m, void *stream);

/* Deterministic force accumulation (on = 1; 0 = off, the default).  The FP64
 * and MIX-32 evaluations then add the pair terms g_ij into the forces
 * (F_i = -dE/dx_i of Sec. 2.2 as sums over the neighbor pairs) and the per-chunk virial
 * terms as exact fixed-point numbers with 64 fractional bits in 64-bit integer
 * limbs, whose sums do not depend on the order in which the GPU's threads add
 * them: forces, energies and virials of an evaluation are then the same bit
 * for bit from run to run, and an MD run resumed from a checkpoint
 * (dp_md_state_save / _load) follows the uninterrupted one bit for bit.
 * Contributions are truncated below 2^-64 (in the units of the force), and
 * each force must stay below 2^62 in magnitude.  Costs three integer atomics
 * per contribution where one FP64 atomic was used, and 288 bytes of device
 * memory per atom of the neighbor list.  The tensor-core precisions
 * (DP_MIX_BF16, _FP16, _BF16X3, _FP8) accumulate the descriptor with FP32
 * atomics and stay reproducible only to their rounding; the flag does not
 * change them.  DP_ERR_ARG for a NULL model or on outside {0, 1}. */
dp_status dp_model_set_deterministic(dp_model *m, int32_t on);

/* ------------------------------------------------------------- tracing */

/* Kernel timing: while enabled, every kernel launch group of this model is
 * bracketed by CUDA events on its stream (a few microseconds per group).
 * dp_profile_enable(m, on) turns it on or off and clears the counters.
 * dp_profile_read waits for the model's stream and returns, for one group,
 * the kernels launched and their summed device time (ms) since the clear.
 * dp_profile_group_name returns the group's name, NULL past the last. */
dp_status dp_profile_enable(dp_model *m, int32_t on);
/* dp_profile_select(m, mask) restricts the timing to the groups whose bit
 * (1 << group) is set in mask (all groups by default), so that a timed run
 * carries the events of the groups it reports and no others.  The mask
 * outlives dp_profile_enable; counters already taken are kept. */
dp_status dp_profile_select(dp_model *m, uint32_t group_mask);
dp_status dp_profile_read(dp_model *m, int32_t group, int64_t *launches, double *ms);
const char *dp_profile_group_name(int32_t group);

/* ---------------------------------------------------------- neighbor list */

/* Build a skin neighbor list (Sec. 5.1: a buffer region around r_c):
 * candidates are every j != i with minimum-image distance < rcut + skin,
 * found with a cell grid of edge >= rcut + skin.  rcut must be >= the
 * model's r_c.  cand_cap is the per-atom candidate capacity (0 = derived
 * from the density).  The list is then formatted once at these coordinates
 * (see dp_nlist_get).  coord [n][3], type [n], box [9] = row-major lattice
 * vectors, host memory.  Errors: DP_ERR_ARG, DP_ERR_BOX, DP_ERR_CAPACITY
 * (a row overflowed cand_cap: build again with a larger one), DP_ERR_CUDA,
 * DP_ERR_OOM. */
dp_status dp_nlist_build(const dp_model *m, int64_t n, const double *coord, const int32_t *type,
                         const double box[9], double rcut, double skin, int32_t cand_cap, dp_nlist **out);

/* Several independent configurations ("frames") of the same n atoms (same
 * types, same box) as one list over nframes * n atoms: frame f holds atoms
 * [f n, (f+1) n) and each frame has its own cell grid, so no neighbor
 * crosses frames.  A training batch is evaluated by one call over it (all
 * frames fill the GPU together).  coord [nframes][n][3], type [n] (shared
 * by every frame), box as for dp_nlist_build; dp_nlist_update /
 * dp_nlist_update_dev then take [nframes][n][3].  dp_compute over such a
 * list returns the sums over the frames of E and W (E_i and F per atom);
 * dp_force_loss_grad_dev sums the per-frame losses and gradients.  MD
 * states build their own single-frame lists.  Errors: as dp_nlist_build. */
dp_status dp_nlist_build_frames(const dp_model *m, int32_t nframes, int64_t n, const double *coord,
                                const int32_t *type, const double box[9], double rcut, double skin,
                                int32_t cand_cap, dp_nlist **out);

/* Rebuild the candidates of an existing list at new coordinates (same n,
 * types, rcut, skin and capacity) and format it there. */
dp_status dp_nlist_update(dp_nlist *nl, const double *coord, const double box[9]);

/* Device-pointer form of dp_nlist_update: d_coord [n][3] in device memory,
 * enqueued on `stream`.  A capacity overflow is recorded in the list and
 * reported (DP_ERR_CAPACITY) by the next dp_nlist_get. */
dp_status dp_nlist_update_dev(dp_nlist *nl, const double *d_coord, void *stream);

/* The formatted list of the last format (build, update or dp_compute):
 * nlist [n][sum(sel)] int32, for each atom the type-0 block then the type-1
 * block and so on; inside a block the neighbors with r < r_c ordered by
 * (floor(r * 1e8), index) ascending, the first sel_t kept, the rest of the
 * block -1 (Sec. 4.1.1).  *n_truncated = number of neighbors dropped
 * because a block overflowed (not an error).  Either output may be NULL. */
dp_status dp_nlist_get(const dp_nlist *nl, int32_t *nlist, int64_t *n_truncated);

void dp_nlist_destroy(dp_nlist *nl);

/* Ghost atoms of a spatial decomposition (Sec. 4.3: each rank evaluates
 * the atoms of its sub-domain with the ghost atoms of a halo around it).
 * Atoms [0, n_centers) of the list are centers; atoms [n_centers, n) are
 * ghosts: they appear in the centers' neighbor rows but have no rows of
 * their own (cleared after every format), so an evaluation gives them
 * energy 0 and no virial, and their forces hold only the reactions
 * F_j -= g_ij of the centers' pairs, which the caller returns to the
 * ghosts' owners.  E and W sum over the centers.  n_centers = n (the
 * default) restores a plain list.  The ghosts' coordinates must be images
 * placed where the centers see them; with a slab along x the box's x edge
 * must exceed the extended region by r_c so that no periodic image of a
 * ghost reaches a center.  Errors: DP_ERR_ARG (NULL, n_centers outside
 * 0..n). */
dp_status dp_nlist_set_centers(dp_nlist *nl, int64_t n_centers);

/* The halo of one side of a slab (Sec. 4.3): of the atoms d_coord [n][3]
 * (device, FP64), d_type [n], those with lo <= x < hi, in index order, as
 * d_idx [count] (their indices), d_out_coord [count][3] (x + shift_x, y, z:
 * the positions in the receiving rank's frame) and d_out_type [count];
 * *d_count = count (device int64).  At most cap are written (count may
 * exceed cap: the caller then retries with more room).  Enqueued on
 * `stream`.  Errors: DP_ERR_ARG, DP_ERR_CUDA. */
dp_status dp_halo_select_dev(int64_t n, const double *d_coord, const int32_t *d_type, double lo, double hi,
                             double shift_x, int64_t cap, int32_t *d_idx, double *d_out_coord, int32_t *d_out_type,
                             int64_t *d_count, void *stream);

/* The reverse halo: d_force[d_idx[k]] += d_f_ghost[k] (3 components) for
 * k < m, all device memory; the indices of one call must be distinct (one
 * call per halo side keeps the sums in a fixed order).  Enqueued on
 * `stream`.  Errors: DP_ERR_ARG, DP_ERR_CUDA. */
dp_status dp_halo_accumulate_dev(int64_t m, const int32_t *d_idx, const double *d_f_ghost, double *d_force,
                                 void *stream);

/* Formatted neighbor list that allocates no device memory.  The paper has
 * no counterpart: this entry point serves callers that cannot allocate
 * device memory, such as a host MD engine whose device memory belongs to
 * its own pool or to a framework's caching allocator, or code that must not
 * let cudaMalloc / cudaFree synchronise the device.  It computes the same
 * canonical list as dp_nlist_build + dp_nlist_get (r < rcut, type blocks of
 * sel_t slots ordered by (floor(r * 1e8), index), -1 padded), from a cell
 * grid held in a fixed static device array of about 1.5 MB that every GPU
 * loading the library keeps until exit.
 *   n <= 131072 atoms, else DP_ERR_ARG; at most 1024 neighbors within rcut
 *   per atom (more sets *d_status = 1 and the list of that atom is partial).
 *   d_coord [n][3], d_type [n] (0..ntypes-1; other values set *d_status = 1
 *   and are left out), d_nlist [n][sum(sel)] output, *d_ntrunc output
 *   (neighbors dropped by full blocks), *d_status output (0 = fine): all
 *   device memory owned by the caller; box, sel: host arrays.
 *   Enqueued on `stream` without host synchronisation.  The first call on
 *   a device looks up the static array's device address (a synchronous
 *   runtime call); make that first call before any stream capture.  Every
 *   call reuses the same static array, so calls that overlap on the GPU
 *   (different streams, or different host threads) race: serialise them. */
dp_status dp_nlist_format_noalloc(int64_t n, const double *d_coord, const int32_t *d_type, const double box[9],
                                  double rcut, int32_t ntypes, const int32_t *sel, int32_t *d_nlist,
                                  unsigned long long *d_ntrunc, int32_t *d_status, void *stream);

/* -------------------------------------------------------------- compute */

/* Energy, per-atom energies, forces and virial at coordinates coord [n][3]
 * (host), formatting the list from its candidates first.  energy [1] eV,
 * atom_energy [n] eV or NULL, force [n][3] eV/A, virial [9] eV (row-major
 * W_ab = -sum d_a g_b, symmetric) or NULL.  The candidates must still be
 * valid for coord (no atom moved more than skin/2 since they were built).
 * Errors: DP_ERR_ARG, DP_ERR_BOX, DP_ERR_UNSUPPORTED (precision not built),
 * DP_ERR_NONFINITE, DP_ERR_CUDA, DP_ERR_OOM. */
dp_status dp_compute(dp_model *m, dp_nlist *nl, const double *coord, const double box[9], dp_precision prec,
                     double *energy, double *atom_energy, double *force, double *virial);

/* Device-pointer form of dp_compute: d_coord [n][3], d_energy [1],
 * d_atom_energy [n] or NULL, d_force [n][3], d_virial [9] or NULL, all in
 * device memory; box stays a host array.  Enqueued on `stream`; no host
 * synchronisation, so non-finite values are not checked here. */
dp_status dp_compute_dev(dp_model *m, dp_nlist *nl, const double *d_coord, const double box[9],
                         dp_precision prec, double *d_energy, double *d_atom_energy, double *d_force,
                         double *d_virial, void *stream);

/* ------------------------------------------------------------ training */

/* Gradient over the parameters of alpha E + beta Edot, where
 * Edot = sum_k v_k . dE/dr_k is the derivative of E along the displacement
 * field v [n][3] (a forward-mode tangent).  With v = F - F_ref this is the
 * primitive of force matching: F = -grad E, so the force term of a loss
 * differentiates to -dEdot/dtheta.  Embedding activations are recomputed in
 * the reverse pass, not stored.  prec: DP_FP64 computes in FP64, any mixed
 * scheme in FP32.  energy, edot: host scalars (may be NULL); grad
 * [n_params] host array, ADDED to (flat order of dp_model_get_params).
 * coord, v host arrays; box must match the list's box.  Errors: as
 * dp_compute. */
dp_status dp_param_grad(dp_model *m, dp_nlist *nl, const double *coord, const double box[9], const double *v,
                        double alpha, double beta, dp_precision prec, double *energy, double *edot, double *grad);

/* Force-matching loss of one configuration and its parameter gradient:
 * L = p_e ((E - E_ref)/n)^2 + p_f/(3n) sum_k |F_k - F_ref,k|^2, using
 * dL/dtheta = 2 p_e (E - E_ref)/n^2 dE/dtheta - 2 p_f/(3n) dEdot/dtheta
 * with v = F - F_ref.  E and F are evaluated in `prec` first.  *loss and
 * grad [n_params] are ADDED to (host memory).  The list must hold one
 * frame (DP_ERR_ARG otherwise). */
dp_status dp_force_loss_grad(dp_model *m, dp_nlist *nl, const double *coord, const double box[9],
                             const double *F_ref, double E_ref, double p_e, double p_f, dp_precision prec,
                             double *loss, double *grad);

/* Device-pointer form: d_coord [n][3], d_F_ref [n][3], d_E_ref [nframes]
 * (one per frame of the list, see dp_nlist_build_frames), d_loss [1] and
 * d_grad [n_params] in device memory (the last two ADDED to), enqueued on
 * `stream` without host synchronisation.  Over frames, the loss and the
 * gradient are the sums of the single-frame ones (n = atoms per frame). */
dp_status dp_force_loss_grad_dev(dp_model *m, dp_nlist *nl, const double *d_coord, const double box[9],
                                 const double *d_F_ref, const double *d_E_ref, double p_e, double p_f,
                                 dp_precision prec, double *d_loss, double *d_grad, void *stream);

/* One Adam step (Kingma and Ba 2015) on the model's device parameters with
 * the device gradient d_grad [n_params]: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, theta -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps);
 * step t >= 1.  The moments are owned by the model (zero at creation).
 * The FP32 and transposed copies are refreshed on the device; call
 * dp_model_sync_params before reading the parameters back or evaluating in
 * a MIX-16 scheme.  Enqueued on `stream`. */
dp_status dp_adam_step(dp_model *m, const double *d_grad, double lr, double beta1, double beta2, double eps,
                       int64_t t, void *stream);

/* Copy the device parameters back into the model's host copy and re-pack
 * the tensor-core images (after dp_adam_step). */
dp_status dp_model_sync_params(dp_model *m);

/* ------------------------------------------------------------------- MD */

/* MD state for velocity-Verlet NVE (Sec. 5.1): coordinates, velocities,
 * types, per-type masses (amu) and the box are copied to the device; a skin
 * list with `skin` A is built there and rebuilt on the device whenever an
 * atom has moved more than skin/2 since the last build. */
dp_status dp_md_state_create(dp_model *m, int64_t n, const double *coord, const double *vel, const int32_t *type,
                             const double *mass_by_type, const double box[9], double skin, int32_t cand_cap,
                             dp_md_state **out);

/* Run nsteps steps of dt_fs: v += dt/2 a; x += dt v (wrapped into the box);
 * recompute F; v += dt/2 a, with a = F/m * 9.648533212e-3 A/fs^2.  After
 * every thermo_every-th step one row (KE eV, PE eV, T K, P bar) is written
 * to thermo [nsteps/thermo_every][4] (NULL or thermo_every <= 0: none); T
 * uses 3n - 3 degrees of freedom and P = (2 KE + tr W)/(3V).  The host
 * synchronises once at the end.  After the first step of a call the steps
 * are replays of one captured step (a CUDA graph kept in the state and
 * captured again when the precision, dt, the profiling selection, the
 * model's buffers or parameters, or the DP_NO_OZAKI / DP_OZ_MIN_ATOMS /
 * DP_SIMT_FIT / DP_BATCH_ATOMS switches change); DP_NO_GRAPH=1 launches
 * every step directly.  Errors: as dp_compute, plus
 * DP_ERR_CAPACITY when a rebuild overflowed the candidate capacity (the
 * steps after the overflow used truncated lists and are not valid: create
 * the state again with a larger cand_cap). */
dp_status dp_md_step(dp_model *m, dp_md_state *s, int64_t nsteps, double dt_fs, dp_precision prec,
                     int32_t thermo_every, double *thermo);

/* Fixed-interval list rebuilds (Sec. 5.1: the paper's production runs
 * build the neighbor list with a 2 A skin every 50 steps).  every > 0: the
 * later steps of dp_md_step and dp_md_step_judged also rebuild the skin
 * list at every every-th step, counted from this call, besides the
 * rebuilds that the displacement criterion (an atom moved more than
 * skin/2) triggers; every = 0 (the default): the displacement criterion
 * alone.  Synchronises the model's stream.  Errors: DP_ERR_ARG (NULL
 * state, every < 0), DP_ERR_CUDA, DP_ERR_OOM. */
dp_status dp_md_set_rebuild_every(dp_md_state *s, int32_t every);

/* The learned fast path with the full model as judge and fallback: nsteps
 * NVE steps of `s` (created with `student`) driven by the student's forces;
 * after every judge_every-th step the full model `teacher` is evaluated at
 * the same coordinates, the force RMSE sqrt(mean_i |F_s,i - F_t,i|^2) is
 * written to rmse_log[w] (w = window index) and, when it exceeds rmse_max,
 * the next window runs on the teacher's forces (fallback_log[w] = 1) until
 * a later judgement is within rmse_max again.  Both models must share
 * types, r_c and sel; the teacher's work runs on the student's stream.  rmse_log, fallback_log:
 * host arrays [nsteps/judge_every] (may be NULL).  The host synchronises
 * once per judgement.  Errors: as dp_md_step. */
dp_status dp_md_step_judged(dp_model *student, dp_model *teacher, dp_md_state *s, int64_t nsteps, double dt_fs,
                            dp_precision student_prec, dp_precision teacher_prec, int32_t judge_every,
                            double rmse_max, double *rmse_log, int32_t *fallback_log);

/* Copy the state out: coord [n][3], vel [n][3] (either may be NULL),
 * *step = steps taken so far, *n_rebuilds = list rebuilds so far (NULL ok). */
dp_status dp_md_state_get(const dp_md_state *s, double *coord, double *vel, int64_t *step, int64_t *n_rebuilds);

/* Checkpoint and resume of an MD state (no counterpart in the paper, whose
 * runs restart through the MD engine) as one flat binary file of FP64
 * values (host byte order): a header {magic 0x4450'4d44 ("DPMD"), version 1,
 * n, ntypes, step, skin, cand_cap, forces valid (0/1), their precision},
 * box [9], mass_by_type [ntypes], type [n], coord [n][3], vel [n][3], and
 * the forces at coord [n][3] (0 when not valid).  dp_md_state_load creates
 * a state with `m` (whose ntypes must match) from such a file; with the
 * saved forces restored, the first step of the resumed run kicks with the
 * same forces as an uninterrupted run would, and the step counter goes on
 * from the saved one (the skin list is rebuilt at the saved coordinates,
 * which changes when later rebuilds happen, not the formatted lists).
 * Errors: DP_ERR_ARG (NULL argument, a file that cannot be opened, read or
 * written, a bad header, a type mismatch, or a file whose size is not the
 * one its header gives; checked before anything is allocated), DP_ERR_CUDA,
 * DP_ERR_OOM. */
dp_status dp_md_state_save(const dp_md_state *s, const char *path);
dp_status dp_md_state_load(dp_model *m, const char *path, dp_md_state **out);

void dp_md_state_destroy(dp_md_state *s);

/* ---------------------------------------------------------- diagnostics */

/* The activation function of the FP64 nets (Fig. 1(e-g)): y[i] = tanh(x[i])
 * for d_x, d_y [n] FP64 in device memory, evaluated by the same device
 * routine the FP64 kernels use (degree-10 Taylor table on intervals of 1/16,
 * library tanh for |x| >= 16).  Enqueued on `stream`.  Exposed so that its
 * accuracy can be tested.  Errors: DP_ERR_ARG (n < 0, NULL with n > 0),
 * DP_ERR_CUDA. */
dp_status dp_tanh_f64_dev(int64_t n, const double *d_x, double *d_y, void *stream);

/* The FP64 product the double-precision fitting net runs on the tensor
 * cores: C = A B^T with A [M][K], Bt = B^T stored as [N][K], C [M][N],
 * row-major FP64 in device memory, by error-free splitting into fp16
 * digits (the scheme of Ozaki, Ogita, Oishi and Rump): per entry an error
 * of the order of K 2^-54 max|A_row| max|B_row|, the size of FP64
 * rounding.  Shapes: K % 16 == 0 and K <= 1808; N % 64 == 0 when
 * K <= 256 (8 digits of 7 bits), else N % 48 == 0 (9 digits of 6 bits).
 * Allocates its digit buffers, runs on `stream` and synchronises it.
 * Exposed so that its accuracy can be tested.  Errors: DP_ERR_ARG (shape), DP_ERR_OOM,
 * DP_ERR_CUDA, DP_ERR_TIMEOUT. */
dp_status dp_ozaki_dgemm_dev(dp_model *m, int64_t M, int32_t N, int32_t K, const double *d_A, const double *d_Bt,
                             double *d_C, void *stream);

/* Test of the bounded device waits (no counterpart in the paper, which
 * describes no failure handling).  which = 1 starves one wait of this
 * model's later evaluations: the tensor-core (MIX-16) embedding kernel no
 * longer issues the bulk copy of its weights, so its wait on that copy
 * runs out after `polls` polls (1 .. 2^20) with nothing in flight; the
 * kernel then sets the device error word, leaves its tile loop, frees its
 * tensor memory and returns, and the host call reports DP_ERR_TIMEOUT.
 * Every other wait keeps its default limit (about a second).  which = 0
 * restores normal evaluation (polls ignored).  Host-side only: it takes
 * effect at the next call and drops captured graphs of the model.
 * Errors: DP_ERR_ARG (NULL model, unknown wait, polls out of range). */
dp_status dp_test_starve_wait(dp_model *m, int32_t which, int64_t polls);

/* Bounds-checked debug build (no counterpart in the paper; the stand-in for a
 * device memory checker).  A library compiled with -DDP_BOUNDS_CHECK checks
 * every index that its kernels read from memory or derive from coordinates
 * (neighbor indexes of the candidate and formatted lists, cell indexes and
 * cell-list slots, atoms of the tensor-core work lists, type ids read back
 * from packed keys) against the buffer it addresses before using it; a bad
 * index is not used (the neighbor counts as padding, the access is skipped)
 * and the first one is recorded.  dp_bounds_checked() returns 1 for such a
 * library and 0 for the default build.  dp_bounds_read() synchronises the
 * device and writes rec[0] = number of bad indexes since the last clear,
 * rec[1] = site of the first (1 type id, 2 cell index, 3 cell-list slot,
 * 4 candidate atom, 5 formatted-list neighbor, 6 work-list atom), rec[2] =
 * the index, rec[3] = the limit it broke; clear != 0 zeroes the record
 * afterwards.  In the default build rec is all zeros.  rec: caller-owned
 * host array of 4.  Errors: DP_ERR_ARG (NULL rec), DP_ERR_CUDA. */
int32_t dp_bounds_checked(void);
dp_status dp_bounds_read(int64_t *rec, int32_t clear);

#ifdef __cplusplus
}
#endif

#endif /* DP_H */

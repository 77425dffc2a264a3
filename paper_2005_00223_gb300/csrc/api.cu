// C-ABI entry points of libdp (declared in include/dp.h): argument checks,
// handle and device-memory management, orchestration of the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "dp_internal.cuh"

namespace dp {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

dp_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA;
}

dp_status ensure_workspace(dp_model *m, size_t bytes)
{
    if (bytes <= m->ws_bytes) return DP_OK;
    if (m->ws) {
        DP_CUDA(cudaStreamSynchronize(m->stream));
        DP_CUDA(cudaDeviceSynchronize());
        cudaFree(m->ws);
        m->ws = nullptr;
        m->ws_bytes = 0;
    }
    DP_CUDA(cudaMalloc((void **)&m->ws, bytes));
    m->ws_bytes = bytes;
    ++m->epoch;
    return DP_OK;
}

dp_status check_box(const double box[9], double rcut, double L[3])
{
    if (!box) {
        set_error("box is NULL");
        return DP_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && box[3 * a + b] != 0.0) {
                set_error("only orthorhombic boxes are supported (box[%d][%d] = %g)", a, b, box[3 * a + b]);
                return DP_ERR_BOX;
            }
    for (int a = 0; a < 3; ++a) {
        L[a] = box[4 * a];
        if (!(L[a] > 0.0) || !isfinite(L[a])) {
            set_error("box length %d is %g", a, L[a]);
            return DP_ERR_BOX;
        }
        if (!(rcut < 0.5 * L[a])) {
            set_error("rcut %g must be below half the box length %g", rcut, L[a]);
            return DP_ERR_BOX;
        }
    }
    return DP_OK;
}

dp_status ensure_aux(dp_model *m, int64_t n)
{
    if (n <= m->aux_n) return DP_OK;
    if (m->d_aux) {
        DP_CUDA(cudaStreamSynchronize(m->stream));
        cudaFree(m->d_aux);
        m->d_aux = nullptr;
    }
    size_t cnt = (size_t)(n > 0 ? n : 1) * (1 + 9 + 3 + 3) + 16;
    DP_CUDA(cudaMalloc((void **)&m->d_aux, sizeof(double) * cnt));
    m->aux_n = n;
    ++m->epoch;
    return DP_OK;
}

struct Aux {
    double *Ei, *Wi, *F, *coord, *scal;
};

static Aux aux_of(dp_model *m)
{
    int64_t n = m->aux_n > 0 ? m->aux_n : 1;
    Aux a;
    a.Ei = m->d_aux;
    a.Wi = a.Ei + n;
    a.F = a.Wi + 9 * n;
    a.coord = a.F + 3 * n;
    a.scal = a.coord + 3 * n;
    return a;
}

// Precisions whose kernels read the formatting kernel's FP64-derived geometry records.
static bool uses_env_records(dp_precision p)
{
    return p == DP_MIX_BF16 || p == DP_MIX_FP16 || p == DP_MIX_BF16X3 || p == DP_MIX_FP8;
}

bool format_shared(const dp_model *a, dp_precision pa, const dp_model *b, dp_precision pb)
{
    // the geometry records carry s(r) and ds/dr, which depend on r_cs as well
    if (a->dev.rcut != b->dev.rcut || a->dev.rcs != b->dev.rcs || a->dev.ntypes != b->dev.ntypes) return false;
    for (int t = 0; t < a->dev.ntypes; ++t)
        if (a->dev.sel[t] != b->dev.sel[t]) return false;
    return !uses_env_records(pb) || uses_env_records(pa);
}

dp_status compute_device(dp_model *m, dp_nlist *nl, const double *d_coord, dp_precision prec, double *d_energy,
                         double *d_atom_energy, double *d_force, double *d_virial, double *d_atom_virial,
                         cudaStream_t st, bool reformat)
{
    m->dev.n_list = nl->n;
    if (reformat) DP_TRY(nlist_format_device(m, nl, d_coord, st, uses_env_records(prec)));
    if (nl->n == 0) {
        DP_CUDA(cudaMemsetAsync(d_energy, 0, sizeof(double), st));
        if (d_virial) DP_CUDA(cudaMemsetAsync(d_virial, 0, 9 * sizeof(double), st));
        return DP_OK;
    }
    dp_status r = DP_OK;
    if (embed_is_wide(m->n_embed, m->embed)) {   // the wide nets run in MIX-16 (bf16) or FP8 only
        if (prec != DP_MIX_BF16 && prec != DP_MIX_FP8) {
            set_error("embedding nets wider than 32-64-128 run in DP_MIX_BF16 or DP_MIX_FP8 only");
            return DP_ERR_UNSUPPORTED;
        }
        r = compute_wide(m, nl, prec == DP_MIX_FP8, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        prec = DP_PRECISION_DONE;
    } else if (prec == DP_MIX_FP8) {
        set_error("DP_MIX_FP8 covers the wide embedding nets (w, 2w, 4w), w = 64 .. 512, only");
        return DP_ERR_UNSUPPORTED;
    }
    switch (prec) {
    case DP_FP64:
        r = compute_fp64(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        break;
    case DP_MIX32:
        r = compute_mix32(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        break;
    case DP_MIX_BF16:
        r = compute_mix16(m, nl, 1, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        break;
    case DP_MIX_FP16:
        r = compute_mix16(m, nl, 0, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        break;
    case DP_MIX_BF16X3:
        r = compute_mix_x3(m, nl, d_energy, d_atom_energy, d_force, d_virial, d_atom_virial, st);
        break;
    case DP_PRECISION_DONE:
        break;
    default:
        set_error("precision %d is not built into this library", (int)prec);
        return DP_ERR_UNSUPPORTED;
    }
    const int64_t nc = centers_of(nl);
    if (r == DP_OK && nc < nl->n)   // ghosts have no neighbors: their fitting-net values are not energies
        DP_CUDA(cudaMemsetAsync(d_atom_energy + nc, 0, sizeof(double) * (size_t)(nl->n - nc), st));
    return r;
}

// SplitMix64 (Steele, Lea and Flood 2014) and Box-Muller normals, cosine
// branch first: the seeded weight generator of dp_model_create.
struct SplitMix64 {
    uint64_t state;
    bool has_spare = false;
    double spare = 0.0;
    explicit SplitMix64(uint64_t s) : state(s) {}
    uint64_t next()
    {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        if (has_spare) {
            has_spare = false;
            return spare;
        }
        double u1 = uniform(), u2 = uniform();
        double rad = sqrt(-2.0 * log(1.0 - u1));
        double ang = 2.0 * M_PI * u2;
        spare = rad * sin(ang);
        has_spare = true;
        return rad * cos(ang);
    }
};

static NetLayout make_layout(int nin, int nlayers, const int *w, bool output_layer)
{
    NetLayout L{};
    int64_t off = 0;
    int win = nin;
    int total = nlayers + (output_layer ? 1 : 0);
    L.n_layers = total;
    for (int k = 0; k < total; ++k) {
        int wout = k < nlayers ? w[k] : 1;
        L.win[k] = win;
        L.wout[k] = wout;
        L.W[k] = off;
        off += (int64_t)win * wout;
        L.b[k] = off;
        off += wout;
        win = wout;
    }
    L.size = off;
    return L;
}

}  // namespace dp

using namespace dp;

extern "C" {

const char *dp_status_string(dp_status st)
{
    switch (st) {
    case DP_OK: return "DP_OK";
    case DP_ERR_ARG: return "DP_ERR_ARG";
    case DP_ERR_CUDA: return "DP_ERR_CUDA";
    case DP_ERR_OOM: return "DP_ERR_OOM";
    case DP_ERR_BOX: return "DP_ERR_BOX";
    case DP_ERR_CAPACITY: return "DP_ERR_CAPACITY";
    case DP_ERR_TIMEOUT: return "DP_ERR_TIMEOUT";
    case DP_ERR_NONFINITE: return "DP_ERR_NONFINITE";
    case DP_ERR_UNSUPPORTED: return "DP_ERR_UNSUPPORTED";
    }
    return "DP_UNKNOWN";
}

const char *dp_last_error(void) { return g_last_error.c_str(); }

static dp_status upload_params(dp_model *m)
{
    ++m->epoch;
    m->oz_stale = true;
    m->oz_emb_stale = true;
    m->oz_fit_stale = true;
    const ModelDev &md = m->dev;
    std::vector<double> pT(m->h_params);
    auto transpose_net = [&](int64_t base, const NetLayout &L) {
        for (int k = 0; k < L.n_layers; ++k) {
            const double *W = m->h_params.data() + base + L.W[k];
            double *WT = pT.data() + base + L.W[k];
            for (int a = 0; a < L.win[k]; ++a)
                for (int o = 0; o < L.wout[k]; ++o) WT[(int64_t)o * L.win[k] + a] = W[(int64_t)a * L.wout[k] + o];
        }
    };
    for (int q = 0; q < m->ntypes * m->ntypes; ++q) transpose_net(md.emb_base + q * md.emb.size, md.emb);
    for (int t = 0; t < m->ntypes; ++t) transpose_net(md.fit_base + t * md.fit.size, md.fit);
    std::vector<float> p32(m->nparams), pT32(m->nparams);
    for (int64_t q = 0; q < m->nparams; ++q) {
        p32[q] = (float)m->h_params[q];
        pT32[q] = (float)pT[q];
    }
    size_t b64 = sizeof(double) * m->nparams, b32 = sizeof(float) * m->nparams;
    DP_CUDA(cudaMemcpyAsync(m->d_params, m->h_params.data(), b64, cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaMemcpyAsync(m->d_paramsT, pT.data(), b64, cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaMemcpyAsync(m->d_params32, p32.data(), b32, cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaMemcpyAsync(m->d_paramsT32, pT32.data(), b32, cudaMemcpyHostToDevice, m->stream));
    DP_CUDA(cudaStreamSynchronize(m->stream));
    return pack_tc_weights(m);
}

dp_status dp_model_create(const dp_model_config *cfg, uint64_t seed, dp_model **out)
{
    if (!cfg || !out || !cfg->sel || !cfg->embed || !cfg->fit) {
        set_error("dp_model_create: NULL argument");
        return DP_ERR_ARG;
    }
    *out = nullptr;
    if (cfg->ntypes < 1 || cfg->ntypes > kMaxTypes) {
        set_error("ntypes %d outside 1..%d", cfg->ntypes, kMaxTypes);
        return DP_ERR_ARG;
    }
    if (!(cfg->rcut > 0) || !(cfg->rcut_smth > 0) || !(cfg->rcut_smth < cfg->rcut)) {
        set_error("need 0 < rcut_smth < rcut (got %g, %g)", cfg->rcut_smth, cfg->rcut);
        return DP_ERR_ARG;
    }
    if (!(cfg->rcut * 1e8 < (double)(1 << 30))) {
        set_error("rcut %g too large for the 30-bit distance field of the neighbor key (max 10.7 A)", cfg->rcut);
        return DP_ERR_UNSUPPORTED;
    }
    int nsel = 0;
    for (int t = 0; t < cfg->ntypes; ++t) {
        if (cfg->sel[t] < 1 || cfg->sel[t] > 4096) {
            set_error("sel[%d] = %d outside 1..4096", t, cfg->sel[t]);
            return DP_ERR_ARG;
        }
        nsel += cfg->sel[t];
    }
    if (cfg->n_embed < 1 || cfg->n_embed > kMaxEmbed || cfg->n_fit < 1 || cfg->n_fit > kMaxFit) {
        set_error("n_embed %d / n_fit %d outside 1..4", cfg->n_embed, cfg->n_fit);
        return DP_ERR_ARG;
    }
    for (int k = 0; k < cfg->n_embed; ++k)
        if (cfg->embed[k] < 1) { set_error("embed width %d < 1", k); return DP_ERR_ARG; }
    for (int k = 0; k < cfg->n_fit; ++k)
        if (cfg->fit[k] < 1 || cfg->fit[k] > kMaxFitWidth) {
            set_error("fit width %d outside 1..%d", cfg->fit[k], kMaxFitWidth);
            return DP_ERR_ARG;
        }
    const int m1 = cfg->embed[cfg->n_embed - 1];
    if (cfg->axis_neuron < 1 || cfg->axis_neuron > m1) {
        set_error("axis_neuron %d outside 1..M1 = %d", cfg->axis_neuron, m1);
        return DP_ERR_ARG;
    }
    if (!embed_shape_supported(cfg->n_embed, cfg->embed)) {
        set_error("embedding shape not compiled in (supported: 25-50-100, 8-16-32, 32-64-128)");
        return DP_ERR_UNSUPPORTED;
    }
    dp_model *m = new (std::nothrow) dp_model();
    if (!m) return DP_ERR_OOM;
    cudaGetDevice(&m->device);
    m->ntypes = cfg->ntypes;
    m->rcut = cfg->rcut;
    m->rcs = cfg->rcut_smth;
    for (int t = 0; t < cfg->ntypes; ++t) m->sel[t] = cfg->sel[t];
    m->n_embed = cfg->n_embed;
    for (int k = 0; k < cfg->n_embed; ++k) m->embed[k] = cfg->embed[k];
    m->m2 = cfg->axis_neuron;
    m->n_fit = cfg->n_fit;
    for (int k = 0; k < cfg->n_fit; ++k) m->fit[k] = cfg->fit[k];
    ModelDev &md = m->dev;
    md.ntypes = m->ntypes;
    md.nsel = nsel;
    md.m1 = m1;
    md.m2 = m->m2;
    md.n_embed = m->n_embed;
    md.n_fit = m->n_fit;
    md.desc_dim = m1 * m->m2;
    int off = 0, coff = 0;
    for (int t = 0; t < m->ntypes; ++t) {
        md.sel[t] = m->sel[t];
        md.sel_off[t] = off;
        md.chunk_off[t] = coff;
        off += m->sel[t];
        coff += (m->sel[t] + kChunk - 1) / kChunk;
    }
    md.sel_off[m->ntypes] = off;
    md.chunk_off[m->ntypes] = coff;
    md.chunks_per_atom = coff;
    md.rcut = m->rcut;
    md.rcs = m->rcs;
    md.inv_sw = 1.0 / (m->rcut - m->rcs);
    md.inv_nsel = 1.0 / (double)nsel;
    md.emb = make_layout(1, m->n_embed, m->embed, false);
    md.fit = make_layout(md.desc_dim, m->n_fit, m->fit, true);
    md.emb_base = 0;
    md.fit_base = (int64_t)m->ntypes * m->ntypes * md.emb.size;
    int asum = 0;
    for (int k = 0; k < m->n_embed; ++k) asum += m->embed[k];
    md.act_stride = asum + m1;
    m->nparams = md.fit_base + (int64_t)m->ntypes * md.fit.size;
    // seeded weights, N(0, 1/fan_in), flat order
    m->h_params.resize(m->nparams);
    SplitMix64 rng(seed);
    auto fill_net = [&](int64_t base, const NetLayout &L) {
        for (int k = 0; k < L.n_layers; ++k) {
            double sc = sqrt(1.0 / (double)L.win[k]);
            for (int64_t q = 0; q < (int64_t)L.win[k] * L.wout[k]; ++q) m->h_params[base + L.W[k] + q] = rng.normal() * sc;
            for (int q = 0; q < L.wout[k]; ++q) m->h_params[base + L.b[k] + q] = rng.normal() * sc;
        }
    };
    for (int q = 0; q < m->ntypes * m->ntypes; ++q) fill_net(md.emb_base + q * md.emb.size, md.emb);
    for (int t = 0; t < m->ntypes; ++t) fill_net(md.fit_base + t * md.fit.size, md.fit);
    dp_status st = DP_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&m->own_stream, cudaStreamNonBlocking);
    m->stream = m->own_stream;
    m->prof = new (std::nothrow) Prof();
    if (!m->prof) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_params, sizeof(double) * m->nparams);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_paramsT, sizeof(double) * m->nparams);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_params32, sizeof(float) * m->nparams);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_paramsT32, sizeof(float) * m->nparams);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_flag, sizeof(int32_t) * 4);
    // the partial sums of the energy / virial reduction and its arrival counter (zeroed once)
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_red, sizeof(double) * (kRedParts * 10 + 1));
    if (e == cudaSuccess) e = cudaMemset(m->d_red + kRedParts * 10, 0, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_err, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(m->d_err, 0, sizeof(int32_t) * 4);
    if (e != cudaSuccess) st = cuda_fail(e, "dp_model_create");
    if (st == DP_OK) {
        md.p = m->d_params;
        md.pT = m->d_paramsT;
        md.p32 = m->d_params32;
        md.pT32 = m->d_paramsT32;
        st = upload_params(m);
    }
    if (st != DP_OK) {
        dp_model_destroy(m);
        return st;
    }
    const char *env = getenv("DP_BATCH_ATOMS");
    m->batch_atoms = env ? atoll(env) : 0;
    if (m->batch_atoms <= 0) {
        // workspace budget of the FP64 path: a quarter of the device memory (at least 12 GiB) of
        // per-atom scratch
        size_t fr = 0, tot = 0;
        size_t budget = (size_t)12 * 1024 * 1024 * 1024;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && tot / 4 > budget) budget = tot / 4;
        size_t per = fp64_bytes_per_atom(md);
        m->batch_atoms = (int64_t)(budget / per);
        if (m->batch_atoms < 256) m->batch_atoms = 256;
    }
    *out = m;
    return DP_OK;
}

dp_status dp_model_n_params(const dp_model *m, int64_t *n)
{
    if (!m || !n) { set_error("dp_model_n_params: NULL argument"); return DP_ERR_ARG; }
    *n = m->nparams;
    return DP_OK;
}

dp_status dp_model_get_params(const dp_model *m, double *flat, int64_t n)
{
    if (!m || !flat) { set_error("dp_model_get_params: NULL argument"); return DP_ERR_ARG; }
    if (n != m->nparams) { set_error("expected %lld parameters, got %lld", (long long)m->nparams, (long long)n); return DP_ERR_ARG; }
    if (m->params_dirty) {
        DP_CUDA(cudaStreamSynchronize(m->stream));
        DP_CUDA(cudaMemcpy(flat, m->d_params, sizeof(double) * n, cudaMemcpyDeviceToHost));
        return DP_OK;
    }
    memcpy(flat, m->h_params.data(), sizeof(double) * n);
    return DP_OK;
}

dp_status dp_model_set_params(dp_model *m, const double *flat, int64_t n)
{
    if (!m || !flat) { set_error("dp_model_set_params: NULL argument"); return DP_ERR_ARG; }
    if (n != m->nparams) { set_error("expected %lld parameters, got %lld", (long long)m->nparams, (long long)n); return DP_ERR_ARG; }
    for (int64_t q = 0; q < n; ++q)
        if (!isfinite(flat[q])) { set_error("parameter %lld is not finite", (long long)q); return DP_ERR_ARG; }
    memcpy(m->h_params.data(), flat, sizeof(double) * n);
    m->params_dirty = false;
    return upload_params(m);
}

void dp_model_destroy(dp_model *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->d_params);
    cudaFree(m->d_paramsT);
    cudaFree(m->d_params32);
    cudaFree(m->d_paramsT32);
    cudaFree(m->ws);
    cudaFree(m->d_aux);
    cudaFree(m->d_flag);
    cudaFree(m->d_red);
    cudaFree(m->d_err);
    cudaFree(m->d_tcw);
    cudaFree(m->d_tcw_x3);
    cudaFree(m->d_tcfit_x3);
    for (unsigned char *p : m->d_fitcl) cudaFree(p);
    cudaFree(m->d_wide);
    cudaFree(m->d_wide_q);
    cudaFree(m->d_ozw);
    cudaFree(m->d_oze);
    cudaFree(m->d_ozw_emb);
    cudaFree(m->d_oze_emb);
    cudaFree(m->d_ozw_fit);
    cudaFree(m->d_oze_fit);
    cudaFree(m->d_tcfit);
    cudaFree(m->d_train);
    cudaFree(m->d_tscr);
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    delete m->prof;
    delete m;
}

// ------------------------------------------------------------ neighbor list


static void nlist_free(dp_nlist *nl)
{
    nlist_graph_drop(nl);
    cudaFreeHost(nl->h_io);
    nl->h_io = nullptr;
    cudaFree(nl->d_type);
    cudaFree(nl->d_cand);
    cudaFree(nl->d_cand_cnt);
    cudaFree(nl->d_ref);
    cudaFree(nl->d_cell_of);
    cudaFree(nl->d_cell_cnt);
    cudaFree(nl->d_cell_start);
    cudaFree(nl->d_cell_atoms);
    cudaFree(nl->d_nlist);
    cudaFree(nl->d_nnei);
    cudaFree(nl->d_ntrunc);
    cudaFree(nl->d_flags);
    cudaFree(nl->d_pos);
    cudaFree(nl->d_posf);
    cudaFree(nl->d_env);
    cudaFree(nl->d_fx);
    cudaFree(nl->d_coord);
    cudaFree(nl->d_order);
}

void dp_nlist_destroy(dp_nlist *nl)
{
    if (!nl) return;
    if (nl->m && nl->m->stream) cudaStreamSynchronize(nl->m->stream);
    nlist_free(nl);
    delete nl;
}

// Reads the device flags after a (re)build; DP_ERR_CAPACITY on overflow.
static dp_status check_build_flags(dp_nlist *nl, cudaStream_t st)
{
    int32_t flags[3];
    DP_CUDA(cudaMemcpyAsync(flags, nl->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaStreamSynchronize(st));
    if (flags[0] & kErrCapacity) {
        set_error("a candidate list exceeded its capacity of %d; build again with a larger cand_cap", nl->cap);
        return DP_ERR_CAPACITY;
    }
    return DP_OK;
}

}  // extern "C"

dp_status dp::nlist_create_internal(const dp_model *m, int64_t n, const int32_t *type, const double box[9],
                                    double rcut, double skin, int32_t cand_cap, dp_nlist **out, int32_t nframes)
{
    if (!m || !out || (n > 0 && !type)) { set_error("dp_nlist_build: NULL argument"); return DP_ERR_ARG; }
    *out = nullptr;
    if (n < 0 || n >= (int64_t)1 << 26) { set_error("atom count %lld outside 0..2^26-1", (long long)n); return DP_ERR_ARG; }
    if (nframes < 1 || n % nframes != 0) { set_error("%lld atoms do not split into %d frames", (long long)n, nframes); return DP_ERR_ARG; }
    if (!(rcut >= m->rcut) || !(skin >= 0) || !isfinite(rcut + skin)) {
        set_error("need rcut >= model rcut (%g) and skin >= 0 (got %g, %g)", m->rcut, rcut, skin);
        return DP_ERR_ARG;
    }
    double L[3];
    DP_TRY(check_box(box, m->rcut, L));
    for (int64_t i = 0; i < n; ++i)
        if (type[i] < 0 || type[i] >= m->ntypes) { set_error("type[%lld] = %d outside 0..%d", (long long)i, type[i], m->ntypes - 1); return DP_ERR_ARG; }
    dp_nlist *nl = new (std::nothrow) dp_nlist();
    if (!nl) return DP_ERR_OOM;
    nl->m = m;
    nl->n = n;
    nl->rcut = rcut;
    nl->skin = skin;
    nl->rlist = rcut + skin;
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        nl->L[k] = L[k];
        vol *= L[k];
        int c = (int)floor(L[k] / nl->rlist);
        nl->nc[k] = c < 1 ? 1 : c;
    }
    nl->nframes = nframes;
    nl->frame_n = n / nframes;
    nl->ncell_frame = (int64_t)nl->nc[0] * nl->nc[1] * nl->nc[2];
    nl->ncell = nl->ncell_frame * nframes;
    if (cand_cap <= 0) {
        double expect = (double)nl->frame_n / vol * 4.0 / 3.0 * M_PI * nl->rlist * nl->rlist * nl->rlist;
        int64_t c = (int64_t)(expect * 1.3) + 64;
        if (c > nl->frame_n) c = nl->frame_n;
        c = (c + 31) / 32 * 32;
        nl->cap = (int32_t)(c < 32 ? 32 : c);
    } else {
        nl->cap = cand_cap;
    }
    if (nl->cap > 6144) {
        set_error("candidate capacity %d above the supported 6144", nl->cap);
        delete nl;
        return DP_ERR_UNSUPPORTED;
    }
    const int nsel = m->dev.nsel;
    int64_t nn = n > 0 ? n : 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    A((void **)&nl->d_type, sizeof(int32_t) * nn);
    A((void **)&nl->d_cand, sizeof(int32_t) * nn * nl->cap);
    A((void **)&nl->d_cand_cnt, sizeof(int32_t) * nn);
    A((void **)&nl->d_ref, sizeof(double) * 4 * nn);
    A((void **)&nl->d_cell_of, sizeof(int32_t) * nn);
    A((void **)&nl->d_cell_cnt, sizeof(int32_t) * (nl->ncell + 1));
    A((void **)&nl->d_cell_start, sizeof(int32_t) * (nl->ncell + 1));
    A((void **)&nl->d_cell_atoms, sizeof(int32_t) * nn);
    A((void **)&nl->d_nlist, sizeof(int32_t) * nn * nsel);
    A((void **)&nl->d_nnei, sizeof(int32_t) * nn * m->ntypes);
    A((void **)&nl->d_ntrunc, sizeof(unsigned long long));
    A((void **)&nl->d_flags, sizeof(int32_t) * 4);
    A((void **)&nl->d_pos, sizeof(double) * 4 * nn);
    A((void **)&nl->d_posf, sizeof(float) * 4 * nn);
    A((void **)&nl->d_coord, sizeof(double) * 3 * nn);
    A((void **)&nl->d_order, sizeof(int32_t) * nn);
    if (e != cudaSuccess) {
        dp_status s = cuda_fail(e, "dp_nlist_build (allocation)");
        nlist_free(nl);
        delete nl;
        return s;
    }
    // type-sorted order (stable), counts and offsets per type
    std::vector<int32_t> order(n);
    nl->type_count.assign(m->ntypes, 0);
    nl->type_off.assign(m->ntypes, 0);
    for (int64_t i = 0; i < n; ++i) nl->type_count[type[i]]++;
    for (int t = 1; t < m->ntypes; ++t) nl->type_off[t] = nl->type_off[t - 1] + nl->type_count[t - 1];
    std::vector<int64_t> fill(nl->type_off);
    for (int64_t i = 0; i < n; ++i) order[fill[type[i]]++] = (int32_t)i;
    cudaStream_t st = m->stream;
    if (n > 0) {
        e = cudaMemcpyAsync(nl->d_type, type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(nl->d_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(nl->d_flags, 0, sizeof(int32_t) * 4, st);
    // cell counts start at zero; every build leaves them zero again
    if (e == cudaSuccess) e = cudaMemsetAsync(nl->d_cell_cnt, 0, sizeof(int32_t) * (nl->ncell + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(nl->d_ntrunc, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dp_status s = cuda_fail(e, "dp_nlist_build (upload)");
        nlist_free(nl);
        delete nl;
        return s;
    }
    *out = nl;
    return DP_OK;
}

extern "C" {

// (Re)build candidates from device coordinates and format at them.
static dp_status nlist_rebuild_device(dp_nlist *nl, const double *d_coord, cudaStream_t st)
{
    dp_model *m = const_cast<dp_model *>(nl->m);
    DP_CUDA(cudaMemsetAsync(nl->d_flags, 0, sizeof(int32_t), st));
    DP_TRY(pack_positions(nl, d_coord, st));
    DP_TRY(nlist_build_device(nl, st, false));
    DP_TRY(check_build_flags(nl, st));
    DP_TRY(nlist_format_device(m, nl, nullptr, st));
    return DP_OK;
}

static bool box_matches(const dp_nlist *nl, const double box[9])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double want = a == b ? nl->L[a] : 0.0;
            if (box[3 * a + b] != want) return false;
        }
    return true;
}

dp_status dp_nlist_build(const dp_model *m, int64_t n, const double *coord, const int32_t *type, const double box[9],
                         double rcut, double skin, int32_t cand_cap, dp_nlist **out)
{
    if (!out || (n > 0 && !coord)) { set_error("dp_nlist_build: NULL argument"); return DP_ERR_ARG; }
    dp_nlist *nl = nullptr;
    DP_TRY(nlist_create_internal(m, n, type, box, rcut, skin, cand_cap, &nl));
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(nl->d_coord, coord, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->stream);
        if (e != cudaSuccess) {
            dp_nlist_destroy(nl);
            return cuda_fail(e, "dp_nlist_build (coordinates)");
        }
        dp_status s = nlist_rebuild_device(nl, nl->d_coord, m->stream);
        if (s == DP_OK) {
            cudaError_t e2 = cudaStreamSynchronize(m->stream);
            if (e2 != cudaSuccess) s = cuda_fail(e2, "dp_nlist_build");
        }
        if (s != DP_OK) {
            dp_nlist_destroy(nl);
            return s;
        }
    }
    *out = nl;
    return DP_OK;
}

dp_status dp_nlist_build_frames(const dp_model *m, int32_t nframes, int64_t n, const double *coord,
                                const int32_t *type, const double box[9], double rcut, double skin,
                                int32_t cand_cap, dp_nlist **out)
{
    if (!out || nframes < 1 || n < 0 || (n > 0 && (!coord || !type))) {
        set_error("dp_nlist_build_frames: NULL or bad argument");
        return DP_ERR_ARG;
    }
    if ((int64_t)nframes * n >= (int64_t)1 << 26) { set_error("dp_nlist_build_frames: too many atoms"); return DP_ERR_ARG; }
    std::vector<int32_t> all((size_t)nframes * n);
    for (int32_t f = 0; f < nframes; ++f)
        for (int64_t i = 0; i < n; ++i) all[(size_t)f * n + i] = type[i];
    dp_nlist *nl = nullptr;
    const int64_t nt = (int64_t)nframes * n;
    DP_TRY(nlist_create_internal(m, nt, all.data(), box, rcut, skin, cand_cap, &nl, nframes));
    if (nt > 0) {
        cudaError_t e = cudaMemcpyAsync(nl->d_coord, coord, sizeof(double) * 3 * nt, cudaMemcpyHostToDevice, m->stream);
        if (e != cudaSuccess) {
            dp_nlist_destroy(nl);
            return cuda_fail(e, "dp_nlist_build_frames (coordinates)");
        }
        dp_status s = nlist_rebuild_device(nl, nl->d_coord, m->stream);
        if (s == DP_OK) {
            cudaError_t e2 = cudaStreamSynchronize(m->stream);
            if (e2 != cudaSuccess) s = cuda_fail(e2, "dp_nlist_build_frames");
        }
        if (s != DP_OK) {
            dp_nlist_destroy(nl);
            return s;
        }
    }
    *out = nl;
    return DP_OK;
}

dp_status dp_nlist_update(dp_nlist *nl, const double *coord, const double box[9])
{
    if (!nl || (nl->n > 0 && !coord) || !box) { set_error("dp_nlist_update: NULL argument"); return DP_ERR_ARG; }
    if (!box_matches(nl, box)) { set_error("box differs from the list's box; build a new list"); return DP_ERR_ARG; }
    if (nl->n == 0) return DP_OK;
    cudaStream_t st = nl->m->stream;
    DP_CUDA(cudaMemcpyAsync(nl->d_coord, coord, sizeof(double) * 3 * nl->n, cudaMemcpyHostToDevice, st));
    DP_TRY(nlist_rebuild_device(nl, nl->d_coord, st));
    DP_CUDA(cudaStreamSynchronize(st));
    return DP_OK;
}

dp_status dp_nlist_update_dev(dp_nlist *nl, const double *d_coord, void *stream)
{
    if (!nl || (nl->n > 0 && !d_coord)) { set_error("dp_nlist_update_dev: NULL argument"); return DP_ERR_ARG; }
    if (nl->n == 0) return DP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DP_TRY(pack_positions(nl, d_coord, st));
    DP_TRY(nlist_build_device(nl, st, false));
    DP_TRY(nlist_format_device(nl->m, nl, nullptr, st));
    return DP_OK;
}

dp_status dp_nlist_get(const dp_nlist *nl, int32_t *nlist, int64_t *n_truncated)
{
    if (!nl) { set_error("dp_nlist_get: NULL list"); return DP_ERR_ARG; }
    cudaStream_t st = nl->m->stream;
    DP_CUDA(cudaStreamSynchronize(st));
    DP_CUDA(cudaDeviceSynchronize());
    if (nl->n > 0) {
        int32_t flags[3];
        DP_CUDA(cudaMemcpy(flags, nl->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
        if (flags[0] & kErrCapacity) {
            set_error("a candidate list exceeded its capacity of %d; build again with a larger cand_cap", nl->cap);
            return DP_ERR_CAPACITY;
        }
    }
    if (nlist && nl->n > 0)
        DP_CUDA(cudaMemcpy(nlist, nl->d_nlist, sizeof(int32_t) * nl->n * nl->m->dev.nsel, cudaMemcpyDeviceToHost));
    if (n_truncated) {
        unsigned long long t = 0;
        DP_CUDA(cudaMemcpy(&t, nl->d_ntrunc, sizeof(t), cudaMemcpyDeviceToHost));
        *n_truncated = (int64_t)t;
    }
    return DP_OK;
}

// -------------------------------------------------------------- compute

static dp_status compute_args(dp_model *m, dp_nlist *nl, const double box[9], dp_precision prec)
{
    if (!m || !nl) { set_error("NULL model or list"); return DP_ERR_ARG; }
    if (nl->m != m) { set_error("the list was built for another model"); return DP_ERR_ARG; }
    if (!box) { set_error("box is NULL"); return DP_ERR_ARG; }
    if (!box_matches(nl, box)) { set_error("box differs from the list's box; build a new list"); return DP_ERR_ARG; }
    if (prec != DP_FP64 && prec != DP_MIX32 && prec != DP_MIX_BF16 && prec != DP_MIX_FP16 && prec != DP_MIX_BF16X3 &&
        prec != DP_MIX_FP8) {
        set_error("unknown precision %d", (int)prec);
        return DP_ERR_ARG;
    }
    return DP_OK;
}

dp_status dp_compute(dp_model *m, dp_nlist *nl, const double *coord, const double box[9], dp_precision prec,
                     double *energy, double *atom_energy, double *force, double *virial)
{
    DP_TRY(compute_args(m, nl, box, prec));
    const int64_t n = nl->n;
    if ((n > 0 && (!coord || !force)) || !energy) { set_error("dp_compute: NULL argument"); return DP_ERR_ARG; }
    DP_TRY(ensure_aux(m, n));
    Aux a = aux_of(m);
    cudaStream_t st = m->stream;
    if (!nl->h_io) DP_CUDA(cudaMallocHost((void **)&nl->h_io, sizeof(double) * (size_t)(7 * n + 12)));
    double *hc = nl->h_io, *hF = hc + 3 * n, *hEi = hF + 3 * n, *scal = hEi + n;   // scal [10], two int32 words
    int32_t *hfl = reinterpret_cast<int32_t *>(scal + 10);
    // the stream work of one evaluation between the pinned staging buffers
    auto body = [&]() -> dp_status {
        if (n > 0) DP_CUDA(cudaMemcpyAsync(a.coord, hc, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        DP_CUDA(cudaMemsetAsync(m->d_flag, 0, sizeof(int32_t), st));
        DP_TRY(compute_device(m, nl, a.coord, prec, a.scal, a.Ei, a.F, a.scal + 1, a.Wi, st));
        DP_TRY(check_nonfinite(a.F, 3 * n, m->d_flag, st));
        DP_TRY(check_nonfinite(a.scal, 10, m->d_flag, st));
        DP_CUDA(cudaMemcpyAsync(hfl + 1, m->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        DP_CUDA(cudaMemcpyAsync(scal, a.scal, sizeof(double) * 10, cudaMemcpyDeviceToHost, st));
        DP_CUDA(cudaMemcpyAsync(hfl, m->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (n > 0) {
            DP_CUDA(cudaMemcpyAsync(hF, a.F, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
            DP_CUDA(cudaMemcpyAsync(hEi, a.Ei, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        }
        return DP_OK;
    };
    if (n > 0) memcpy(hc, coord, sizeof(double) * 3 * n);
    // After one direct call with a key (precision, the model's buffers and parameters, the routing
    // switches) the calls are replays of one captured graph; not while profiling or with DP_NO_GRAPH.
    const bool use_graph = n > 0 && !(m->prof && m->prof->on) && getenv("DP_NO_GRAPH") == nullptr;
    const std::string env = route_env();
    if (!(nl->cgraph_prec == prec && nl->cgraph_epoch == m->epoch && nl->cgraph_env == env)) {
        nlist_graph_drop(nl);
        nl->cgraph_prec = prec;
        nl->cgraph_epoch = m->epoch;
        nl->cgraph_env = env;
        nl->cgraph_direct = 0;
    }
    if (use_graph && !nl->cgraph_exec && nl->cgraph_direct >= 1) {
        const uint64_t ep = m->epoch;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const dp_status bs = body();
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(st, &g);
            cudaGraphExec_t x = nullptr;
            const bool ok = bs == DP_OK && e == cudaSuccess && g != nullptr && m->epoch == ep &&
                            cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
            if (ok) {
                nl->cgraph = g;
                nl->cgraph_exec = x;
            } else {
                if (x) cudaGraphExecDestroy(x);
                if (g) cudaGraphDestroy(g);
                if (m->epoch != ep) {   // a buffer was set up inside the capture: redo its contents directly
                    m->oz_stale = true;
                    m->oz_emb_stale = true;
                    m->oz_fit_stale = true;
                }
                nl->cgraph_direct = -1000000;   // no further capture with this key
            }
        }
        (void)cudaGetLastError();
    }
    if (use_graph && nl->cgraph_exec) {
        DP_CUDA(cudaGraphLaunch(nl->cgraph_exec, st));
    } else {
        DP_TRY(body());
        ++nl->cgraph_direct;
    }
    DP_CUDA(cudaStreamSynchronize(st));
    const int32_t flag = hfl[0], derr = hfl[1];
    if (derr) {
        cudaMemsetAsync(m->d_err, 0, sizeof(int32_t), st);
        set_error("a bounded device wait gave up (tensor-core pipeline); results are invalid");
        return DP_ERR_TIMEOUT;
    }
    if (flag) { set_error("non-finite energy, virial or force"); return DP_ERR_NONFINITE; }
    *energy = scal[0];
    if (virial) memcpy(virial, scal + 1, 9 * sizeof(double));
    if (n > 0) memcpy(force, hF, sizeof(double) * 3 * n);
    if (atom_energy && n > 0) memcpy(atom_energy, hEi, sizeof(double) * n);
    return DP_OK;
}

dp_status dp_compute_dev(dp_model *m, dp_nlist *nl, const double *d_coord, const double box[9], dp_precision prec,
                         double *d_energy, double *d_atom_energy, double *d_force, double *d_virial, void *stream)
{
    DP_TRY(compute_args(m, nl, box, prec));
    const int64_t n = nl->n;
    if ((n > 0 && (!d_coord || !d_force)) || !d_energy) { set_error("dp_compute_dev: NULL argument"); return DP_ERR_ARG; }
    DP_TRY(ensure_aux(m, n));
    Aux a = aux_of(m);
    cudaStream_t st = (cudaStream_t)stream;
    DP_TRY(compute_device(m, nl, d_coord, prec, d_energy, d_atom_energy ? d_atom_energy : a.Ei, d_force,
                          d_virial ? d_virial : a.scal + 1, a.Wi, st));
    return DP_OK;
}

}  // extern "C"

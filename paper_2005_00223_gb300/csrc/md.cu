// Velocity-Verlet NVE on the device (Sec. 5.1): half kick, drift with
// wrapping into the box, skin-list rebuild on the device when any atom has
// moved more than skin/2 since the last build (no host round trip), force
// evaluation, half kick, and thermo rows (KE, PE, T, P) every k steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "dp_internal.cuh"
#include "geom.cuh"

namespace dp {

namespace {

constexpr double kAccel = 9.648533212e-3;   // 1 eV/(A amu) in A/fs^2
constexpr double kKB = 8.617333262e-5;      // eV/K
constexpr double kEvA3ToBar = 1.602176634e6;
constexpr int kThermoThreads = 512;

__global__ void k_kick(int64_t n, double *__restrict__ v, const double *__restrict__ f,
                       const int32_t *__restrict__ type, const double *__restrict__ minv, double half_dt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = half_dt * minv[type[i]];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[3 * i + k] += s * f[3 * i + k];
}

// The first half kick v += (dt/2) F/m, the drift x += dt v wrapped into
// [0, L) with the packed position arrays refreshed, and the displacement
// check against the list's reference positions, one atom per thread.
__global__ void k_kick_drift_check(int64_t n, double *__restrict__ v, const double *__restrict__ f,
                                   const int32_t *__restrict__ type, const double *__restrict__ minv, double half_dt,
                                   double *__restrict__ x, double dt, BoxDev bx, Pos4 *__restrict__ pos,
                                   float4 *__restrict__ posf, const Pos4 *__restrict__ ref, double lim2,
                                   int32_t *flags, unsigned long long *steps, int every)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0 && every > 0) {   // fixed-interval rebuilds: every `every`-th step builds the list again
        const unsigned long long c = *steps + 1;
        *steps = c;
        if (c % (unsigned long long)every == 0) flags[1] = 1;
    }
    if (i >= n) return;
    const int ti = type[i];
    const double s = half_dt * minv[ti];
    double p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double vk = v[3 * i + k] + s * f[3 * i + k];
        v[3 * i + k] = vk;
        double y = x[3 * i + k] + dt * vk;
        y -= bx.L[k] * floor(y * bx.invL[k]);
        x[3 * i + k] = y;
        p[k] = y;
    }
    const Pos4 pi = Pos4{p[0], p[1], p[2], (double)ti};
    pos[i] = pi;
    posf[i] = wrapped_f32(p, ti, bx);
    double d[3];
    const double r = min_image_r(ref[i], pi, bx, d);
    if (r * r > lim2) flags[1] = 1;
}

__global__ void __launch_bounds__(kThermoThreads) k_thermo(int64_t n, const double *__restrict__ v,
                                                          const int32_t *__restrict__ type,
                                                          const double *__restrict__ mass,
                                                          const double *__restrict__ scal, double vol,
                                                          double *__restrict__ row)
{
    __shared__ double s[kThermoThreads];
    const int t = threadIdx.x;
    double ke = 0.0;
    for (int64_t i = t; i < n; i += kThermoThreads) {
        double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        ke += 0.5 * mass[type[i]] * v2 / kAccel;
    }
    s[t] = ke;
    __syncthreads();
    for (int h = kThermoThreads / 2; h > 0; h >>= 1) {
        if (t < h) s[t] += s[t + h];
        __syncthreads();
    }
    if (t == 0) {
        double k = s[0];
        row[0] = k;
        row[1] = scal[0];
        row[2] = n > 1 ? 2.0 * k / ((3.0 * n - 3.0) * kKB) : 0.0;
        row[3] = (2.0 * k + scal[1] + scal[5] + scal[9]) / (3.0 * vol) * kEvA3ToBar;
    }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// One velocity-Verlet step after the force of the previous one: half kick,
// drift and displacement check, conditional list rebuild, formatting and
// force evaluation, half kick.
dp_status md_step_body(dp_model *m, dp_md_state *s, dp_precision prec, double dt_fs, const BoxDev &bx, double lim,
                       double *Wi, cudaStream_t st)
{
    dp_nlist *nl = s->nl;
    const int64_t n = s->n;
    {
        ProfScope ps(m->prof, PG_MD, 1, st);
        DP_CUDA(cudaMemsetAsync(nl->d_flags + 1, 0, sizeof(int32_t), st));
        k_kick_drift_check<<<nblk(n), 256, 0, st>>>(n, s->d_v, s->d_f, nl->d_type, s->d_minv, 0.5 * dt_fs, s->d_x,
                                                    dt_fs, bx, (Pos4 *)nl->d_pos, (float4 *)nl->d_posf,
                                                    (const Pos4 *)nl->d_ref, lim * lim, nl->d_flags, s->d_steps,
                                                    s->rebuild_every);
    }
    DP_CUDA(cudaGetLastError());
    DP_TRY(nlist_build_device(nl, st, true));
    DP_TRY(compute_device(m, nl, nullptr, prec, s->d_scal, s->d_e, s->d_f, s->d_scal + 1, Wi, st));
    {
        ProfScope ps(m->prof, PG_MD, 1, st);
        k_kick<<<nblk(n), 256, 0, st>>>(n, s->d_v, s->d_f, nl->d_type, s->d_minv, 0.5 * dt_fs);
    }
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace

// The launches of a step depend on the routing switches read from the
// environment as well as on the model's buffers (m->epoch) and the call's
// arguments; a captured step is replayed only while all of them are those
// of its capture.
std::string route_env()
{
    std::string k;
    for (const char *v : {"DP_NO_OZAKI", "DP_OZ_MIN_ATOMS", "DP_SIMT_FIT", "DP_BATCH_ATOMS", "DP_FIT_ONE_CTA"}) {
        const char *e = getenv(v);
        k += e ? e : "-";
        k += '|';
    }
    return k;
}

namespace {

void graph_drop(dp_md_state *s)
{
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->graph_exec = nullptr;
    s->graph = nullptr;
    Prof *p = s->m ? s->m->prof : nullptr;
    for (const auto &c : s->graph_scopes) {
        if (p) {
            p->pool.push_back(c.ea);
            p->pool.push_back(c.eb);
        } else {
            cudaEventDestroy(c.ea);
            cudaEventDestroy(c.eb);
        }
    }
    s->graph_scopes.clear();
}

cudaGraphNode_t event_node(const std::vector<cudaGraphNode_t> &nodes, cudaEvent_t ev)
{
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        cudaEvent_t e = nullptr;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeEventRecord &&
            cudaGraphEventRecordNodeGetEvent(nd, &e) == cudaSuccess && e == ev)
            return nd;
    }
    return nullptr;
}

// Captures one step (md_step_body) into s->graph_exec.  Returns false, with
// the stream and the model as before, when the step cannot be captured; the
// caller then keeps launching it directly.
bool graph_capture(dp_model *m, dp_md_state *s, dp_precision prec, double dt_fs, const BoxDev &bx, double lim,
                   double *Wi, cudaStream_t st)
{
    graph_drop(s);
    Prof *p = m->prof;
    const uint64_t ep = m->epoch;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (p) {
        p->capturing = true;
        p->captured.clear();
    }
    const dp_status body = md_step_body(m, s, prec, dt_fs, bx, lim, Wi, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    std::vector<Prof::Rec> caps;
    if (p) {
        p->capturing = false;
        caps.swap(p->captured);
    }
    bool ok = body == DP_OK && e == cudaSuccess && g != nullptr && m->epoch == ep;
    cudaGraphExec_t x = nullptr;
    if (ok) ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
    std::vector<dp_md_state::GraphScope> scopes;
    if (ok && !caps.empty()) {
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        for (const Prof::Rec &r : caps) {
            dp_md_state::GraphScope c{r.g, r.n, event_node(nodes, r.a), event_node(nodes, r.b), r.a, r.b};
            ok = ok && c.na && c.nb;
            scopes.push_back(c);
        }
    }
    if (!ok) {
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        for (const Prof::Rec &r : caps) {
            p->pool.push_back(r.a);
            p->pool.push_back(r.b);
        }
        if (m->epoch != ep) {   // a buffer was set up inside the capture: redo its contents directly
            m->oz_stale = true;
            m->oz_emb_stale = true;
            m->oz_fit_stale = true;
        }
        (void)cudaGetLastError();
        return false;
    }
    s->graph = g;
    s->graph_exec = x;
    s->graph_scopes.swap(scopes);
    s->graph_prec = prec;
    s->graph_dt = dt_fs;
    s->graph_epoch = m->epoch;
    s->graph_prof = p && p->on;
    s->graph_mask = p && p->on ? p->mask : 0u;
    s->graph_env = route_env();
    return true;
}

// One replay of the captured step, its timing events pointed at fresh ones.
dp_status graph_step(dp_model *m, dp_md_state *s, cudaStream_t st)
{
    Prof *p = m->prof;
    for (const auto &c : s->graph_scopes) {
        cudaEvent_t a = p->get(), b = p->get();
        DP_CUDA(cudaGraphExecEventRecordNodeSetEvent(s->graph_exec, c.na, a));
        DP_CUDA(cudaGraphExecEventRecordNodeSetEvent(s->graph_exec, c.nb, b));
        p->pending.push_back({c.g, c.n, a, b});
    }
    DP_CUDA(cudaGraphLaunch(s->graph_exec, st));
    return DP_OK;
}

}  // namespace
}  // namespace dp

using namespace dp;

extern "C" {

void dp_md_state_destroy(dp_md_state *s)
{
    if (!s) return;
    if (s->m && s->m->stream) cudaStreamSynchronize(s->m->stream);
    graph_drop(s);
    dp_nlist_destroy(s->nl);
    cudaFree(s->d_x);
    cudaFree(s->d_v);
    cudaFree(s->d_f);
    cudaFree(s->d_minv);
    cudaFree(s->d_mass);
    cudaFree(s->d_e);
    cudaFree(s->d_scal);
    cudaFree(s->d_thermo);
    cudaFree(s->d_steps);
    delete s;
}

dp_status dp_md_set_rebuild_every(dp_md_state *s, int32_t every)
{
    if (!s || every < 0) {
        set_error("dp_md_set_rebuild_every: NULL state or negative interval");
        return DP_ERR_ARG;
    }
    cudaStream_t st = s->m->stream;
    if (every > 0 && !s->d_steps) DP_CUDA(cudaMalloc((void **)&s->d_steps, sizeof(unsigned long long)));
    if (s->d_steps) DP_CUDA(cudaMemsetAsync(s->d_steps, 0, sizeof(unsigned long long), st));
    if (every != s->rebuild_every) graph_drop(s);   // the interval is an argument of the captured step
    s->rebuild_every = every;
    DP_CUDA(cudaStreamSynchronize(st));
    return DP_OK;
}

dp_status dp_md_state_create(dp_model *m, int64_t n, const double *coord, const double *vel, const int32_t *type,
                             const double *mass_by_type, const double box[9], double skin, int32_t cand_cap,
                             dp_md_state **out)
{
    if (!m || !out || !mass_by_type || (n > 0 && (!coord || !vel || !type))) {
        set_error("dp_md_state_create: NULL argument");
        return DP_ERR_ARG;
    }
    *out = nullptr;
    for (int t = 0; t < m->ntypes; ++t)
        if (!(mass_by_type[t] > 0)) { set_error("mass of type %d is %g", t, mass_by_type[t]); return DP_ERR_ARG; }
    dp_md_state *s = new (std::nothrow) dp_md_state();
    if (!s) return DP_ERR_OOM;
    s->m = m;
    s->n = n;
    memcpy(s->box, box, sizeof(s->box));
    dp_status st = nlist_create_internal(m, n, type, box, m->rcut, skin, cand_cap, &s->nl);
    if (st != DP_OK) {
        delete s;
        return st;
    }
    int64_t nn = n > 0 ? n : 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    A((void **)&s->d_x, sizeof(double) * 3 * nn);
    A((void **)&s->d_v, sizeof(double) * 3 * nn);
    A((void **)&s->d_f, sizeof(double) * 3 * nn);
    A((void **)&s->d_e, sizeof(double) * nn);
    A((void **)&s->d_minv, sizeof(double) * kMaxTypes);
    A((void **)&s->d_mass, sizeof(double) * kMaxTypes);
    A((void **)&s->d_scal, sizeof(double) * 16);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "dp_md_state_create (allocation)");
        dp_md_state_destroy(s);
        return st;
    }
    double minv[kMaxTypes] = {0}, mass[kMaxTypes] = {0};
    for (int t = 0; t < m->ntypes; ++t) {
        mass[t] = mass_by_type[t];
        minv[t] = kAccel / mass_by_type[t];
    }
    cudaStream_t cs = m->stream;
    if (n > 0) {
        e = cudaMemcpyAsync(s->d_x, coord, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_v, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, cs);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_minv, minv, sizeof(minv), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_mass, mass, sizeof(mass), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "dp_md_state_create (upload)");
        dp_md_state_destroy(s);
        return st;
    }
    if (n > 0) {
        // initial candidate list at the starting coordinates
        dp_nlist *nl = s->nl;
        st = pack_positions(nl, s->d_x, cs);
        if (st == DP_OK) st = nlist_build_device(nl, cs, false);
        if (st == DP_OK) {
            int32_t flags[3];
            e = cudaMemcpyAsync(flags, nl->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) st = cuda_fail(e, "dp_md_state_create (build)");
            else if (flags[0] & kErrCapacity) {
                set_error("a candidate list exceeded its capacity of %d", nl->cap);
                st = DP_ERR_CAPACITY;
            }
        }
        if (st != DP_OK) {
            dp_md_state_destroy(s);
            return st;
        }
    }
    *out = s;
    return DP_OK;
}

dp_status dp_md_step(dp_model *m, dp_md_state *s, int64_t nsteps, double dt_fs, dp_precision prec,
                     int32_t thermo_every, double *thermo)
{
    if (!m || !s || s->m != m) { set_error("dp_md_step: NULL or mismatched handle"); return DP_ERR_ARG; }
    if (nsteps < 0 || !(dt_fs > 0) || !isfinite(dt_fs)) { set_error("need nsteps >= 0 and dt > 0"); return DP_ERR_ARG; }
    if (prec != DP_FP64 && prec != DP_MIX32 && prec != DP_MIX_BF16 && prec != DP_MIX_FP16 && prec != DP_MIX_BF16X3 &&
        prec != DP_MIX_FP8) {
        set_error("unknown precision %d", (int)prec);
        return DP_ERR_ARG;
    }
    const int64_t n = s->n;
    if (n == 0 || nsteps == 0) return DP_OK;
    dp_nlist *nl = s->nl;
    cudaStream_t st = m->stream;
    const int64_t rows = (thermo && thermo_every > 0) ? nsteps / thermo_every : 0;
    if (rows > s->thermo_cap) {
        DP_CUDA(cudaStreamSynchronize(st));
        cudaFree(s->d_thermo);
        s->d_thermo = nullptr;
        DP_CUDA(cudaMalloc((void **)&s->d_thermo, sizeof(double) * 4 * rows));
        s->thermo_cap = rows;
    }
    DP_TRY(ensure_aux(m, n));
    double *Wi = m->d_aux + m->aux_n;       // per-atom virial scratch (after the E_i block)
    BoxDev bx = make_box(nl);
    double vol = nl->L[0] * nl->L[1] * nl->L[2];
    DP_CUDA(cudaMemsetAsync(m->d_flag, 0, sizeof(int32_t), st));
    DP_CUDA(cudaMemsetAsync(nl->d_flags, 0, sizeof(int32_t), st));
    if (!s->forces_valid || s->forces_prec != prec) {
        DP_TRY(pack_positions(nl, s->d_x, st));
        DP_TRY(compute_device(m, nl, nullptr, prec, s->d_scal, s->d_e, s->d_f, s->d_scal + 1, Wi, st));
        s->forces_valid = true;
        s->forces_prec = prec;
    }
    const double lim = 0.5 * nl->skin;
    // Steps run as replays of one captured step (CUDA graph) unless
    // DP_NO_GRAPH is set; a step is captured after one direct step of this
    // call, so that every buffer and weight image it uses is in place.
    const bool prof_on = m->prof && m->prof->on;
    if (s->graph_exec && !(s->graph_prec == prec && s->graph_dt == dt_fs && s->graph_epoch == m->epoch &&
                           s->graph_prof == prof_on && s->graph_mask == (prof_on ? m->prof->mask : 0u) &&
                           s->graph_env == route_env()))
        graph_drop(s);
    const bool use_graph = getenv("DP_NO_GRAPH") == nullptr;
    bool can_capture = use_graph;
    int64_t row = 0;
    for (int64_t k = 1; k <= nsteps; ++k) {
        if (can_capture && !s->graph_exec && k >= 2)
            can_capture = graph_capture(m, s, prec, dt_fs, bx, lim, Wi, st);
        if (use_graph && s->graph_exec) DP_TRY(graph_step(m, s, st));
        else DP_TRY(md_step_body(m, s, prec, dt_fs, bx, lim, Wi, st));
        if (rows && k % thermo_every == 0 && row < rows) {
            ProfScope ps(m->prof, PG_THERMO, 1, st);
            k_thermo<<<1, kThermoThreads, 0, st>>>(n, s->d_v, nl->d_type, s->d_mass, s->d_scal, vol,
                                                   s->d_thermo + 4 * row);
            ++row;
        }
        DP_CUDA(cudaGetLastError());
    }
    s->step += nsteps;
    {
        ProfScope ps(m->prof, PG_CHECK, 2, st);
        DP_TRY(check_nonfinite(s->d_f, 3 * n, m->d_flag, st));
        DP_TRY(check_nonfinite(s->d_x, 3 * n, m->d_flag, st));
    }
    int32_t flag = 0, flags[3], derr = 0;
    DP_CUDA(cudaMemcpyAsync(&flag, m->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(&derr, m->d_err, sizeof(derr), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(flags, nl->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    std::vector<double> th(4 * rows);
    if (rows) DP_CUDA(cudaMemcpyAsync(th.data(), s->d_thermo, sizeof(double) * 4 * rows, cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaStreamSynchronize(st));
    if (derr) {
        cudaMemsetAsync(m->d_err, 0, sizeof(int32_t), st);
        set_error("a bounded device wait gave up during MD (tensor-core pipeline); the trajectory is invalid");
        return DP_ERR_TIMEOUT;
    }
    if (flags[0] & kErrCapacity) {
        set_error("a candidate list rebuild exceeded its capacity of %d; the trajectory after it is invalid", nl->cap);
        return DP_ERR_CAPACITY;
    }
    if (flag) { set_error("non-finite forces or coordinates during MD"); return DP_ERR_NONFINITE; }
    if (rows) memcpy(thermo, th.data(), sizeof(double) * 4 * rows);
    return DP_OK;
}

dp_status dp_md_state_save(const dp_md_state *s, const char *path)
{
    if (!s || !path) { set_error("dp_md_state_save: NULL argument"); return DP_ERR_ARG; }
    const int64_t n = s->n;
    const int nt = s->m->ntypes;
    cudaStream_t st = s->m->stream;
    std::vector<double> buf(9 + 9 + nt + 10 * (size_t)n, 0.0);
    double *h = buf.data();
    double *box = h + 9, *mass = box + 9, *ty = mass + nt, *x = ty + n, *v = x + 3 * n, *f = v + 3 * n;
    std::vector<int32_t> type(n > 0 ? n : 1);
    DP_CUDA(cudaStreamSynchronize(st));
    if (n > 0) {
        DP_CUDA(cudaMemcpy(type.data(), s->nl->d_type, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        DP_CUDA(cudaMemcpy(x, s->d_x, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
        DP_CUDA(cudaMemcpy(v, s->d_v, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
        if (s->forces_valid) DP_CUDA(cudaMemcpy(f, s->d_f, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    }
    DP_CUDA(cudaMemcpy(mass, s->d_mass, sizeof(double) * nt, cudaMemcpyDeviceToHost));
    const double hdr[9] = {(double)0x44504d44, 1.0, (double)n, (double)nt, (double)s->step, s->nl->skin,
                           (double)s->nl->cap, s->forces_valid ? 1.0 : 0.0, (double)s->forces_prec};
    memcpy(h, hdr, sizeof(hdr));
    memcpy(box, s->box, sizeof(double) * 9);
    for (int64_t i = 0; i < n; ++i) ty[i] = (double)type[i];
    FILE *fp = fopen(path, "wb");
    if (!fp) { set_error("dp_md_state_save: cannot open %s", path); return DP_ERR_ARG; }
    const size_t wrote = fwrite(h, sizeof(double), buf.size(), fp);
    const bool ok = fclose(fp) == 0 && wrote == buf.size();
    if (!ok) { set_error("dp_md_state_save: cannot write %s", path); return DP_ERR_ARG; }
    return DP_OK;
}

dp_status dp_md_state_load(dp_model *m, const char *path, dp_md_state **out)
{
    if (!m || !path || !out) { set_error("dp_md_state_load: NULL argument"); return DP_ERR_ARG; }
    *out = nullptr;
    FILE *fp = fopen(path, "rb");
    if (!fp) { set_error("dp_md_state_load: cannot open %s", path); return DP_ERR_ARG; }
    double hdr[9];
    if (fread(hdr, sizeof(double), 9, fp) != 9 || hdr[0] != (double)0x44504d44 || hdr[1] != 1.0 || hdr[2] < 0 ||
        hdr[3] != (double)m->ntypes || hdr[2] != floor(hdr[2])) {
        fclose(fp);
        set_error("dp_md_state_load: %s is not an MD checkpoint of this model's types", path);
        return DP_ERR_ARG;
    }
    const int64_t n = hdr[2] < 2147483648.0 ? (int64_t)hdr[2] : -1;
    const int nt = m->ntypes;
    // the file must hold exactly the header and 9 + ntypes + 10 n values: checked before allocating
    long end = -1;
    if (n >= 0 && fseek(fp, 0, SEEK_END) == 0) end = ftell(fp);
    if (n < 0 || end != (long)(sizeof(double) * (9 + 9 + nt + 10 * (size_t)n)) ||
        fseek(fp, (long)(sizeof(double) * 9), SEEK_SET) != 0) {
        fclose(fp);
        set_error("dp_md_state_load: %s does not have the size its header gives", path);
        return DP_ERR_ARG;
    }
    std::vector<double> body(9 + nt + 10 * (size_t)n);
    const size_t got = fread(body.data(), sizeof(double), body.size(), fp);
    fclose(fp);
    if (got != body.size()) { set_error("dp_md_state_load: %s is truncated", path); return DP_ERR_ARG; }
    const double *box = body.data(), *mass = box + 9, *ty = mass + nt, *x = ty + n, *v = x + 3 * n, *f = v + 3 * n;
    std::vector<int32_t> type(n > 0 ? n : 1);
    for (int64_t i = 0; i < n; ++i) {
        if (!(ty[i] >= 0 && ty[i] < nt)) { set_error("dp_md_state_load: bad type of atom %lld", (long long)i); return DP_ERR_ARG; }
        type[i] = (int32_t)ty[i];
    }
    dp_md_state *s = nullptr;
    DP_TRY(dp_md_state_create(m, n, x, v, type.data(), mass, box, hdr[5], (int32_t)hdr[6], &s));
    s->step = (int64_t)hdr[4];
    if (hdr[7] == 1.0 && n > 0) {
        const cudaError_t e = cudaMemcpy(s->d_f, f, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            dp_md_state_destroy(s);
            return cuda_fail(e, "dp_md_state_load (forces)");
        }
        s->forces_valid = true;
        s->forces_prec = (dp_precision)(int)hdr[8];
    }
    *out = s;
    return DP_OK;
}

dp_status dp_md_state_get(const dp_md_state *s, double *coord, double *vel, int64_t *step, int64_t *n_rebuilds)
{
    if (!s) { set_error("dp_md_state_get: NULL state"); return DP_ERR_ARG; }
    cudaStream_t st = s->m->stream;
    DP_CUDA(cudaStreamSynchronize(st));
    if (coord && s->n) DP_CUDA(cudaMemcpy(coord, s->d_x, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost));
    if (vel && s->n) DP_CUDA(cudaMemcpy(vel, s->d_v, sizeof(double) * 3 * s->n, cudaMemcpyDeviceToHost));
    if (step) *step = s->step;
    if (n_rebuilds) {
        int32_t f[3] = {0, 0, 0};
        if (s->n) DP_CUDA(cudaMemcpy(f, s->nl->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
        *n_rebuilds = f[2];
    }
    return DP_OK;
}

}  // extern "C"

// ------------------------------------------------------------ judged MD

namespace dp {
namespace {

// Force RMSE between two force arrays (one block, fixed order): out[0] = sqrt(mean |a - b|^2 per atom).
__global__ void __launch_bounds__(512) k_force_rmse(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                                   double *__restrict__ out)
{
    __shared__ double s[512];
    const int t = threadIdx.x;
    double acc = 0.0;
    for (int64_t q = t; q < 3 * n; q += 512) {
        const double d = a[q] - b[q];
        acc += d * d;
    }
    s[t] = acc;
    __syncthreads();
    for (int h = 256; h > 0; h >>= 1) {
        if (t < h) s[t] += s[t + h];
        __syncthreads();
    }
    if (t == 0) out[0] = n > 0 ? sqrt(s[0] / (double)n) : 0.0;
}

}  // namespace
}  // namespace dp

extern "C" {

dp_status dp_md_step_judged(dp_model *student, dp_model *teacher, dp_md_state *s, int64_t nsteps, double dt_fs,
                            dp_precision student_prec, dp_precision teacher_prec, int32_t judge_every,
                            double rmse_max, double *rmse_log, int32_t *fallback_log)
{
    if (!student || !teacher || !s || s->m != student) { set_error("dp_md_step_judged: NULL or mismatched handle"); return DP_ERR_ARG; }
    if (nsteps < 0 || !(dt_fs > 0) || judge_every < 1 || !(rmse_max >= 0)) { set_error("dp_md_step_judged: bad argument"); return DP_ERR_ARG; }
    if (student->ntypes != teacher->ntypes || student->rcut != teacher->rcut || student->dev.nsel != teacher->dev.nsel) {
        set_error("student and teacher must share types, cut-off and sel");
        return DP_ERR_ARG;
    }
    for (int t = 0; t < student->ntypes; ++t)
        if (student->sel[t] != teacher->sel[t]) { set_error("student and teacher must share sel"); return DP_ERR_ARG; }
    const int64_t n = s->n;
    if (n == 0 || nsteps == 0) return DP_OK;
    // the teacher runs on the student's stream for the duration of the call
    DP_CUDA(cudaStreamSynchronize(teacher->stream));
    cudaStream_t teacher_stream = teacher->stream;
    teacher->stream = student->stream;
    struct Restore {
        dp_model *t;
        cudaStream_t s;
        ~Restore() { t->stream = s; }
    } restore{teacher, teacher_stream};
    dp_nlist *nl = s->nl;
    cudaStream_t st = student->stream;
    DP_TRY(ensure_aux(student, n));
    DP_TRY(ensure_aux(teacher, n));
    double *Wi_s = student->d_aux + student->aux_n, *Wi_t = teacher->d_aux + teacher->aux_n;
    // teacher scratch: forces, atom energies, scalars
    double *Ft = teacher->d_aux + teacher->aux_n * 10;      // F slot of the teacher's aux area
    double *Et = teacher->d_aux;                            // E_i slot
    double *St = teacher->d_aux + teacher->aux_n * 16;      // scalar slot
    BoxDev bx = make_box(nl);
    DP_CUDA(cudaMemsetAsync(student->d_flag, 0, sizeof(int32_t), st));
    DP_CUDA(cudaMemsetAsync(nl->d_flags, 0, sizeof(int32_t), st));
    bool use_teacher = false;
    // forces of the active model at the starting coordinates
    DP_TRY(pack_positions(nl, s->d_x, st));
    DP_TRY(compute_device(student, nl, nullptr, student_prec, s->d_scal, s->d_e, s->d_f, s->d_scal + 1, Wi_s, st));
    s->forces_valid = false;
    const double lim = 0.5 * nl->skin;
    int64_t win = 0;
    for (int64_t k = 1; k <= nsteps; ++k) {
        dp_model *act = use_teacher ? teacher : student;
        dp_precision ap = use_teacher ? teacher_prec : student_prec;
        double *Wi = use_teacher ? Wi_t : Wi_s;
        {
            ProfScope ps(student->prof, PG_MD, 1, st);
            DP_CUDA(cudaMemsetAsync(nl->d_flags + 1, 0, sizeof(int32_t), st));
            k_kick_drift_check<<<nblk(n), 256, 0, st>>>(n, s->d_v, s->d_f, nl->d_type, s->d_minv, 0.5 * dt_fs, s->d_x,
                                                        dt_fs, bx, (Pos4 *)nl->d_pos, (float4 *)nl->d_posf,
                                                        (const Pos4 *)nl->d_ref, lim * lim, nl->d_flags,
                                                        s->d_steps, s->rebuild_every);
        }
        DP_CUDA(cudaGetLastError());
        DP_TRY(nlist_build_device(nl, st, true));
        DP_TRY(compute_device(act, nl, nullptr, ap, s->d_scal, s->d_e, s->d_f, s->d_scal + 1, Wi, st));
        {
            ProfScope ps(student->prof, PG_MD, 1, st);
            k_kick<<<nblk(n), 256, 0, st>>>(n, s->d_v, s->d_f, nl->d_type, s->d_minv, 0.5 * dt_fs);
        }
        DP_CUDA(cudaGetLastError());
        if (k % judge_every == 0) {
            // judge: the other model at the same coordinates (formatting is shared)
            double *Fo = s->d_f;                            // forces of the model that drove this step
            double *Fs = use_teacher ? Ft : s->d_f;
            double *Fteach = use_teacher ? s->d_f : Ft;
            if (use_teacher) {
                DP_TRY(compute_device(student, nl, nullptr, student_prec, St + 1, Et, Ft, St + 2, Wi_s, st,
                                      !format_shared(teacher, teacher_prec, student, student_prec)));
            } else {
                DP_TRY(compute_device(teacher, nl, nullptr, teacher_prec, St + 1, Et, Ft, St + 2, Wi_t, st,
                                      !format_shared(student, student_prec, teacher, teacher_prec)));
            }
            k_force_rmse<<<1, 512, 0, st>>>(n, Fs, Fteach, St);
            DP_CUDA(cudaGetLastError());
            double rmse = 0.0;
            DP_CUDA(cudaMemcpyAsync(&rmse, St, sizeof(double), cudaMemcpyDeviceToHost, st));
            DP_CUDA(cudaStreamSynchronize(st));
            const bool next_teacher = !(rmse <= rmse_max);
            if (rmse_log) rmse_log[win] = rmse;
            if (fallback_log) fallback_log[win] = next_teacher ? 1 : 0;
            ++win;
            if (next_teacher != use_teacher) {
                // the next step starts from the newly active model's forces at these coordinates
                DP_CUDA(cudaMemcpyAsync(s->d_f, Fo == Fs ? Fteach : Fs, sizeof(double) * 3 * n,
                                        cudaMemcpyDeviceToDevice, st));
            }
            use_teacher = next_teacher;
        }
    }
    s->step += nsteps;
    int32_t flags[3], flag = 0, derr = 0;
    DP_TRY(check_nonfinite(s->d_x, 3 * n, student->d_flag, st));
    DP_CUDA(cudaMemcpyAsync(flags, nl->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(&flag, student->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(&derr, student->d_err, sizeof(derr), cudaMemcpyDeviceToHost, st));
    int32_t derr2 = 0;
    DP_CUDA(cudaMemcpyAsync(&derr2, teacher->d_err, sizeof(derr2), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaStreamSynchronize(st));
    if (derr || derr2) { set_error("a bounded device wait gave up during MD"); return DP_ERR_TIMEOUT; }
    if (flags[0] & kErrCapacity) { set_error("a candidate list rebuild exceeded its capacity"); return DP_ERR_CAPACITY; }
    if (flag) { set_error("non-finite coordinates during MD"); return DP_ERR_NONFINITE; }
    return DP_OK;
}

}  // extern "C"

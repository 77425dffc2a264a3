// Tracing: CUDA-event timing of kernel launch groups (dp_profile_*), and the
// caller-selected stream (dp_model_set_stream).
#include <cuda_runtime.h>

#include "dp_internal.cuh"

namespace dp {

cudaEvent_t Prof::get()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Prof::drain()
{
    for (const Rec &r : pending) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.g] += t;
        launches[r.g] += r.n;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}

void Prof::clear()
{
    for (const Rec &r : pending) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    for (int g = 0; g < PG_COUNT; ++g) {
        launches[g] = 0;
        ms[g] = 0.0;
    }
}

Prof::~Prof()
{
    clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

// While a stream is captured into a graph the events become event-record
// nodes of the graph (cudaEventRecordExternal); the MD loop points them at
// fresh events before every replay.
static void record(const Prof *p, cudaEvent_t e, cudaStream_t st)
{
    if (p->capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

ProfScope::ProfScope(Prof *p_, int g_, int n_, cudaStream_t st_) : p(p_), g(g_), n(n_), st(st_)
{
    if (p && p->on && (p->mask >> g & 1u)) {
        a = p->get();
        record(p, a, st);
    }
}

ProfScope::~ProfScope()
{
    if (a) {
        cudaEvent_t b = p->get();
        record(p, b, st);
        (p->capturing ? p->captured : p->pending).push_back({g, n, a, b});
    }
}

}  // namespace dp

using namespace dp;

static const char *kGroupNames[PG_COUNT] = {"nlist_build", "nlist_format", "pack", "embed_fwd", "fitting",
                                             "embed_bwd", "reduce", "md_update", "thermo", "nonfinite_check",
                                             "tc_worklist", "descriptor", "param_grad", "optimizer",
                                             "embed_fwd_l2", "embed_bwd_l2"};

extern "C" {

dp_status dp_test_starve_wait(dp_model *m, int32_t which, int64_t polls)
{
    if (!m) {
        set_error("dp_test_starve_wait: NULL model");
        return DP_ERR_ARG;
    }
    if (which != WT_NONE && which != WT_EMBED_FWD_WEIGHTS) {
        set_error("dp_test_starve_wait: unknown wait %d", (int)which);
        return DP_ERR_ARG;
    }
    if (which != WT_NONE && (polls < 1 || polls > (1LL << 20))) {
        set_error("dp_test_starve_wait: polls must be 1 .. 2^20");
        return DP_ERR_ARG;
    }
    m->dev.wait_test = which;
    m->dev.wait_short = which == WT_NONE ? 0 : polls;
    ++m->epoch;   // captured graphs hold the old kernel arguments
    return DP_OK;
}

int32_t dp_bounds_checked(void)
{
#ifdef DP_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

dp_status dp_bounds_read(int64_t *rec, int32_t clear)
{
    if (!rec) {
        set_error("dp_bounds_read: NULL record");
        return DP_ERR_ARG;
    }
    DP_CUDA(cudaDeviceSynchronize());
    cudaError_t (*const readers[])(unsigned long long *, bool) = {
        bounds_read_nlist, bounds_read_simt, bounds_read_oz_embed, bounds_read_tc,
        bounds_read_tc_x3, bounds_read_wide, bounds_read_grad};
    unsigned long long total = 0, first[4] = {0ull, 0ull, 0ull, 0ull};
    for (auto rd : readers) {
        unsigned long long r[4];
        DP_CUDA(rd(r, clear != 0));
        if (r[0] && !total) {
            for (int k = 1; k < 4; ++k) first[k] = r[k];
        }
        total += r[0];
    }
    rec[0] = (int64_t)total;
    for (int k = 1; k < 4; ++k) rec[k] = (int64_t)first[k];
    return DP_OK;
}

dp_status dp_model_set_stream(dp_model *m, void *stream)
{
    if (!m) {
        set_error("dp_model_set_stream: NULL model");
        return DP_ERR_ARG;
    }
    DP_CUDA(cudaStreamSynchronize(m->stream));
    m->stream = stream ? (cudaStream_t)stream : m->own_stream;
    return DP_OK;
}

dp_status dp_model_set_deterministic(dp_model *m, int32_t on)
{
    if (!m || (on != 0 && on != 1)) {
        set_error("dp_model_set_deterministic: NULL model or on not 0 / 1");
        return DP_ERR_ARG;
    }
    if (m->deterministic != on) {
        m->deterministic = on;
        ++m->epoch;   // captured evaluations and MD steps are re-captured
    }
    return DP_OK;
}

dp_status dp_profile_enable(dp_model *m, int32_t on)
{
    if (!m || !m->prof) {
        set_error("dp_profile_enable: NULL model");
        return DP_ERR_ARG;
    }
    DP_CUDA(cudaStreamSynchronize(m->stream));
    m->prof->clear();
    m->prof->on = on != 0;
    return DP_OK;
}

dp_status dp_profile_select(dp_model *m, uint32_t group_mask)
{
    if (!m || !m->prof) {
        set_error("dp_profile_select: NULL model");
        return DP_ERR_ARG;
    }
    DP_CUDA(cudaStreamSynchronize(m->stream));
    m->prof->drain();
    m->prof->mask = group_mask;
    return DP_OK;
}

dp_status dp_profile_read(dp_model *m, int32_t group, int64_t *launches, double *ms)
{
    if (!m || !m->prof || group < 0 || group >= PG_COUNT) {
        set_error("dp_profile_read: bad model or group %d", group);
        return DP_ERR_ARG;
    }
    DP_CUDA(cudaStreamSynchronize(m->stream));
    m->prof->drain();
    if (launches) *launches = m->prof->launches[group];
    if (ms) *ms = m->prof->ms[group];
    return DP_OK;
}

const char *dp_profile_group_name(int32_t group)
{
    return (group >= 0 && group < PG_COUNT) ? kGroupNames[group] : nullptr;
}

}  // extern "C"

// Training entry points: parameter gradient of alpha E + beta Edot, the
// force-matching loss and its gradient, Adam on the device parameters, and
// the refresh of the derived parameter copies.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "dp_internal.cuh"

namespace dp {
namespace {

// FP32 copy and transposed copies of every parameter (same flat offsets; a
// W of fan_in x fan_out is stored transposed in pT / pT32).
__global__ void k_refresh(ModelDev md, int64_t np, const double *__restrict__ p, double *__restrict__ pT,
                          float *__restrict__ p32, float *__restrict__ pT32)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const double x = p[q];
    p32[q] = (float)x;
    int64_t base, off;
    const NetLayout *L;
    if (q < md.fit_base) {
        base = (q / md.emb.size) * md.emb.size;
        L = &md.emb;
    } else {
        base = md.fit_base + ((q - md.fit_base) / md.fit.size) * md.fit.size;
        L = &md.fit;
    }
    off = q - base;
    int64_t tq = q;
    for (int k = 0; k < L->n_layers; ++k) {
        if (off >= L->W[k] && off < L->b[k]) {
            const int64_t r = off - L->W[k];
            const int64_t a = r / L->wout[k], o = r - a * L->wout[k];
            tq = base + L->W[k] + o * L->win[k] + a;
        }
    }
    pT[tq] = x;
    pT32[tq] = (float)x;
}

__global__ void k_adam(int64_t np, double *__restrict__ p, const double *__restrict__ g, double *__restrict__ mo,
                       double *__restrict__ ve, double lr, double b1, double b2, double eps, double c1, double c2)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const double gq = g[q];
    const double mq = b1 * mo[q] + (1.0 - b1) * gq;
    const double vq = b2 * ve[q] + (1.0 - b2) * gq * gq;
    mo[q] = mq;
    ve[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrt(vq / c2) + eps);
}

// Scratch of the training calls: coord, F_ref, F, v [3n] each; E_i, Edot_i,
// W_i (9n); scalars; the loss weights [beta, alpha per frame] and the
// per-frame losses (at most n frames).
struct TScr {
    double *coord, *Fref, *F, *v, *Ei, *Edi, *Wi, *scal, *ab, *lf, *grad;
};

dp_status ensure_tscr(dp_model *m, int64_t n, TScr *t)
{
    int64_t nn = n > 0 ? n : 1;
    size_t need = (size_t)nn * (3 * 4 + 2 + 9 + 2) + 32 + 1 + (size_t)m->nparams;
    if (nn > m->tscr_n) {
        if (m->d_tscr) {
            DP_CUDA(cudaStreamSynchronize(m->stream));
            cudaFree(m->d_tscr);
            m->d_tscr = nullptr;
        }
        DP_CUDA(cudaMalloc((void **)&m->d_tscr, sizeof(double) * need));
        m->tscr_n = nn;
    }
    double *b = m->d_tscr;
    nn = m->tscr_n;
    t->coord = b; b += 3 * nn;
    t->Fref = b; b += 3 * nn;
    t->F = b; b += 3 * nn;
    t->v = b; b += 3 * nn;
    t->Ei = b; b += nn;
    t->Edi = b; b += nn;
    t->Wi = b; b += 9 * nn;
    t->scal = b; b += 32;
    t->ab = b; b += nn + 1;
    t->lf = b; b += nn;
    t->grad = b;
    return DP_OK;
}

dp_status check_args(dp_model *m, dp_nlist *nl, const double box[9])
{
    if (!m || !nl || !box) { set_error("NULL model, list or box"); return DP_ERR_ARG; }
    if (nl->m != m) { set_error("the list was built for another model"); return DP_ERR_ARG; }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (box[3 * a + b] != (a == b ? nl->L[a] : 0.0)) { set_error("box differs from the list's box"); return DP_ERR_ARG; }
    return DP_OK;
}

dp_status finish_sync(dp_model *m, cudaStream_t st)
{
    int32_t derr = 0;
    DP_CUDA(cudaMemcpyAsync(&derr, m->d_err, sizeof(derr), cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaStreamSynchronize(st));
    if (derr) {
        cudaMemset(m->d_err, 0, sizeof(int32_t));
        set_error("a bounded device wait gave up; results are invalid");
        return DP_ERR_TIMEOUT;
    }
    return DP_OK;
}

}  // namespace

dp_status refresh_params_device(dp_model *m, cudaStream_t st)
{
    ProfScope ps(m->prof, PG_OPT, 1, st);
    k_refresh<<<(unsigned)((m->nparams + 255) / 256), 256, 0, st>>>(m->dev, m->nparams, m->d_params, m->d_paramsT,
                                                                    m->d_params32, m->d_paramsT32);
    DP_CUDA(cudaGetLastError());
    return DP_OK;
}

}  // namespace dp

using namespace dp;

extern "C" {

dp_status dp_param_grad(dp_model *m, dp_nlist *nl, const double *coord, const double box[9], const double *v,
                        double alpha, double beta, dp_precision prec, double *energy, double *edot, double *grad)
{
    DP_TRY(check_args(m, nl, box));
    const int64_t n = nl->n;
    if ((n > 0 && (!coord || !v)) || !grad) { set_error("dp_param_grad: NULL argument"); return DP_ERR_ARG; }
    cudaStream_t st = m->stream;
    TScr t;
    DP_TRY(ensure_tscr(m, n, &t));
    if (n > 0) {
        DP_CUDA(cudaMemcpyAsync(t.coord, coord, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        DP_CUDA(cudaMemcpyAsync(t.v, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    }
    // weights [beta, alpha of every frame]
    std::vector<double> ab(1 + (size_t)nl->nframes, alpha);
    ab[0] = beta;
    DP_CUDA(cudaMemcpyAsync(t.ab, ab.data(), sizeof(double) * ab.size(), cudaMemcpyHostToDevice, st));
    DP_CUDA(cudaMemsetAsync(t.grad, 0, sizeof(double) * m->nparams, st));
    DP_TRY(nlist_format_device(m, nl, t.coord, st));
    if (n > 0) {
        DP_TRY(param_grad_device(m, nl, t.v, t.ab, prec, t.Ei, t.Edi, t.grad, st));
        DP_TRY(reduce_energy_virial(t.Ei, nullptr, n, t.scal, nullptr, m->d_red, st));
        DP_TRY(reduce_energy_virial(t.Edi, nullptr, n, t.scal + 1, nullptr, m->d_red, st));
    } else {
        DP_CUDA(cudaMemsetAsync(t.scal, 0, 2 * sizeof(double), st));
    }
    std::vector<double> g(m->nparams);
    double sc[2];
    DP_CUDA(cudaMemcpyAsync(g.data(), t.grad, sizeof(double) * m->nparams, cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(sc, t.scal, sizeof(sc), cudaMemcpyDeviceToHost, st));
    DP_TRY(finish_sync(m, st));
    for (int64_t q = 0; q < m->nparams; ++q) grad[q] += g[q];
    if (energy) *energy = sc[0];
    if (edot) *edot = sc[1];
    return DP_OK;
}

static dp_status loss_grad_enqueue(dp_model *m, dp_nlist *nl, const double *d_coord, const double *d_F_ref,
                                   const double *d_E_ref, double p_e, double p_f, dp_precision prec, double *d_loss,
                                   double *d_grad, cudaStream_t st)
{
    const int64_t n = nl->n;
    TScr t;
    DP_TRY(ensure_tscr(m, n, &t));
    if (n == 0) return DP_OK;
    DP_TRY(compute_device(m, nl, d_coord, prec, t.scal, t.Ei, t.F, t.scal + 1, t.Wi, st));
    DP_TRY(loss_terms_device(n, nl->frame_n, t.F, d_F_ref, t.Ei, d_E_ref, p_e, p_f, t.v, t.ab, t.lf, d_loss, st));
    return param_grad_device(m, nl, t.v, t.ab, prec, t.Ei, t.Edi, d_grad, st);
}

dp_status dp_force_loss_grad(dp_model *m, dp_nlist *nl, const double *coord, const double box[9],
                             const double *F_ref, double E_ref, double p_e, double p_f, dp_precision prec,
                             double *loss, double *grad)
{
    DP_TRY(check_args(m, nl, box));
    const int64_t n = nl->n;
    if ((n > 0 && (!coord || !F_ref)) || !grad || !loss) { set_error("dp_force_loss_grad: NULL argument"); return DP_ERR_ARG; }
    if (nl->nframes != 1) { set_error("dp_force_loss_grad takes one configuration; use dp_force_loss_grad_dev for frames"); return DP_ERR_ARG; }
    cudaStream_t st = m->stream;
    TScr t;
    DP_TRY(ensure_tscr(m, n, &t));
    if (n > 0) {
        DP_CUDA(cudaMemcpyAsync(t.coord, coord, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
        DP_CUDA(cudaMemcpyAsync(t.Fref, F_ref, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    }
    double hs[2] = {E_ref, 0.0};
    DP_CUDA(cudaMemcpyAsync(t.scal + 16, hs, sizeof(hs), cudaMemcpyHostToDevice, st));   // E_ref, loss
    DP_CUDA(cudaMemsetAsync(t.grad, 0, sizeof(double) * m->nparams, st));
    DP_TRY(loss_grad_enqueue(m, nl, t.coord, t.Fref, t.scal + 16, p_e, p_f, prec, t.scal + 17, t.grad, st));
    std::vector<double> g(m->nparams);
    double lo = 0.0;
    DP_CUDA(cudaMemcpyAsync(g.data(), t.grad, sizeof(double) * m->nparams, cudaMemcpyDeviceToHost, st));
    DP_CUDA(cudaMemcpyAsync(&lo, t.scal + 17, sizeof(double), cudaMemcpyDeviceToHost, st));
    DP_TRY(finish_sync(m, st));
    for (int64_t q = 0; q < m->nparams; ++q) grad[q] += g[q];
    *loss += lo;
    return DP_OK;
}

dp_status dp_force_loss_grad_dev(dp_model *m, dp_nlist *nl, const double *d_coord, const double box[9],
                                 const double *d_F_ref, const double *d_E_ref, double p_e, double p_f,
                                 dp_precision prec, double *d_loss, double *d_grad, void *stream)
{
    DP_TRY(check_args(m, nl, box));
    if ((nl->n > 0 && (!d_coord || !d_F_ref || !d_E_ref)) || !d_loss || !d_grad) {
        set_error("dp_force_loss_grad_dev: NULL argument");
        return DP_ERR_ARG;
    }
    return loss_grad_enqueue(m, nl, d_coord, d_F_ref, d_E_ref, p_e, p_f, prec, d_loss, d_grad, (cudaStream_t)stream);
}

dp_status dp_adam_step(dp_model *m, const double *d_grad, double lr, double beta1, double beta2, double eps,
                       int64_t t, void *stream)
{
    if (!m || !d_grad || t < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1)) {
        set_error("dp_adam_step: bad argument");
        return DP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->d_train) {
        DP_CUDA(cudaMalloc((void **)&m->d_train, sizeof(double) * 2 * m->nparams));
        DP_CUDA(cudaMemsetAsync(m->d_train, 0, sizeof(double) * 2 * m->nparams, st));
    }
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    {
        ProfScope ps(m->prof, PG_OPT, 1, st);
        k_adam<<<(unsigned)((m->nparams + 255) / 256), 256, 0, st>>>(m->nparams, m->d_params, d_grad, m->d_train,
                                                                     m->d_train + m->nparams, lr, beta1, beta2, eps,
                                                                     c1, c2);
    }
    DP_CUDA(cudaGetLastError());
    DP_TRY(refresh_params_device(m, st));
    m->params_dirty = true;
    ++m->epoch;
    m->oz_stale = true;
    m->oz_emb_stale = true;
    m->oz_fit_stale = true;
    return DP_OK;
}

dp_status dp_model_sync_params(dp_model *m)
{
    if (!m) { set_error("dp_model_sync_params: NULL model"); return DP_ERR_ARG; }
    DP_CUDA(cudaDeviceSynchronize());
    DP_CUDA(cudaMemcpy(m->h_params.data(), m->d_params, sizeof(double) * m->nparams, cudaMemcpyDeviceToHost));
    m->params_dirty = false;
    return pack_tc_weights(m);
}

}  // extern "C"

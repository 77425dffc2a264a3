/*
 * Oracle: a plain, slow, FP64 CPU implementation of the DeepPot-SE (se_a)
 * energy / force / virial evaluation and of velocity-Verlet NVE.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this code.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through the seeded inputs of the dpsynth module.
 *
 * Every routine follows the definition of the method step by step, with no
 * blocking, fusion or reordering: loops run in index order, sums are plain
 * left-to-right sums, and the file is compiled with -ffp-contract=off so no
 * multiply-add is fused.  Parallelism (OpenMP) only spreads independent
 * atoms over threads; every floating-point reduction that mixes atoms
 * (forces, virial, total energy) runs serially in index order.
 *
 * Sections of the paper followed (Jia et al., SC20):
 *   Sec. 2 "Deep Potential Molecular Dynamics" and Fig. 1: E = sum_i E_i,
 *       E_i = N(D(R_i)); environment matrix, embedding net, descriptor,
 *       fitting net with the dense / skip-connected layers of Fig. 1(e-g);
 *       smoothness of order 2 in the coordinates.
 *   Sec. 4.1.1 "Increasing computational granularity": neighbor list sorted
 *       by type, then by distance, padded per type to sel, nearest kept on
 *       overflow.
 *   Sec. 4.1.2 "Optimization of customized TensorFlow operators": the
 *       neighbor element (type, distance, index) and its compressed key
 *       order type > floor(r * 1e8) > index.
 *   Sec. 5.1: velocity-Verlet integration.
 * Readings where the paper is silent (switching polynomial, descriptor
 * normalisation, residual rule, units) are listed in the design notes and
 * restated at each routine below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_BOX (-4)
#define ORC_ERR_MEM (-3)

/* Model description; the parameter vector is flat in the documented order:
 * embedding nets per (ti, tj) in row-major pair order, then fitting nets
 * per ti; inside a net, per layer W (fan_in x fan_out, row-major) then b. */
typedef struct {
    int32_t ntypes;
    double rcut, rcut_smth;
    const int32_t *sel;      /* [ntypes] */
    int32_t n_embed;
    const int32_t *embed;    /* [n_embed] widths after the 1-wide input */
    int32_t m2;
    int32_t n_fit;
    const int32_t *fit;      /* [n_fit] hidden widths; output width is 1 */
    const double *params;
} orc_model;

/* ---------------------------------------------------------------- layout */

static int64_t embed_net_size(const orc_model *m)
{
    int64_t sz = 0, win = 1;
    for (int k = 0; k < m->n_embed; ++k) {
        sz += win * m->embed[k] + m->embed[k];
        win = m->embed[k];
    }
    return sz;
}

static int64_t fit_net_size(const orc_model *m)
{
    int64_t sz = 0, win = (int64_t)m->embed[m->n_embed - 1] * m->m2;
    for (int k = 0; k < m->n_fit; ++k) {
        sz += win * m->fit[k] + m->fit[k];
        win = m->fit[k];
    }
    sz += win + 1;
    return sz;
}

int64_t orc_n_params(const orc_model *m)
{
    return (int64_t)m->ntypes * m->ntypes * embed_net_size(m) + (int64_t)m->ntypes * fit_net_size(m);
}

static const double *embed_net(const orc_model *m, int ti, int tj)
{
    return m->params + (int64_t)(ti * m->ntypes + tj) * embed_net_size(m);
}

static const double *fit_net(const orc_model *m, int ti)
{
    return m->params + (int64_t)m->ntypes * m->ntypes * embed_net_size(m) + (int64_t)ti * fit_net_size(m);
}

static int nsel_total(const orc_model *m)
{
    int s = 0;
    for (int t = 0; t < m->ntypes; ++t) s += m->sel[t];
    return s;
}

/* -------------------------------------------------- geometry (Sec. 4.1.2) */

/* Orthorhombic box check: off-diagonal entries must be zero. */
static int box_lengths(const double *box, double L[3], double invL[3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && box[3 * a + b] != 0.0) return ORC_ERR_BOX;
    for (int a = 0; a < 3; ++a) {
        L[a] = box[4 * a];
        if (!(L[a] > 0.0)) return ORC_ERR_BOX;
        invL[a] = 1.0 / L[a];
    }
    return ORC_OK;
}

/* Minimum-image difference d = r_j - r_i:  d_k -= L_k * rint(d_k / L_k),
 * with the reciprocal 1/L_k taken once; rint rounds half to even. */
void orc_minimg(const double L[3], const double invL[3], const double *ri, const double *rj, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        double dk = rj[k] - ri[k];
        double nk = rint(dk * invL[k]);
        d[k] = dk - L[k] * nk;
    }
}

/* |d| with the fixed operation order (dx*dx + dy*dy) + dz*dz, then IEEE sqrt. */
double orc_norm(const double d[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return sqrt(r2);
}

/* ---------------------------------------- neighbor list (Sec. 4.1.1-4.1.2) */

typedef struct {
    int32_t type;
    uint64_t q;    /* floor(|r_ij| * 1e8) */
    int64_t j;
} orc_nbr;

/* Order of the compressed neighbor element: type first, then the truncated
 * distance floor(r * 1e8), then the atom index. */
static int nbr_cmp(const void *pa, const void *pb)
{
    const orc_nbr *a = (const orc_nbr *)pa, *b = (const orc_nbr *)pb;
    if (a->type != b->type) return a->type < b->type ? -1 : 1;
    if (a->q != b->q) return a->q < b->q ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    return 0;
}

/* Format one atom's list from a set of candidate indices: keep j != i with
 * min-image r < rcut (strict), sort by (type, floor(r*1e8), j), keep the
 * first sel_t of each type block, pad the rest with -1.  Returns the number
 * of neighbors dropped by truncation; counts[t] receives the real count of
 * type t before truncation (may be NULL). */
static int64_t format_row(const orc_model *m, int64_t i, int64_t ncand, const int64_t *cand,
                          const double *coord, const int32_t *type, const double L[3], const double invL[3],
                          orc_nbr *buf, int32_t *row, int32_t *counts)
{
    int64_t cnt = 0;
    for (int64_t c = 0; c < ncand; ++c) {
        int64_t j = cand[c];
        if (j == i) continue;
        double d[3];
        orc_minimg(L, invL, coord + 3 * i, coord + 3 * j, d);
        double r = orc_norm(d);
        if (!(r < m->rcut)) continue;
        buf[cnt].type = type[j];
        buf[cnt].q = (uint64_t)floor(r * 1e8);
        buf[cnt].j = j;
        ++cnt;
    }
    qsort(buf, (size_t)cnt, sizeof(orc_nbr), nbr_cmp);
    int nsel = nsel_total(m);
    for (int s = 0; s < nsel; ++s) row[s] = -1;
    int64_t dropped = 0, k = 0;
    int off = 0;
    for (int t = 0; t < m->ntypes; ++t) {
        int64_t ct = 0;
        while (k < cnt && buf[k].type == t) {
            if (ct < m->sel[t]) row[off + ct] = (int32_t)buf[k].j;
            ++ct;
            ++k;
        }
        if (ct > m->sel[t]) dropped += ct - m->sel[t];
        if (counts) counts[t] = (int32_t)ct;
        off += m->sel[t];
    }
    return dropped;
}

/* Formatted neighbor list of all atoms.  Candidates are either every atom
 * (use_cells = 0, the O(N^2) definition) or the atoms of the surrounding
 * cells of a cell grid with cell edge >= rcut (use_cells = 1).  Either way
 * the result is the unique canonical list.  nlist is [n][sum(sel)]. */
int orc_nlist(const orc_model *m, int64_t n, const double *coord, const int32_t *type, const double *box,
              int use_cells, int32_t *nlist, int64_t *n_truncated, int32_t *counts)
{
    double L[3], invL[3];
    if (box_lengths(box, L, invL) != ORC_OK) return ORC_ERR_BOX;
    for (int k = 0; k < 3; ++k)
        if (!(m->rcut < 0.5 * L[k])) return ORC_ERR_BOX;
    int nsel = nsel_total(m);
    int nc[3] = {1, 1, 1};
    int64_t *cell_start = NULL, *cell_atoms = NULL;
    if (use_cells) {
        for (int k = 0; k < 3; ++k) {
            nc[k] = (int)floor(L[k] / m->rcut);
            if (nc[k] < 1) nc[k] = 1;
        }
        int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
        cell_start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
        cell_atoms = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        int64_t *fill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
        if (!cell_start || !cell_atoms || !cell_of || !fill) return ORC_ERR_MEM;
        for (int64_t i = 0; i < n; ++i) {
            int c3[3];
            for (int k = 0; k < 3; ++k) {
                double f = coord[3 * i + k] * invL[k];
                f -= floor(f);
                int c = (int)(f * nc[k]);
                if (c >= nc[k]) c = nc[k] - 1;
                if (c < 0) c = 0;
                c3[k] = c;
            }
            cell_of[i] = ((int64_t)c3[0] * nc[1] + c3[1]) * nc[2] + c3[2];
            cell_start[cell_of[i] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
        for (int64_t i = 0; i < n; ++i) cell_atoms[cell_start[cell_of[i]] + fill[cell_of[i]]++] = i;
        free(cell_of);
        free(fill);
    }
    int64_t total_drop = 0;
    int err = ORC_OK;
#pragma omp parallel reduction(+ : total_drop)
    {
        orc_nbr *buf = (orc_nbr *)malloc(sizeof(orc_nbr) * (size_t)(n > 0 ? n : 1));
        int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!buf || !cand) {
#pragma omp atomic write
            err = ORC_ERR_MEM;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < n; ++i) {
                int64_t nc_i = 0;
                if (!use_cells) {
                    for (int64_t j = 0; j < n; ++j) cand[nc_i++] = j;
                } else {
                    int c3[3];
                    for (int k = 0; k < 3; ++k) {
                        double f = coord[3 * i + k] * invL[k];
                        f -= floor(f);
                        int c = (int)(f * nc[k]);
                        if (c >= nc[k]) c = nc[k] - 1;
                        if (c < 0) c = 0;
                        c3[k] = c;
                    }
                    /* distinct neighbor cells: -1..1 when the grid has >= 3
                     * cells along an axis, else every cell of that axis */
                    int lo[3], hi[3];
                    for (int k = 0; k < 3; ++k) {
                        if (nc[k] >= 3) { lo[k] = -1; hi[k] = 1; }
                        else { lo[k] = -c3[k]; hi[k] = nc[k] - 1 - c3[k]; }
                    }
                    for (int a = lo[0]; a <= hi[0]; ++a)
                        for (int b = lo[1]; b <= hi[1]; ++b)
                            for (int c = lo[2]; c <= hi[2]; ++c) {
                                int x = (c3[0] + a + nc[0]) % nc[0];
                                int y = (c3[1] + b + nc[1]) % nc[1];
                                int z = (c3[2] + c + nc[2]) % nc[2];
                                int64_t cell = ((int64_t)x * nc[1] + y) * nc[2] + z;
                                for (int64_t p = cell_start[cell]; p < cell_start[cell + 1]; ++p)
                                    cand[nc_i++] = cell_atoms[p];
                            }
                }
                total_drop += format_row(m, i, nc_i, cand, coord, type, L, invL, buf,
                                         nlist + i * nsel, counts ? counts + i * m->ntypes : NULL);
            }
        }
        free(buf);
        free(cand);
    }
    free(cell_start);
    free(cell_atoms);
    if (n_truncated) *n_truncated = total_drop;
    return err;
}

/* -------------------------------------- switching function (Sec. 2, Fig. 1) */

/* s(r): 1/r below r_cs; (1/r) * (u^3 (-6u^2 + 15u - 10) + 1) with
 * u = (r - r_cs)/(r_c - r_cs) on [r_cs, r_c); 0 from r_c on.  The quintic
 * makes s twice continuously differentiable, the order the paper states.
 * *ds receives ds/dr. */
double orc_switch(double r, double rcs, double rc, double *ds)
{
    if (r < rcs) {
        if (ds) *ds = -1.0 / (r * r);
        return 1.0 / r;
    }
    if (r < rc) {
        double u = (r - rcs) / (rc - rcs);
        double poly = u * u * u * (-6.0 * u * u + 15.0 * u - 10.0) + 1.0;
        double dpoly_du = -30.0 * u * u * (u - 1.0) * (u - 1.0);
        double dpoly_dr = dpoly_du / (rc - rcs);
        if (ds) *ds = -poly / (r * r) + dpoly_dr / r;
        return poly / r;
    }
    if (ds) *ds = 0.0;
    return 0.0;
}

/* Environment-matrix row of one neighbor (Sec. 2: the row records the
 * relative position): R = (s, s dx/r, s dy/r, s dz/r) and its Jacobian
 * dR[c][k] = dR_c / dd_k (row-major 4 x 3). */
void orc_env_row(const double d[3], double rcs, double rc, double R[4], double dR[12])
{
    double r = orc_norm(d);
    double ds;
    double s = orc_switch(r, rcs, rc, &ds);
    double sr = s / r;                               /* s / r */
    double dsr_dr = ds / r - s / (r * r);            /* d(s/r)/dr */
    R[0] = s;
    for (int k = 0; k < 3; ++k) R[1 + k] = sr * d[k];
    for (int k = 0; k < 3; ++k) dR[k] = ds * d[k] / r;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k)
            dR[3 * (1 + a) + k] = (a == k ? sr : 0.0) + d[a] * dsr_dr * d[k] / r;
}

/* ------------------------------------------- nets (Fig. 1(c)-(g), Sec. 4.2) */

/* One hidden layer: z = x W + b, t = tanh(z), and the skip rule of
 * Fig. 1(e)-(g): y = x + t when fan_out = fan_in, y = (x, x) + t when
 * fan_out = 2 fan_in, y = t otherwise.  Returns the parameter stride. */
static int64_t layer_forward(int nin, int nout, const double *p, const double *x, double *t, double *y)
{
    const double *W = p, *b = p + (int64_t)nin * nout;
    for (int o = 0; o < nout; ++o) {
        double z = b[o];
        for (int k = 0; k < nin; ++k) z += x[k] * W[(int64_t)k * nout + o];
        t[o] = tanh(z);
    }
    for (int o = 0; o < nout; ++o) {
        if (nout == nin) y[o] = x[o] + t[o];
        else if (nout == 2 * nin) y[o] = x[o % nin] + t[o];
        else y[o] = t[o];
    }
    return (int64_t)nin * nout + nout;
}

/* Reverse of layer_forward: dx from dy, using t (tanh' = 1 - t^2). */
static void layer_backward(int nin, int nout, const double *p, const double *t, const double *dy,
                           double *dz, double *dx)
{
    const double *W = p;
    for (int o = 0; o < nout; ++o) dz[o] = dy[o] * (1.0 - t[o] * t[o]);
    for (int k = 0; k < nin; ++k) {
        double acc = 0.0;
        for (int o = 0; o < nout; ++o) acc += dz[o] * W[(int64_t)k * nout + o];
        if (nout == nin) acc += dy[k];
        else if (nout == 2 * nin) acc += dy[k] + dy[k + nin];
        dx[k] = acc;
    }
}

static int embed_act_size(const orc_model *m)
{
    int s = 0;
    for (int k = 0; k < m->n_embed; ++k) s += m->embed[k];
    return s;
}

/* Embedding net on the scalar s: stores every layer's t and y (y of the
 * last layer is the embedding row G). */
static void embed_forward(const orc_model *m, const double *net, double s, double *t_all, double *y_all)
{
    const double *x = &s;
    int nin = 1, off = 0;
    const double *p = net;
    for (int k = 0; k < m->n_embed; ++k) {
        int nout = m->embed[k];
        p += layer_forward(nin, nout, p, x, t_all + off, y_all + off);
        x = y_all + off;
        off += nout;
        nin = nout;
    }
}

/* dE/ds of the embedding net given dE/dG (dG has the last width). */
static double embed_backward(const orc_model *m, const double *net, const double *t_all, const double *dG,
                             double *work_a, double *work_b, double *work_z)
{
    int off_last = embed_act_size(m) - m->embed[m->n_embed - 1];
    memcpy(work_a, dG, sizeof(double) * (size_t)m->embed[m->n_embed - 1]);
    double *dy = work_a, *dx = work_b;
    int off = off_last;
    for (int k = m->n_embed - 1; k >= 0; --k) {
        int nout = m->embed[k];
        int nin = k == 0 ? 1 : m->embed[k - 1];
        const double *p = net;
        int win = 1;
        for (int q = 0; q < k; ++q) {
            p += (int64_t)win * m->embed[q] + m->embed[q];
            win = m->embed[q];
        }
        layer_backward(nin, nout, p, t_all + off, dy, work_z, dx);
        if (k > 0) off -= m->embed[k - 1];
        double *tmp = dy; dy = dx; dx = tmp;
    }
    return dy[0];
}

/* ----------------------------------------------- one atom (E_i, dE_i/dd_ij) */

typedef struct {
    double *R, *dR, *t, *y, *T, *dT, *D, *dD, *fit_t, *fit_y, *fa, *fb, *fz, *ea, *eb, *ez, *dG;
    int64_t *cand;
} orc_work;

static void work_free(orc_work *w)
{
    free(w->R); free(w->dR); free(w->t); free(w->y); free(w->T); free(w->dT); free(w->D); free(w->dD);
    free(w->fit_t); free(w->fit_y); free(w->fa); free(w->fb); free(w->fz); free(w->ea); free(w->eb);
    free(w->ez); free(w->dG);
}

static int work_alloc(const orc_model *m, orc_work *w)
{
    int nsel = nsel_total(m), na = embed_act_size(m), m1 = m->embed[m->n_embed - 1];
    int nd = m1 * m->m2, nf = 0, maxf = nd;
    for (int k = 0; k < m->n_fit; ++k) { nf += m->fit[k]; if (m->fit[k] > maxf) maxf = m->fit[k]; }
    memset(w, 0, sizeof(*w));
    w->R = malloc(sizeof(double) * 4 * nsel);
    w->dR = malloc(sizeof(double) * 12 * nsel);
    w->t = malloc(sizeof(double) * (size_t)na * nsel);
    w->y = malloc(sizeof(double) * (size_t)na * nsel);
    w->T = malloc(sizeof(double) * 4 * m1);
    w->dT = malloc(sizeof(double) * 4 * m1);
    w->D = malloc(sizeof(double) * nd);
    w->dD = malloc(sizeof(double) * nd);
    w->fit_t = malloc(sizeof(double) * (nf + 1));
    w->fit_y = malloc(sizeof(double) * (nf + 1));
    w->fa = malloc(sizeof(double) * (maxf + 1));
    w->fb = malloc(sizeof(double) * (maxf + 1));
    w->fz = malloc(sizeof(double) * (maxf + 1));
    w->ea = malloc(sizeof(double) * (na + 1));
    w->eb = malloc(sizeof(double) * (na + 1));
    w->ez = malloc(sizeof(double) * (na + 1));
    w->dG = malloc(sizeof(double) * m1);
    if (!w->R || !w->dR || !w->t || !w->y || !w->T || !w->dT || !w->D || !w->dD || !w->fit_t || !w->fit_y ||
        !w->fa || !w->fb || !w->fz || !w->ea || !w->eb || !w->ez || !w->dG) {
        work_free(w);
        return ORC_ERR_MEM;
    }
    return ORC_OK;
}

/* E_i and g_ij = dE_i/dd_ij (d_ij = r_j - r_i, min image) for every slot of
 * atom i's formatted list row (padded slots get g = 0).
 *   T = (1/sum(sel)) sum_j G_j^T R_j         (M1 x 4, sum over real slots)
 *   D[a][b] = sum_c T[a][c] T[b][c], b < M2   (flattened a*M2 + b)
 *   E_i = fitting net of type(i) on D
 * then the chain rule backwards through the same steps. */
static int atom_eval(const orc_model *m, int64_t i, const int32_t *row, const double *coord, const int32_t *type,
                     const double L[3], const double invL[3], orc_work *w, double *Ei, double *g, double *Dout,
                     double *d_out)
{
    int nsel = nsel_total(m), na = embed_act_size(m), m1 = m->embed[m->n_embed - 1], m2 = m->m2;
    int ti = type[i];
    double inv_nsel = 1.0 / (double)nsel;
    /* environment rows */
    for (int s = 0; s < nsel; ++s) {
        int32_t j = row[s];
        if (j < 0) {
            for (int c = 0; c < 4; ++c) w->R[4 * s + c] = 0.0;
            for (int c = 0; c < 12; ++c) w->dR[12 * s + c] = 0.0;
            if (d_out) d_out[3 * s] = d_out[3 * s + 1] = d_out[3 * s + 2] = 0.0;
            continue;
        }
        double d[3];
        orc_minimg(L, invL, coord + 3 * i, coord + 3 * (int64_t)j, d);
        orc_env_row(d, m->rcut_smth, m->rcut, w->R + 4 * s, w->dR + 12 * s);
        if (d_out) { d_out[3 * s] = d[0]; d_out[3 * s + 1] = d[1]; d_out[3 * s + 2] = d[2]; }
    }
    /* embedding rows and T */
    for (int q = 0; q < 4 * m1; ++q) w->T[q] = 0.0;
    int off = 0;
    for (int tj = 0; tj < m->ntypes; ++tj) {
        const double *net = embed_net(m, ti, tj);
        for (int s = off; s < off + m->sel[tj]; ++s) {
            if (row[s] < 0) continue;
            embed_forward(m, net, w->R[4 * s], w->t + (int64_t)s * na, w->y + (int64_t)s * na);
            const double *G = w->y + (int64_t)s * na + (na - m1);
            for (int a = 0; a < m1; ++a)
                for (int c = 0; c < 4; ++c) w->T[4 * a + c] += G[a] * w->R[4 * s + c];
        }
        off += m->sel[tj];
    }
    for (int q = 0; q < 4 * m1; ++q) w->T[q] *= inv_nsel;
    /* descriptor */
    for (int a = 0; a < m1; ++a)
        for (int b = 0; b < m2; ++b) {
            double acc = 0.0;
            for (int c = 0; c < 4; ++c) acc += w->T[4 * a + c] * w->T[4 * b + c];
            w->D[a * m2 + b] = acc;
        }
    if (Dout) memcpy(Dout, w->D, sizeof(double) * (size_t)m1 * m2);
    /* fitting net forward */
    const double *p = fit_net(m, ti);
    const double *x = w->D;
    int nin = m1 * m2, foff = 0;
    for (int k = 0; k < m->n_fit; ++k) {
        int nout = m->fit[k];
        p += layer_forward(nin, nout, p, x, w->fit_t + foff, w->fit_y + foff);
        x = w->fit_y + foff;
        foff += nout;
        nin = nout;
    }
    const double *Wout = p, *bout = p + nin;
    double e = bout[0];
    for (int k = 0; k < nin; ++k) e += x[k] * Wout[k];
    *Ei = e;
    if (!g) return ORC_OK;
    /* fitting net backward: dE/dD */
    double *dy = w->fa;
    for (int k = 0; k < nin; ++k) dy[k] = Wout[k];
    for (int k = m->n_fit - 1; k >= 0; --k) {
        int nout = m->fit[k];
        int kin = k == 0 ? m1 * m2 : m->fit[k - 1];
        const double *pk = fit_net(m, ti);
        int win = m1 * m2;
        for (int q = 0; q < k; ++q) { pk += (int64_t)win * m->fit[q] + m->fit[q]; win = m->fit[q]; }
        foff -= nout;
        double *dx = (k == 0) ? w->dD : (dy == w->fa ? w->fb : w->fa);
        layer_backward(kin, nout, pk, w->fit_t + foff, dy, w->fz, dx);
        dy = dx;
    }
    /* dE/dT[a][c] = sum_b dD[a][b] T[b][c] + [a < M2] sum_a' dD[a'][a] T[a'][c] */
    for (int a = 0; a < m1; ++a)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int b = 0; b < m2; ++b) acc += w->dD[a * m2 + b] * w->T[4 * b + c];
            if (a < m2)
                for (int a2 = 0; a2 < m1; ++a2) acc += w->dD[a2 * m2 + a] * w->T[4 * a2 + c];
            w->dT[4 * a + c] = acc;
        }
    /* per slot: dE/dG_j, dE/dR_j, back through the embedding net, then d */
    off = 0;
    for (int tj = 0; tj < m->ntypes; ++tj) {
        const double *net = embed_net(m, ti, tj);
        for (int s = off; s < off + m->sel[tj]; ++s) {
            double *gs = g + 3 * s;
            gs[0] = gs[1] = gs[2] = 0.0;
            if (row[s] < 0) continue;
            const double *R = w->R + 4 * s;
            const double *G = w->y + (int64_t)s * na + (na - m1);
            for (int a = 0; a < m1; ++a) {
                double acc = 0.0;
                for (int c = 0; c < 4; ++c) acc += w->dT[4 * a + c] * R[c];
                w->dG[a] = acc * inv_nsel;
            }
            double dRr[4];
            for (int c = 0; c < 4; ++c) {
                double acc = 0.0;
                for (int a = 0; a < m1; ++a) acc += w->dT[4 * a + c] * G[a];
                dRr[c] = acc * inv_nsel;
            }
            double ds = embed_backward(m, net, w->t + (int64_t)s * na, w->dG, w->ea, w->eb, w->ez);
            dRr[0] += ds;
            const double *J = w->dR + 12 * s;
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int c = 0; c < 4; ++c) acc += dRr[c] * J[3 * c + k];
                gs[k] = acc;
            }
        }
        off += m->sel[tj];
    }
    return ORC_OK;
}

/* E_i, g_ij and (optionally) D of one atom, for sampled checks. */
int orc_atom(const orc_model *m, int64_t i, const int32_t *row, const double *coord, const int32_t *type,
             const double *box, double *Ei, double *g, double *D)
{
    double L[3], invL[3];
    if (box_lengths(box, L, invL) != ORC_OK) return ORC_ERR_BOX;
    orc_work w;
    if (work_alloc(m, &w) != ORC_OK) return ORC_ERR_MEM;
    int st = atom_eval(m, i, row, coord, type, L, invL, &w, Ei, g, D, NULL);
    work_free(&w);
    return st;
}

/* Energy, per-atom energies, forces and virial of the whole system.
 *   E = sum_i E_i (index order)
 *   F_i += g_ij,  F_j -= g_ij    (F = -dE/dr, g_ij = dE_i/dd_ij)
 *   W_ab = -sum_ij d_ij,a g_ij,b
 * Atoms are evaluated in parallel in blocks; every sum that mixes atoms is
 * done serially in index order afterwards.  Any output may be NULL. */
int orc_compute(const orc_model *m, int64_t n, const double *coord, const int32_t *type, const double *box,
                const int32_t *nlist, double *E, double *Ei_out, double *F, double *W, int nthreads)
{
    double L[3], invL[3];
    if (box_lengths(box, L, invL) != ORC_OK) return ORC_ERR_BOX;
    int nsel = nsel_total(m);
    const int64_t BLK = 2048;
    double *gb = (double *)malloc(sizeof(double) * (size_t)BLK * nsel * 3);
    double *db = (double *)malloc(sizeof(double) * (size_t)BLK * nsel * 3);
    double *eb = (double *)malloc(sizeof(double) * (size_t)BLK);
    if (!gb || !db || !eb) { free(gb); free(db); free(eb); return ORC_ERR_MEM; }
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    double esum = 0.0, wsum[9] = {0};
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t i0 = 0; i0 < n; i0 += BLK) {
        int64_t nb = n - i0 < BLK ? n - i0 : BLK;
#pragma omp parallel
        {
            orc_work w;
            int ok = work_alloc(m, &w) == ORC_OK;
            if (!ok) {
#pragma omp atomic write
                err = ORC_ERR_MEM;
            }
#pragma omp for schedule(dynamic, 4)
            for (int64_t b = 0; b < nb; ++b) {
                if (!ok) continue;
                int64_t i = i0 + b;
                atom_eval(m, i, nlist + i * nsel, coord, type, L, invL, &w, eb + b,
                          (F || W) ? gb + b * nsel * 3 : NULL, NULL, db + b * nsel * 3);
            }
            if (ok) work_free(&w);
        }
        if (err != ORC_OK) break;
        for (int64_t b = 0; b < nb; ++b) {
            int64_t i = i0 + b;
            esum += eb[b];
            if (Ei_out) Ei_out[i] = eb[b];
            if (!(F || W)) continue;
            const int32_t *row = nlist + i * nsel;
            for (int s = 0; s < nsel; ++s) {
                if (row[s] < 0) continue;
                const double *g = gb + (b * nsel + s) * 3;
                const double *d = db + (b * nsel + s) * 3;
                if (F) {
                    for (int k = 0; k < 3; ++k) {
                        F[3 * i + k] += g[k];
                        F[3 * (int64_t)row[s] + k] -= g[k];
                    }
                }
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) wsum[3 * a + c] -= d[a] * g[c];
            }
        }
    }
    free(gb); free(db); free(eb);
    if (err != ORC_OK) return err;
    if (E) *E = esum;
    if (W) memcpy(W, wsum, sizeof(wsum));
    return ORC_OK;
}

/* -------------------------------------------- velocity-Verlet NVE (Sec. 5.1) */

/* Units: A, fs, amu, eV.  a = F/m * 9.648533212e-3 A/fs^2;
 * KE = 1/2 m v^2 / 9.648533212e-3 eV; T = 2 KE / ((3N - 3) k_B);
 * P = (2 KE + tr W) / (3 V) eV/A^3, reported in bar (x 1.602176634e6).
 * Each step: v += dt/2 a; x += dt v; x wrapped into [0, L); F(x) from a
 * freshly built exact neighbor list; v += dt/2 a.  Thermo rows (KE, PE, T,
 * P) are written after every thermo_every-th step. */
int orc_md_nve(const orc_model *m, int64_t n, double *coord, double *vel, const int32_t *type,
               const double *mass_by_type, const double *box, int64_t nsteps, double dt, int32_t thermo_every,
               double *thermo, int nthreads)
{
    const double ACC = 9.648533212e-3, KB = 8.617333262e-5, EV_A3_TO_BAR = 1.602176634e6;
    double L[3], invL[3];
    if (box_lengths(box, L, invL) != ORC_OK) return ORC_ERR_BOX;
    int nsel = nsel_total(m);
    int32_t *nl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * nsel);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!nl || !F) { free(nl); free(F); return ORC_ERR_MEM; }
    double E, W[9];
    int st = orc_nlist(m, n, coord, type, box, 1, nl, NULL, NULL);
    if (st == ORC_OK) st = orc_compute(m, n, coord, type, box, nl, &E, NULL, F, W, nthreads);
    int64_t row = 0;
    for (int64_t step = 1; st == ORC_OK && step <= nsteps; ++step) {
        for (int64_t i = 0; i < n; ++i) {
            double minv = ACC / mass_by_type[type[i]];
            for (int k = 0; k < 3; ++k) vel[3 * i + k] += 0.5 * dt * F[3 * i + k] * minv;
        }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                double x = coord[3 * i + k] + dt * vel[3 * i + k];
                coord[3 * i + k] = x - L[k] * floor(x * invL[k]);
            }
        st = orc_nlist(m, n, coord, type, box, 1, nl, NULL, NULL);
        if (st != ORC_OK) break;
        st = orc_compute(m, n, coord, type, box, nl, &E, NULL, F, W, nthreads);
        if (st != ORC_OK) break;
        for (int64_t i = 0; i < n; ++i) {
            double minv = ACC / mass_by_type[type[i]];
            for (int k = 0; k < 3; ++k) vel[3 * i + k] += 0.5 * dt * F[3 * i + k] * minv;
        }
        if (thermo && thermo_every > 0 && step % thermo_every == 0) {
            double ke = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double v2 = 0.0;
                for (int k = 0; k < 3; ++k) v2 += vel[3 * i + k] * vel[3 * i + k];
                ke += 0.5 * mass_by_type[type[i]] * v2 / ACC;
            }
            double vol = L[0] * L[1] * L[2];
            thermo[4 * row + 0] = ke;
            thermo[4 * row + 1] = E;
            thermo[4 * row + 2] = 2.0 * ke / ((3.0 * n - 3.0) * KB);
            thermo[4 * row + 3] = (2.0 * ke + W[0] + W[4] + W[8]) / (3.0 * vol) * EV_A3_TO_BAR;
            ++row;
        }
    }
    free(nl);
    free(F);
    return st;
}

/* ------------------------- parameter gradient of alpha E + beta Edot ------- */
/*
 * Edot = sum_k v_k . dE/dr_k is the directional derivative of E along the
 * displacement field v (forward-mode tangent): per atom i, with
 * dd_ij = v_j - v_i, the tangent of the environment row is J dd_ij, and every
 * layer carries (x, x') with z' = x' W, t' = (1 - t^2) z', y' = skip(x') + t'.
 * The force-matching loss L = p_e (dE/N)^2 + p_f/(3N) sum |F - F_ref|^2 has
 * dL/dtheta = 2 p_e dE/N^2 dE/dtheta - 2 p_f/(3N) dEdot/dtheta with
 * v = F - F_ref held fixed (F = -grad E), so the gradient of alpha E +
 * beta Edot over theta is the one primitive needed.  It is computed by
 * reverse mode through the primal and tangent programs; per layer, with
 * adjoints (y_bar, y'_bar):
 *   z'_bar = y'_bar (1 - t^2);  t_bar = y_bar + y'_bar z' (-2 t);
 *   z_bar = t_bar (1 - t^2);
 *   W_bar += x^T z_bar + x'^T z'_bar;  b_bar += z_bar;
 *   x_bar = z_bar W^T + skip^T(y_bar);  x'_bar = z'_bar W^T + skip^T(y'_bar).
 */

typedef struct {
    int nin, nout;
    const double *W, *b;
    double *Wg, *bg;
} orc_layer;

/* primal + tangent forward of one tanh layer; stores t and z' */
static void layer_fwd_tan(const orc_layer *L, const double *x, const double *xd, double *t, double *zd, double *y,
                          double *yd)
{
    for (int o = 0; o < L->nout; ++o) {
        double z = L->b[o], zdo = 0.0;
        for (int k = 0; k < L->nin; ++k) {
            z += x[k] * L->W[(int64_t)k * L->nout + o];
            zdo += xd[k] * L->W[(int64_t)k * L->nout + o];
        }
        t[o] = tanh(z);
        zd[o] = zdo;
    }
    for (int o = 0; o < L->nout; ++o) {
        double td = (1.0 - t[o] * t[o]) * zd[o];
        double sx = 0.0, sxd = 0.0;
        if (L->nout == L->nin) { sx = x[o]; sxd = xd[o]; }
        else if (L->nout == 2 * L->nin) { sx = x[o % L->nin]; sxd = xd[o % L->nin]; }
        y[o] = sx + t[o];
        yd[o] = sxd + td;
    }
}

/* reverse of layer_fwd_tan: accumulates W_bar, b_bar; writes x_bar, x'_bar */
static void layer_rev_tan(const orc_layer *L, const double *x, const double *xd, const double *t, const double *zd,
                          const double *yb, const double *ydb, double *xb, double *xdb, double *zb, double *zdb)
{
    for (int o = 0; o < L->nout; ++o) {
        double g = 1.0 - t[o] * t[o];
        zdb[o] = ydb[o] * g;
        double tb = yb[o] + ydb[o] * zd[o] * (-2.0 * t[o]);
        zb[o] = tb * g;
        L->bg[o] += zb[o];
    }
    for (int k = 0; k < L->nin; ++k)
        for (int o = 0; o < L->nout; ++o)
            L->Wg[(int64_t)k * L->nout + o] += x[k] * zb[o] + xd[k] * zdb[o];
    if (!xb) return;
    for (int k = 0; k < L->nin; ++k) {
        double a = 0.0, ad = 0.0;
        for (int o = 0; o < L->nout; ++o) {
            a += zb[o] * L->W[(int64_t)k * L->nout + o];
            ad += zdb[o] * L->W[(int64_t)k * L->nout + o];
        }
        if (L->nout == L->nin) { a += yb[k]; ad += ydb[k]; }
        else if (L->nout == 2 * L->nin) { a += yb[k] + yb[k + L->nin]; ad += ydb[k] + ydb[k + L->nin]; }
        xb[k] = a;
        xdb[k] = ad;
    }
}

/* formula(Xb, Y)[a][c] = sum_b Xb[a][b] Y[b][c] + [a < M2] sum_a' Xb[a'][a] Y[a'][c] */
static void desc_adjoint(int m1, int m2, const double *Xb, const double *Y, double *out, int accumulate)
{
    for (int a = 0; a < m1; ++a)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int b = 0; b < m2; ++b) acc += Xb[a * m2 + b] * Y[4 * b + c];
            if (a < m2)
                for (int a2 = 0; a2 < m1; ++a2) acc += Xb[a2 * m2 + a] * Y[4 * a2 + c];
            out[4 * a + c] = accumulate ? out[4 * a + c] + acc : acc;
        }
}

static void make_layers(const orc_model *m, const double *net, double *gnet, int nin, int nlayers, const int32_t *w,
                        orc_layer *out)
{
    int win = nin;
    int64_t off = 0;
    for (int k = 0; k < nlayers; ++k) {
        out[k].nin = win;
        out[k].nout = w[k];
        out[k].W = net + off;
        out[k].Wg = gnet + off;
        off += (int64_t)win * w[k];
        out[k].b = net + off;
        out[k].bg = gnet + off;
        off += w[k];
        win = w[k];
    }
    (void)m;
}

/* One atom: adds d(alpha E_i + beta Edot_i)/dtheta into g (flat parameter order);
 * returns E_i and Edot_i. */
static int atom_jvp_grad(const orc_model *m, int64_t i, const int32_t *row, const double *coord, const int32_t *type,
                         const double *v, const double L[3], const double invL[3], double alpha, double beta,
                         double *Ei, double *Edi, double *g)
{
    const int nsel = nsel_total(m), m1 = m->embed[m->n_embed - 1], m2 = m->m2, ne = m->n_embed, nf = m->n_fit;
    const int nd = m1 * m2;
    int na = 0, wmax = nd;
    for (int k = 0; k < ne; ++k) { na += m->embed[k]; if (m->embed[k] > wmax) wmax = m->embed[k]; }
    int nfa = 0;
    for (int k = 0; k < nf; ++k) { nfa += m->fit[k]; if (m->fit[k] > wmax) wmax = m->fit[k]; }
    const double inv = 1.0 / (double)nsel;
    const int ti = type[i];
    /* per-slot storage: R, Rd, then for each embedding layer t, zd, y, yd */
    double *R = calloc((size_t)nsel * 4, sizeof(double)), *Rd = calloc((size_t)nsel * 4, sizeof(double));
    double *et = malloc(sizeof(double) * (size_t)nsel * na), *ezd = malloc(sizeof(double) * (size_t)nsel * na);
    double *ey = malloc(sizeof(double) * (size_t)nsel * na), *eyd = malloc(sizeof(double) * (size_t)nsel * na);
    double *T = calloc(4 * (size_t)m1, sizeof(double)), *Td = calloc(4 * (size_t)m1, sizeof(double));
    double *Tb = calloc(4 * (size_t)m1, sizeof(double)), *Tdb = calloc(4 * (size_t)m1, sizeof(double));
    double *D = malloc(sizeof(double) * nd), *Dd = malloc(sizeof(double) * nd);
    double *ft = malloc(sizeof(double) * (nfa + 1)), *fzd = malloc(sizeof(double) * (nfa + 1));
    double *fy = malloc(sizeof(double) * (nfa + 1)), *fyd = malloc(sizeof(double) * (nfa + 1));
    double *b1 = malloc(sizeof(double) * wmax), *b2 = malloc(sizeof(double) * wmax);
    double *b3 = malloc(sizeof(double) * wmax), *b4 = malloc(sizeof(double) * wmax);
    double *zb = malloc(sizeof(double) * wmax), *zdb = malloc(sizeof(double) * wmax);
    if (!R || !Rd || !et || !ezd || !ey || !eyd || !T || !Td || !Tb || !Tdb || !D || !Dd || !ft || !fzd || !fy ||
        !fyd || !b1 || !b2 || !b3 || !b4 || !zb || !zdb)
        return ORC_ERR_MEM;
    orc_layer EL[8], FL[8];
    /* environment rows and their tangents */
    for (int s = 0; s < nsel; ++s) {
        int32_t j = row[s];
        if (j < 0) continue;
        double d[3], J[12];
        orc_minimg(L, invL, coord + 3 * i, coord + 3 * (int64_t)j, d);
        orc_env_row(d, m->rcut_smth, m->rcut, R + 4 * s, J);
        double dd[3];
        for (int k = 0; k < 3; ++k) dd[k] = v[3 * (int64_t)j + k] - v[3 * i + k];
        for (int c = 0; c < 4; ++c) Rd[4 * s + c] = J[3 * c] * dd[0] + J[3 * c + 1] * dd[1] + J[3 * c + 2] * dd[2];
    }
    /* embedding forward (primal + tangent), T and T' */
    int off = 0;
    for (int tj = 0; tj < m->ntypes; ++tj) {
        make_layers(m, embed_net(m, ti, tj), g + (embed_net(m, ti, tj) - m->params), 1, ne, m->embed, EL);
        for (int s = off; s < off + m->sel[tj]; ++s) {
            if (row[s] < 0) continue;
            const double *x = R + 4 * s, *xd = Rd + 4 * s;   /* input s and s' */
            int ao = 0;
            for (int k = 0; k < ne; ++k) {
                layer_fwd_tan(&EL[k], x, xd, et + (int64_t)s * na + ao, ezd + (int64_t)s * na + ao,
                              ey + (int64_t)s * na + ao, eyd + (int64_t)s * na + ao);
                x = ey + (int64_t)s * na + ao;
                xd = eyd + (int64_t)s * na + ao;
                ao += m->embed[k];
            }
            for (int a = 0; a < m1; ++a)
                for (int c = 0; c < 4; ++c) {
                    T[4 * a + c] += x[a] * R[4 * s + c];
                    Td[4 * a + c] += xd[a] * R[4 * s + c] + x[a] * Rd[4 * s + c];
                }
        }
        off += m->sel[tj];
    }
    for (int q = 0; q < 4 * m1; ++q) { T[q] *= inv; Td[q] *= inv; }
    for (int a = 0; a < m1; ++a)
        for (int b = 0; b < m2; ++b) {
            double acc = 0.0, accd = 0.0;
            for (int c = 0; c < 4; ++c) {
                acc += T[4 * a + c] * T[4 * b + c];
                accd += Td[4 * a + c] * T[4 * b + c] + T[4 * a + c] * Td[4 * b + c];
            }
            D[a * m2 + b] = acc;
            Dd[a * m2 + b] = accd;
        }
    /* fitting forward (primal + tangent) */
    const double *fnet = fit_net(m, ti);
    double *gfnet = g + (fnet - m->params);
    make_layers(m, fnet, gfnet, nd, nf, m->fit, FL);
    const double *x = D, *xd = Dd;
    int fo = 0;
    for (int k = 0; k < nf; ++k) {
        layer_fwd_tan(&FL[k], x, xd, ft + fo, fzd + fo, fy + fo, fyd + fo);
        x = fy + fo;
        xd = fyd + fo;
        fo += m->fit[k];
    }
    const int wl = m->fit[nf - 1];
    int64_t outW = 0;
    {
        int win = nd;
        for (int k = 0; k < nf; ++k) { outW += (int64_t)win * m->fit[k] + m->fit[k]; win = m->fit[k]; }
    }
    const double *Wout = fnet + outW, *bout = Wout + wl;
    double e = bout[0], ed = 0.0;
    for (int k = 0; k < wl; ++k) { e += x[k] * Wout[k]; ed += xd[k] * Wout[k]; }
    *Ei = e;
    *Edi = ed;
    /* reverse: output layer */
    double *Woutg = gfnet + outW;
    for (int k = 0; k < wl; ++k) Woutg[k] += alpha * x[k] + beta * xd[k];
    Woutg[wl] += alpha;
    double *yb = b1, *ydb = b2, *xb = b3, *xdb = b4;
    for (int k = 0; k < wl; ++k) { yb[k] = alpha * Wout[k]; ydb[k] = beta * Wout[k]; }
    double *Db = malloc(sizeof(double) * nd), *Ddb = malloc(sizeof(double) * nd);
    if (!Db || !Ddb) return ORC_ERR_MEM;
    for (int k = nf - 1; k >= 0; --k) {
        fo -= m->fit[k];
        const double *xk = k == 0 ? D : fy + fo - m->fit[k - 1];
        const double *xdk = k == 0 ? Dd : fyd + fo - m->fit[k - 1];
        double *oxb = k == 0 ? Db : xb, *oxdb = k == 0 ? Ddb : xdb;
        layer_rev_tan(&FL[k], xk, xdk, ft + fo, fzd + fo, yb, ydb, oxb, oxdb, zb, zdb);
        if (k > 0) {
            double *t1 = yb, *t2 = ydb;
            yb = xb; ydb = xdb; xb = t1; xdb = t2;
        }
    }
    /* descriptor and contraction adjoints */
    desc_adjoint(m1, m2, Db, T, Tb, 0);
    desc_adjoint(m1, m2, Ddb, Td, Tb, 1);
    desc_adjoint(m1, m2, Ddb, T, Tdb, 0);
    /* per slot: back through the embedding net */
    double *Gb = malloc(sizeof(double) * m1), *Gdb = malloc(sizeof(double) * m1);
    double *eb1 = malloc(sizeof(double) * wmax), *eb2 = malloc(sizeof(double) * wmax);
    double *eb3 = malloc(sizeof(double) * wmax), *eb4 = malloc(sizeof(double) * wmax);
    if (!Gb || !Gdb || !eb1 || !eb2 || !eb3 || !eb4) return ORC_ERR_MEM;
    off = 0;
    for (int tj = 0; tj < m->ntypes; ++tj) {
        make_layers(m, embed_net(m, ti, tj), g + (embed_net(m, ti, tj) - m->params), 1, ne, m->embed, EL);
        for (int s = off; s < off + m->sel[tj]; ++s) {
            if (row[s] < 0) continue;
            for (int a = 0; a < m1; ++a) {
                double acc = 0.0, accd = 0.0;
                for (int c = 0; c < 4; ++c) {
                    acc += Tb[4 * a + c] * R[4 * s + c] + Tdb[4 * a + c] * Rd[4 * s + c];
                    accd += Tdb[4 * a + c] * R[4 * s + c];
                }
                Gb[a] = acc * inv;
                Gdb[a] = accd * inv;
            }
            double *cyb = Gb, *cydb = Gdb, *cxb = eb1, *cxdb = eb2;
            int ao = na - m1;
            for (int k = ne - 1; k >= 0; --k) {
                const double *xk = k == 0 ? R + 4 * s : ey + (int64_t)s * na + ao - m->embed[k - 1];
                const double *xdk = k == 0 ? Rd + 4 * s : eyd + (int64_t)s * na + ao - m->embed[k - 1];
                layer_rev_tan(&EL[k], xk, xdk, et + (int64_t)s * na + ao, ezd + (int64_t)s * na + ao, cyb, cydb,
                              k == 0 ? NULL : cxb, k == 0 ? NULL : cxdb, eb3, eb4);
                if (k > 0) {
                    ao -= m->embed[k - 1];
                    /* the input adjoints just written become the next layer's output adjoints */
                    double *t1 = cyb, *t2 = cydb;
                    cyb = cxb; cydb = cxdb;
                    cxb = t1; cxdb = t2;
                }
            }
        }
        off += m->sel[tj];
    }
    free(R); free(Rd); free(et); free(ezd); free(ey); free(eyd); free(T); free(Td); free(Tb); free(Tdb);
    free(D); free(Dd); free(ft); free(fzd); free(fy); free(fyd); free(b1); free(b2); free(b3); free(b4);
    free(zb); free(zdb); free(Db); free(Ddb); free(Gb); free(Gdb); free(eb1); free(eb2); free(eb3); free(eb4);
    return ORC_OK;
}

/* Gradient of alpha E + beta Edot over the flat parameters (added into grad),
 * with Edot = sum_k v_k . dE/dr_k; E and Edot are returned (summed in index
 * order).  Atoms run in parallel with a private gradient per thread; the
 * private gradients are added in thread order. */
int orc_jvp_grad(const orc_model *m, int64_t n, const double *coord, const int32_t *type, const double *box,
                 const int32_t *nlist, const double *v, double alpha, double beta, double *E_out, double *Ed_out,
                 double *grad, int nthreads)
{
    double L[3], invL[3];
    if (box_lengths(box, L, invL) != ORC_OK) return ORC_ERR_BOX;
    const int nsel = nsel_total(m);
    const int64_t np = orc_n_params(m);
    double *Ei = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)), *Edi = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!Ei || !Edi) return ORC_ERR_MEM;
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    double *priv = calloc((size_t)nt * np, sizeof(double));
    if (!priv) return ORC_ERR_MEM;
    int err = ORC_OK;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gp = priv + (size_t)tid * np;
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; ++i) {
            int st = atom_jvp_grad(m, i, nlist + i * nsel, coord, type, v, L, invL, alpha, beta, Ei + i, Edi + i, gp);
            if (st != ORC_OK) {
#pragma omp atomic write
                err = st;
            }
        }
    }
    if (err == ORC_OK) {
        for (int t = 0; t < nt; ++t)
            for (int64_t q = 0; q < np; ++q) grad[q] += priv[(size_t)t * np + q];
        double e = 0.0, ed = 0.0;
        for (int64_t i = 0; i < n; ++i) { e += Ei[i]; ed += Edi[i]; }
        if (E_out) *E_out = e;
        if (Ed_out) *Ed_out = ed;
    }
    free(priv); free(Ei); free(Edi);
    return err;
}

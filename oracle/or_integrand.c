/*
 * Oracle: the per-event integrand (Sec. 2.1: random numbers to event weight) and the
 * VEGAS passes (sums, per-bin histograms, refinement, combination).
 * TEST INFRASTRUCTURE ONLY (see mf_oracle.h).
 *
 * The event pipeline runs in the order of Sec. 2.1 of the paper: random
 * numbers, VEGAS map, kinematics (parton map, RAMBO, lab boost, cuts),
 * PDFs (Sec. 1), squared matrix element (Sec. 2.2), weight, and histogram
 * accumulation.  Events are independent; the per-event weights are reduced
 * in event order afterwards.
 */
#include "mf_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static const double GEV2_TO_PB = 0.3893793721e9;   /* (hbar c)^2 in pb GeV^2 */

static void final_masses(int proc, const or_params *P, double *m, int *n)
{
    switch (proc) {
    case OR_GG_TT: case OR_UU_TT: m[0] = P->mt; m[1] = P->mt; *n = 2; break;
    case OR_GG_TTG: case OR_UG_TTU: m[0] = P->mt; m[1] = P->mt; m[2] = 0.0; *n = 3; break;
    case OR_GG_TTGG: m[0] = P->mt; m[1] = P->mt; m[2] = 0.0; m[3] = 0.0; *n = 4; break;
    case OR_GG_TTGGG: m[0] = P->mt; m[1] = P->mt; m[2] = m[3] = m[4] = 0.0; *n = 5; break;
    default: *n = 2; m[0] = m[1] = 0.0;
    }
}

/* PDF flavour index in the grid: 0 gluon, 1 u, 2 ubar */
static void pdf_flavours(int proc, int *f1, int *f2)
{
    switch (proc) {
    case OR_UU_TT: *f1 = 1; *f2 = 2; break;
    case OR_UG_TTU: *f1 = 1; *f2 = 0; break;
    default: *f1 = 0; *f2 = 0;
    }
}

int or_event(int proc, const or_params *P, const or_pdf *pdf, const double *grid,
             uint64_t event, uint32_t iteration, const int *mask_override, or_event_out *o)
{
    or_proc_info info;
    if (or_proc_info_get(proc, &info)) return 1;
    memset(o, 0, sizeof(*o));
    int D = info.dim, nb = P->n_bins;
    or_uniforms(P->seed, event, iteration, P->channel, D, o->u);
    o->jac_vegas = or_vegas_map(grid, D, nb, o->u, o->x, o->bins);

    if (proc == OR_EE_MUMU) {
        double s = P->sqrt_s * P->sqrt_s, E = 0.5 * P->sqrt_s;
        double c = 2.0 * o->x[0] - 1.0, sn = sqrt(1.0 - c * c), phi = 2.0 * M_PI * o->x[1];
        double pp[4][4] = {
            { E, 0, 0, E }, { E, 0, 0, -E },
            { E, E * sn * cos(phi), E * sn * sin(phi), E * c },
            { E, -E * sn * cos(phi), -E * sn * sin(phi), -E * c },
        };
        memcpy(o->p, pp, sizeof(pp));
        memcpy(o->plab, pp, sizeof(pp));
        o->x1 = o->x2 = 1.0; o->shat = s; o->jac_parton = 1.0;
        o->w_ps = 1.0 / (8.0 * M_PI);               /* 2-body massless, dcos dphi */
        o->mask = mask_override ? *mask_override : 1;
        o->me2 = o->mask ? or_me2(proc, P, &o->p[0][0]) : 0.0;
        o->w = o->mask ? o->me2 / (2.0 * s) * o->w_ps * o->jac_vegas * GEV2_TO_PB : 0.0;
        return 0;
    }

    double S = P->sqrt_s * P->sqrt_s;
    double m[5]; int nf;
    final_masses(proc, P, m, &nf);
    double msum = 0.0;
    for (int i = 0; i < nf; ++i) msum += m[i];
    double tau0 = msum * msum / S;
    or_parton_map(o->x[0], o->x[1], tau0, &o->x1, &o->x2, &o->jac_parton);
    o->shat = o->x1 * o->x2 * S;
    double rs = sqrt(o->shat);
    double pf[5 * 4];
    if (or_rambo(nf, rs, m, o->x + 2, pf, &o->w_ps)) { o->w = 0.0; return 0; }
    double half = 0.5 * rs;
    double pin[2][4] = { { half, 0, 0, half }, { half, 0, 0, -half } };
    memcpy(o->p[0], pin[0], sizeof(pin[0]));
    memcpy(o->p[1], pin[1], sizeof(pin[1]));
    for (int i = 0; i < nf; ++i) memcpy(o->p[2 + i], pf + 4 * i, 4 * sizeof(double));

    /* longitudinal boost to the lab: rapidity y = ln(x1/x2)/2 */
    double sq = sqrt(o->x1 * o->x2);
    double ch = (o->x1 + o->x2) / (2.0 * sq), sh = (o->x1 - o->x2) / (2.0 * sq);
    for (int i = 0; i < 2 + nf; ++i) {
        o->plab[i][0] = ch * o->p[i][0] + sh * o->p[i][3];
        o->plab[i][1] = o->p[i][1];
        o->plab[i][2] = o->p[i][2];
        o->plab[i][3] = ch * o->p[i][3] + sh * o->p[i][0];
    }
    o->mask = mask_override ? *mask_override : or_cuts(proc, P, &o->plab[0][0]);
    o->muf2 = or_muf2(proc, P, &o->p[0][0]);
    int f1, f2;
    pdf_flavours(proc, &f1, &f2);
    o->f1 = or_pdf_xf(pdf, f1, o->x1, o->muf2) / o->x1;
    o->f2 = or_pdf_xf(pdf, f2, o->x2, o->muf2) / o->x2;
    if (!o->mask) { o->me2 = 0.0; o->w = 0.0; return 0; }
    o->me2 = or_me2(proc, P, &o->p[0][0]);
    o->w = o->f1 * o->f2 * o->me2 / (2.0 * o->shat) * o->w_ps * o->jac_parton * o->jac_vegas * GEV2_TO_PB;
    return 0;
}

/* or_event for a list of events, in parallel over events (independent calls). */
int or_events(int proc, const or_params *P, const or_pdf *pdf, const double *grid, const uint64_t *events,
              int64_t n, uint32_t iteration, or_event_out *out, int n_threads)
{
    int rc = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : rc)
#endif
    for (int64_t i = 0; i < n; ++i) rc |= or_event(proc, P, pdf, grid, events[i], iteration, NULL, out + i);
    return rc;
}

/*
 * Observable histogram (the pipeline's histogram accumulation, Sec. 2.1; the
 * p_T distribution of Sec. 3, Fig. 2): the transverse momentum of the first
 * final-state particle, p_T = sqrt(px^2 + py^2), in nobs uniform bins on
 * [lo, hi) with an underflow bin 0 (also for a non-finite p_T) and an
 * overflow bin nobs + 1.
 */
int or_obs_bin(double px, double py, int nobs, double lo, double hi)
{
    double pt = sqrt(px * px + py * py);
    double inv_w = (double)nobs / (hi - lo);
    if (!(pt >= lo)) return 0;
    double t = (pt - lo) * inv_w;
    if (!(t < (double)nobs)) return nobs + 1;
    return 1 + (int)t;
}

/* one pass; with nobs > 0 also obs[(nobs + 2) * 2]: per bin sum w/N and sum (w/N)^2 */
static int pass_impl(int proc, const or_params *P, const or_pdf *pdf, const double *grid, int64_t n,
                     uint32_t iteration, const uint8_t *mask_in, uint8_t *mask_out,
                     double *sum_w, double *sum_w2, double *hist, int64_t *n_pass, int n_threads,
                     int nobs, double lo, double hi, double *obs)
{
    or_proc_info info;
    if (or_proc_info_get(proc, &info) || n <= 0) return 1;
    int D = info.dim, nb = P->n_bins;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    uint8_t *bins = (uint8_t *)malloc((size_t)n * (size_t)D);
    uint8_t *mk = (uint8_t *)malloc((size_t)n);
    int *ob = (int *)malloc(sizeof(int) * (size_t)n);
    if (!w || !bins || !mk || !ob) { free(w); free(bins); free(mk); free(ob); return 2; }
    /* one serial event first so that lazily built colour tables exist before the threads start */
    {
        or_event_out o;
        int mo = mask_in ? mask_in[0] : 0;
        or_event(proc, P, pdf, grid, 0, iteration, mask_in ? &mo : NULL, &o);
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < n; ++e) {
        or_event_out o;
        int mo = mask_in ? mask_in[e] : 0;
        or_event(proc, P, pdf, grid, (uint64_t)e, iteration, mask_in ? &mo : NULL, &o);
        w[e] = o.w;
        mk[e] = (uint8_t)o.mask;
        memcpy(bins + (size_t)e * D, o.bins, (size_t)D);
        ob[e] = nobs > 0 ? or_obs_bin(o.p[2][1], o.p[2][2], nobs, lo, hi) : 0;
    }
    double sw = 0.0, sw2 = 0.0;
    int64_t np = 0;
    if (hist) memset(hist, 0, sizeof(double) * (size_t)D * nb);
    if (nobs > 0) memset(obs, 0, sizeof(double) * 2 * (size_t)(nobs + 2));
    for (int64_t e = 0; e < n; ++e) {
        double we = w[e] / (double)n;
        double w2 = we * we;
        sw += we; sw2 += w2;
        np += mk[e];
        if (hist)
            for (int d = 0; d < D; ++d) hist[d * nb + bins[(size_t)e * D + d]] += w2;
        if (nobs > 0) { obs[2 * ob[e]] += we; obs[2 * ob[e] + 1] += w2; }
        if (mask_out) mask_out[e] = mk[e];
    }
    *sum_w = sw; *sum_w2 = sw2;
    if (n_pass) *n_pass = np;
    free(w); free(bins); free(mk); free(ob);
    return 0;
}

int or_pass(int proc, const or_params *P, const or_pdf *pdf, const double *grid, int64_t n,
            uint32_t iteration, const uint8_t *mask_in, uint8_t *mask_out,
            double *sum_w, double *sum_w2, double *hist, int64_t *n_pass, int n_threads)
{
    return pass_impl(proc, P, pdf, grid, n, iteration, mask_in, mask_out, sum_w, sum_w2, hist, n_pass,
                     n_threads, 0, 0.0, 1.0, NULL);
}

int or_pass_obs(int proc, const or_params *P, const or_pdf *pdf, const double *grid, int64_t n,
                uint32_t iteration, int nobs, double lo, double hi, double *sum_w, double *sum_w2,
                double *obs, int n_threads)
{
    if (nobs < 1 || !(hi > lo) || !obs) return 1;
    return pass_impl(proc, P, pdf, grid, n, iteration, NULL, NULL, sum_w, sum_w2, NULL, NULL, n_threads,
                     nobs, lo, hi, obs);
}

/*
 * VEGAS integration with the observable histogram.  Reading (the paper does
 * not say how iterations combine into a distribution): every iteration fills
 * per bin I_jk = sum w/N and its variance V_jk = (N sum (w/N)^2 - I_jk^2)/(N-1);
 * the bins combine with the integral's inverse-variance weights
 * l_k = (1/V_k) / sum_i (1/V_i): H_j = sum_k l_k I_jk, err_j^2 = sum_k l_k^2 V_jk,
 * so that sum_j H_j equals the combined cross section.
 */
int or_integrate_obs(int proc, const or_params *P, const or_pdf *pdf, int64_t n, int n_iter,
                     int nobs, double lo, double hi, double *obs_hist, double *obs_err, double *obs_iter,
                     or_result *res, int n_threads)
{
    or_proc_info info;
    if (or_proc_info_get(proc, &info) || n < 2 || n_iter < 1 || nobs < 1 || !(hi > lo)) return 1;
    int D = info.dim, nb = P->n_bins, n2 = nobs + 2;
    double *grid = (double *)malloc(sizeof(double) * (size_t)D * (nb + 1));
    double *hist = (double *)malloc(sizeof(double) * (size_t)D * nb);
    double *I = (double *)malloc(sizeof(double) * (size_t)n_iter);
    double *V = (double *)malloc(sizeof(double) * (size_t)n_iter);
    double *IJ = (double *)malloc(sizeof(double) * (size_t)n_iter * n2);
    double *VJ = (double *)malloc(sizeof(double) * (size_t)n_iter * n2);
    double *obs = (double *)malloc(sizeof(double) * 2 * (size_t)n2);
    or_vegas_init(grid, D, nb);
    int64_t np_tot = 0;
    for (int it = 0; it < n_iter; ++it) {
        double sw, sw2; int64_t np;
        int rc = pass_impl(proc, P, pdf, grid, n, (uint32_t)it, NULL, NULL, &sw, &sw2, hist, &np, n_threads,
                           nobs, lo, hi, obs);
        if (rc) { free(grid); free(hist); free(I); free(V); free(IJ); free(VJ); free(obs); return rc; }
        I[it] = sw;
        V[it] = ((double)n * sw2 - sw * sw) / (double)(n - 1);
        for (int j = 0; j < n2; ++j) {
            double a = obs[2 * j], b = obs[2 * j + 1];
            IJ[(size_t)it * n2 + j] = a;
            VJ[(size_t)it * n2 + j] = ((double)n * b - a * a) / (double)(n - 1);
            if (obs_iter) {
                obs_iter[((size_t)it * n2 + j) * 2] = a;
                obs_iter[((size_t)it * n2 + j) * 2 + 1] = VJ[(size_t)it * n2 + j];
            }
        }
        np_tot += np;
        if (it < n_iter - 1) or_vegas_refine(hist, grid, D, nb, P->alpha);
    }
    or_vegas_combine(n_iter, I, V, &res->sigma, &res->error, &res->chi2dof);
    res->n_pass = np_tot;
    double inv_sum = 0.0;
    for (int k = 0; k < n_iter; ++k) inv_sum += 1.0 / V[k];
    for (int j = 0; j < n2; ++j) {
        double h = 0.0, e2 = 0.0;
        for (int k = 0; k < n_iter; ++k) {
            double l = (1.0 / V[k]) / inv_sum;
            h += l * IJ[(size_t)k * n2 + j];
            e2 += l * l * VJ[(size_t)k * n2 + j];
        }
        obs_hist[j] = h;
        obs_err[j] = sqrt(e2 > 0.0 ? e2 : 0.0);
    }
    free(grid); free(hist); free(I); free(V); free(IJ); free(VJ); free(obs);
    return 0;
}

int or_integrate(int proc, const or_params *P, const or_pdf *pdf, int64_t n, int n_iter,
                 double *grid_io, double *per_iter, or_result *res, int n_threads)
{
    or_proc_info info;
    if (or_proc_info_get(proc, &info) || n < 2 || n_iter < 1) return 1;
    int D = info.dim, nb = P->n_bins;
    double *grid = (double *)malloc(sizeof(double) * (size_t)D * (nb + 1));
    double *hist = (double *)malloc(sizeof(double) * (size_t)D * nb);
    double *I = (double *)malloc(sizeof(double) * (size_t)n_iter);
    double *V = (double *)malloc(sizeof(double) * (size_t)n_iter);
    or_vegas_init(grid, D, nb);
    int64_t np_tot = 0;
    for (int it = 0; it < n_iter; ++it) {
        double sw, sw2; int64_t np;
        int rc = or_pass(proc, P, pdf, grid, n, (uint32_t)it, NULL, NULL, &sw, &sw2, hist, &np, n_threads);
        if (rc) { free(grid); free(hist); free(I); free(V); return rc; }
        I[it] = sw;
        V[it] = ((double)n * sw2 - sw * sw) / (double)(n - 1);
        np_tot += np;
        if (per_iter) { per_iter[2 * it] = I[it]; per_iter[2 * it + 1] = V[it]; }
        if (it < n_iter - 1) or_vegas_refine(hist, grid, D, nb, P->alpha);
    }
    or_vegas_combine(n_iter, I, V, &res->sigma, &res->error, &res->chi2dof);
    res->n_pass = np_tot;
    if (grid_io) memcpy(grid_io, grid, sizeof(double) * (size_t)D * (nb + 1));
    free(grid); free(hist); free(I); free(V);
    return 0;
}

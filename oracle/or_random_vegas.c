/*
 * Oracle: random numbers (Philox) and the VEGAS integrator (map, per-bin sums,
 * refinement and the combination of iterations).
 * TEST INFRASTRUCTURE ONLY (see mf_oracle.h).
 *
 * The paper's integrator (Sec. 1, the VegasFlow library; Sec. 2.1, where the
 * per-event pipeline starts from random numbers and ends in histogram
 * filling) is the classic adaptive VEGAS of Lepage (J. Comput. Phys. 27
 * (1978) 192).  Random numbers come from the
 * counter-based Philox4x32-10 generator of Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here from
 * its published definition.
 */
#include "mf_oracle.h"
#include <math.h>
#include <string.h>

/* Philox4x32-10: ten rounds of the Philox S-box on a 4-word counter, the key
 * bumped by the Weyl constants between rounds (Salmon et al. 2011, Sec. 3). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key increments */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two 32-bit words -> one double in the open interval (0,1): the top 26 bits
 * of each word form a 52-bit integer k and u = (k + 1/2) 2^-52, which is
 * exact in binary64, never 0 and never 1. */
double or_u01(uint32_t a, uint32_t b)
{
    uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return ((double)k + 0.5) * (1.0 / 4503599627370496.0);
}

/* Uniform stream of one event: Philox block b (counter = event low/high words,
 * iteration, channel<<8 | b; key = seed low/high words) gives dimensions 2b
 * and 2b+1 from output words (0,1) and (2,3). */
void or_uniforms(uint64_t seed, uint64_t event, uint32_t iteration, uint32_t channel,
                 int dim, double *u)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int b = 0; 2 * b < dim; ++b) {
        uint32_t ctr[4] = { (uint32_t)event, (uint32_t)(event >> 32), iteration,
                            (channel << 8) | (uint32_t)b };
        uint32_t o[4];
        or_philox4x32_10(ctr, key, o);
        u[2 * b] = or_u01(o[0], o[1]);
        if (2 * b + 1 < dim) u[2 * b + 1] = or_u01(o[2], o[3]);
    }
}

/* Uniform starting grid: nb equal bins per dimension on [0,1]. */
void or_vegas_init(double *grid, int dim, int nb)
{
    for (int d = 0; d < dim; ++d)
        for (int i = 0; i <= nb; ++i)
            grid[d * (nb + 1) + i] = (double)i / (double)nb;
}

/* VEGAS map (Lepage 1978, Sec. 2): u in (0,1) -> bin b = floor(nb u) and the
 * point x inside bin b at the same fractional position; the Jacobian is the
 * product over dimensions of nb times the bin width. */
double or_vegas_map(const double *grid, int dim, int nb, const double *u, double *x, uint8_t *bins)
{
    double jac = 1.0;
    for (int d = 0; d < dim; ++d) {
        const double *e = grid + d * (nb + 1);
        double y = u[d] * (double)nb;
        int b = (int)y;
        if (b > nb - 1) b = nb - 1;
        double frac = y - (double)b;
        double width = e[b + 1] - e[b];
        x[d] = fma(width, frac, e[b]);
        jac = jac * ((double)nb * width);
        if (bins) bins[d] = (uint8_t)b;
    }
    return jac;
}

/* Grid refinement (Lepage 1978, Sec. 3): smooth the per-bin sums of (f J)^2
 * with neighbours, normalise, damp with ((r-1)/ln r)^alpha, then move the
 * edges so that every new bin holds the same share of the damped weights.
 * A dimension whose histogram is all zero keeps its grid. */
void or_vegas_refine(const double *hist, double *grid, int dim, int nb, double alpha)
{
    double s[256], w[256], newe[257];
    for (int d = 0; d < dim; ++d) {
        const double *h = hist + d * nb;
        double *e = grid + d * (nb + 1);
        double tot_h = 0.0;
        for (int i = 0; i < nb; ++i) tot_h += h[i];
        if (!(tot_h > 0.0)) continue;
        s[0] = (7.0 * h[0] + h[1]) / 8.0;
        for (int i = 1; i < nb - 1; ++i) s[i] = (h[i - 1] + 6.0 * h[i] + h[i + 1]) / 8.0;
        s[nb - 1] = (h[nb - 2] + 7.0 * h[nb - 1]) / 8.0;
        double sum = 0.0;
        for (int i = 0; i < nb; ++i) sum += s[i];
        double wsum = 0.0;
        for (int i = 0; i < nb; ++i) {
            double r = s[i] / sum;
            if (r > 0.0 && r < 1.0) w[i] = pow((r - 1.0) / log(r), alpha);
            else if (r >= 1.0) w[i] = 1.0;
            else w[i] = 0.0;
            wsum += w[i];
        }
        double delta = wsum / (double)nb;
        newe[0] = 0.0; newe[nb] = 1.0;
        double acc = 0.0;
        int j = 0;
        for (int k = 1; k < nb; ++k) {
            double target = (double)k * delta;
            while (j < nb - 1 && acc + w[j] < target) { acc += w[j]; ++j; }
            double frac = (w[j] > 0.0) ? (target - acc) / w[j] : 0.0;
            if (frac > 1.0) frac = 1.0;
            newe[k] = e[j] + frac * (e[j + 1] - e[j]);
        }
        memcpy(e, newe, sizeof(double) * (size_t)(nb + 1));
    }
}

/* Inverse-variance weighted mean of the iteration estimates, its error and
 * chi^2 per degree of freedom (Lepage 1978). */
void or_vegas_combine(int n_iter, const double *I, const double *var,
                      double *mean, double *err, double *chi2dof)
{
    double sw = 0.0, swi = 0.0;
    for (int k = 0; k < n_iter; ++k) {
        double wk = 1.0 / var[k];
        sw += wk; swi += wk * I[k];
    }
    double m = swi / sw;
    double chi2 = 0.0;
    for (int k = 0; k < n_iter; ++k) chi2 += (I[k] - m) * (I[k] - m) / var[k];
    *mean = m;
    *err = sqrt(1.0 / sw);
    *chi2dof = n_iter > 1 ? chi2 / (double)(n_iter - 1) : 0.0;
}

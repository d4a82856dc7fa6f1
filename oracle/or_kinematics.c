/*
 * Oracle: parton-luminosity map (a3), RAMBO phase space (a4), fiducial cuts
 * (a5), factorisation scale (a6) and log-bicubic PDF interpolation (a7).
 * TEST INFRASTRUCTURE ONLY (see mf_oracle.h).
 *
 * Sec. 1 of the paper lists the ingredients: a phase-space generator that also
 * applies fiducial cuts, and GPU PDF interpolation (PDFFlow).  The generator
 * here is RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359)
 * with its massive extension; the interpolation is the log-bicubic scheme of
 * LHAPDF6 (Buckley et al., Eur. Phys. J. C 75 (2015) 132), separable cubic
 * Hermite in ln x then ln Q^2 with finite-difference node derivatives.
 */
#include "mf_oracle.h"
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Parton-luminosity map: tau = tau0^x0, x1 = tau^v, x2 = tau^(1-v); dx1 dx2 = tau |ln tau| |ln tau0| dx0 dv. */
void or_parton_map(double x0, double v, double tau0, double *x1, double *x2, double *jac)
{
    double lt0 = log(tau0);
    double lt = x0 * lt0;
    double tau = exp(lt);
    *x1 = exp(v * lt);
    *x2 = exp((1.0 - v) * lt);
    *jac = tau * (-lt) * (-lt0);
}

static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* Volume of massless n-body phase space (KSE 1986):
 * (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!). */
double or_rambo_massless_volume(int n, double shat)
{
    return pow(2.0 * M_PI, 4.0 - 3.0 * n) * pow(M_PI / 2.0, n - 1) * pow(shat, n - 2)
           / (factorial(n - 1) * factorial(n - 2));
}

/* RAMBO (Kleiss, Stirling, Ellis 1986).  Four uniforms per particle give an isotropic massless momentum
 * with energy -ln(u3 u4); a conformal transformation (boost + scale) brings
 * the sum to (sqrt(shat), 0); masses are then restored by a common rescaling
 * xi of the three-momenta found by Newton's method, with the massive weight
 * factor of KSE 1986. */
int or_rambo(int n, double sqrt_shat, const double *masses, const double *u, double *p, double *weight)
{
    double q[8][4];
    double Q[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        double c = 2.0 * u[4 * i] - 1.0;
        double s = sqrt(1.0 - c * c);
        double f = 2.0 * M_PI * u[4 * i + 1];
        double e = -log(u[4 * i + 2] * u[4 * i + 3]);
        q[i][0] = e;
        q[i][1] = e * s * cos(f);
        q[i][2] = e * s * sin(f);
        q[i][3] = e * c;
        for (int m = 0; m < 4; ++m) Q[m] += q[i][m];
    }
    double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
    double b[3] = { -Q[1] / M, -Q[2] / M, -Q[3] / M };
    double x = sqrt_shat / M;
    double gam = Q[0] / M;
    double a = 1.0 / (1.0 + gam);
    for (int i = 0; i < n; ++i) {
        double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
        p[4 * i + 0] = x * (gam * q[i][0] + bq);
        for (int m = 1; m < 4; ++m)
            p[4 * i + m] = x * (q[i][m] + b[m - 1] * q[i][0] + a * bq * b[m - 1]);
    }
    double w = or_rambo_massless_volume(n, sqrt_shat * sqrt_shat);

    double msum = 0.0; int massive = 0;
    for (int i = 0; i < n; ++i) { msum += masses[i]; if (masses[i] != 0.0) massive = 1; }
    if (!massive) { *weight = w; return 0; }
    if (msum >= sqrt_shat) { *weight = 0.0; return 1; }

    double xi = sqrt(1.0 - (msum / sqrt_shat) * (msum / sqrt_shat));
    double p2[8];
    for (int i = 0; i < n; ++i) p2[i] = p[4 * i + 0] * p[4 * i + 0];
    for (int it = 0; it < 100; ++it) {
        double f = -sqrt_shat, fp = 0.0;
        for (int i = 0; i < n; ++i) {
            double ei = sqrt(masses[i] * masses[i] + xi * xi * p2[i]);
            f += ei;
            fp += xi * p2[i] / ei;
        }
        double step = f / fp;
        xi -= step;
        if (fabs(f) < 1e-15 * sqrt_shat) break;
    }
    double sk = 0.0, sk2e = 0.0, prod = 1.0;
    for (int i = 0; i < n; ++i) {
        double kabs = xi * p[4 * i + 0];                /* |k_i| = xi |p_i| = xi E_i (massless) */
        double e = sqrt(masses[i] * masses[i] + kabs * kabs);
        for (int m = 1; m < 4; ++m) p[4 * i + m] *= xi;
        p[4 * i + 0] = e;
        sk += kabs;
        sk2e += kabs * kabs / e;
        prod *= kabs / e;
    }
    w *= pow(sk / sqrt_shat, 2 * n - 3) * prod * sqrt_shat / sk2e;
    *weight = w;
    return 0;
}

static double pt2_of(const double *p) { return p[1] * p[1] + p[2] * p[2]; }

/* Fiducial cuts on the final light partons in the lab frame:
 * pT > pt_min, |eta| < eta_max (tested as |pz| < pT sinh(eta_max)), and
 * Delta R > dr_min between every pair of final gluons.  Returns 1 when the
 * event passes. */
int or_cuts(int proc, const or_params *P, const double *plab)
{
    int light[3], nl = 0;
    if (proc == OR_GG_TTG || proc == OR_UG_TTU) { light[0] = 4; nl = 1; }
    else if (proc == OR_GG_TTGG) { light[0] = 4; light[1] = 5; nl = 2; }
    else if (proc == OR_GG_TTGGG) { light[0] = 4; light[1] = 5; light[2] = 6; nl = 3; }
    else return 1;
    double sh = P->eta_max > 0.0 ? sinh(P->eta_max) : 0.0;
    for (int j = 0; j < nl; ++j) {
        const double *p = plab + 4 * light[j];
        double pt2 = pt2_of(p);
        if (P->pt_min > 0.0 && !(pt2 > P->pt_min * P->pt_min)) return 0;
        if (P->eta_max > 0.0 && !(fabs(p[3]) < sqrt(pt2) * sh)) return 0;
    }
    if ((proc == OR_GG_TTGG || proc == OR_GG_TTGGG) && P->dr_min > 0.0) {
        for (int i = 0; i < nl; ++i)
            for (int j = i + 1; j < nl; ++j) {
                const double *a = plab + 4 * light[i], *b = plab + 4 * light[j];
                double pta = sqrt(pt2_of(a)), ptb = sqrt(pt2_of(b));
                double ea = asinh(a[3] / pta), eb = asinh(b[3] / ptb);
                double dphi = atan2(a[2], a[1]) - atan2(b[2], b[1]);
                if (dphi > M_PI) dphi -= 2.0 * M_PI;
                if (dphi < -M_PI) dphi += 2.0 * M_PI;
                double dr2 = (ea - eb) * (ea - eb) + dphi * dphi;
                if (!(dr2 > P->dr_min * P->dr_min)) return 0;
            }
    }
    return 1;
}

/* Factorisation scale: mu_F = m_t for the 2 -> 2 top channels, H_T/2 with H_T the sum of the
 * final-state transverse masses otherwise; returns mu_F^2. */
double or_muf2(int proc, const or_params *P, const double *p)
{
    if (proc == OR_GG_TT || proc == OR_UU_TT) return P->mt * P->mt;
    if (proc == OR_EE_MUMU) return 0.0;
    int n_ext = proc == OR_GG_TTGGG ? 7 : (proc == OR_GG_TTGG ? 6 : 5);
    double ht = 0.0;
    for (int i = 2; i < n_ext; ++i) {
        double m = (i == 2 || i == 3) ? P->mt : 0.0;
        ht += sqrt(m * m + pt2_of(p + 4 * i));
    }
    return 0.25 * ht * ht;
}

/* One-dimensional cubic Hermite on a uniform grid: values v[0..n-1], spacing h,
 * interval i, local coordinate t in [0,1]; node derivatives are central
 * differences inside and one-sided differences at the two ends. */
static double node_deriv(const double *v, int n, int i, double h)
{
    if (i == 0) return (v[1] - v[0]) / h;
    if (i == n - 1) return (v[n - 1] - v[n - 2]) / h;
    return (v[i + 1] - v[i - 1]) / (2.0 * h);
}

static double hermite(double f0, double f1, double d0, double d1, double h, double t)
{
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    return h00 * f0 + h10 * h * d0 + h01 * f1 + h11 * h * d1;
}

/* PDF: x f(x, Q^2) by cubic Hermite in ln x along every Q^2 row that the
 * Q^2 step needs, then cubic Hermite in ln Q^2 over those row values.
 * ln Q^2 outside the grid is clamped to its edge. */
double or_pdf_xf(const or_pdf *pdf, int flav, double x, double q2)
{
    int nx = pdf->nx, nq = pdf->nq;
    double lx0 = log(pdf->x_min), lx1 = 0.0;
    double lq0 = log(pdf->q2_min), lq1 = log(pdf->q2_max);
    double hx = (lx1 - lx0) / (double)(nx - 1);
    double hq = (lq1 - lq0) / (double)(nq - 1);
    double lx = log(x), lq = log(q2);
    if (lq < lq0) lq = lq0;
    if (lq > lq1) lq = lq1;
    int i = (int)floor((lx - lx0) / hx);
    if (i < 0) i = 0;
    if (i > nx - 2) i = nx - 2;
    int j = (int)floor((lq - lq0) / hq);
    if (j < 0) j = 0;
    if (j > nq - 2) j = nq - 2;
    double t = (lx - (lx0 + i * hx)) / hx;
    double s = (lq - (lq0 + j * hq)) / hq;
    const double *g = pdf->xf + (size_t)flav * nx * nq;

    /* rows j-1 .. j+2 (those that exist), each interpolated in ln x */
    double row[4]; int r0 = j - 1;
    double col[256];
    for (int r = 0; r < 4; ++r) {
        int jr = r0 + r;
        if (jr < 0 || jr >= nq) { row[r] = 0.0; continue; }
        for (int ii = 0; ii < nx; ++ii) col[ii] = g[(size_t)ii * nq + jr];
        row[r] = hermite(col[i], col[i + 1], node_deriv(col, nx, i, hx), node_deriv(col, nx, i + 1, hx), hx, t);
    }
    /* derivatives in ln Q^2 at rows j and j+1 from the interpolated row values */
    double dj, dj1;
    if (j == 0) dj = (row[2] - row[1]) / hq; else dj = (row[2] - row[0]) / (2.0 * hq);
    if (j + 1 == nq - 1) dj1 = (row[2] - row[1]) / hq; else dj1 = (row[3] - row[1]) / (2.0 * hq);
    return hermite(row[1], row[2], dj, dj1, hq, s);
}

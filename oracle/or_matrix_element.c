/*
 * Oracle: squared matrix elements (Sec. 2.2: wavefunctions, amplitudes, colour sum).
 * TEST INFRASTRUCTURE ONLY (see mf_oracle.h).
 *
 * Sec. 2.2 of the paper: the squared amplitude is the sum over external
 * helicities and colours of the Feynman-rule amplitude.  The oracle reaches it
 * by routes that differ on purpose from the CUDA path (which sums Feynman
 * diagrams built from helicity wavefunctions and a colour-flow matrix):
 *
 *  - e+e- -> mu+mu- (photon + Z) and q qbar -> t tbar: closed forms.
 *  - g g -> t tbar + (k-2) gluons: Berends-Giele colour-ordered recursion
 *    (Berends & Giele, Nucl. Phys. B306 (1988) 759) for the partial
 *    amplitudes, with the colour matrix summed by brute force over explicit
 *    Gell-Mann matrices; Dirac-representation spinors in the spin-z basis and
 *    linear gluon polarisations.
 *  - u g -> t tbar u: the five Feynman diagrams written out with explicit
 *    Dirac matrices, summed over every explicit colour index.
 *  - g g -> t tbar: also the closed form of Combridge (Nucl. Phys. B151
 *    (1979) 429), used as a pin of the recursion.
 *
 * Feynman rules (metric +,-,-,-; D = d - i g A^a T^a; Feynman gauge):
 *   quark-gluon vertex  i g gamma^mu T^a
 *   quark propagator    i (pslash + m) / (p^2 - m^2)
 *   gluon propagator    -i g_{mu nu} delta^{ab} / k^2
 *   three-gluon vertex  g f^{abc} [g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu
 *                                  + g^{rho mu}(k3-k1)^nu], momenta incoming
 *   four-gluon vertex   -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sigma}-g^{mu sigma}g^{nu rho})
 *                               + f^{ace}f^{bde}(g^{mu nu}g^{rho sigma}-g^{mu sigma}g^{nu rho})
 *                               + f^{ade}f^{bce}(g^{mu nu}g^{rho sigma}-g^{mu rho}g^{nu sigma})]
 * Colour-ordered rules follow from f^{abc} T^c = -i [T^a, T^b].
 */
#include "mf_oracle.h"
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- Dirac algebra */

static cplx GAM[4][4][4];   /* GAM[mu][row][col], Dirac representation */
static int gam_ready = 0;

static void gamma_init(void)
{
    if (gam_ready) return;
    memset(GAM, 0, sizeof(GAM));
    /* gamma^0 = diag(1,1,-1,-1) */
    GAM[0][0][0] = 1; GAM[0][1][1] = 1; GAM[0][2][2] = -1; GAM[0][3][3] = -1;
    /* gamma^k = [[0, sigma_k], [-sigma_k, 0]] */
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                GAM[k + 1][r][c + 2] = sig[k][r][c];
                GAM[k + 1][r + 2][c] = -sig[k][r][c];
            }
    gam_ready = 1;
}

static cplx mdot(const cplx *a, const cplx *b)
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* a-slash = gamma^mu a_mu = gamma^0 a^0 - gamma^k a^k */
static void slash(const cplx *a, cplx S[4][4])
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            S[r][c] = GAM[0][r][c] * a[0] - GAM[1][r][c] * a[1] - GAM[2][r][c] * a[2] - GAM[3][r][c] * a[3];
}

static void row_times(const cplx *row, cplx M[4][4], cplx *out)
{
    cplx t[4];
    for (int c = 0; c < 4; ++c) {
        t[c] = 0;
        for (int r = 0; r < 4; ++r) t[c] += row[r] * M[r][c];
    }
    memcpy(out, t, sizeof(t));
}

static cplx row_col(const cplx *row, const cplx *col)
{
    cplx s = 0;
    for (int i = 0; i < 4; ++i) s += row[i] * col[i];
    return s;
}

/* propagator numerator and denominator folded: i (qslash + m) / (q^2 - m^2) */
static void quark_prop(const double *q, double m, cplx P[4][4])
{
    cplx qc[4] = { q[0], q[1], q[2], q[3] };
    slash(qc, P);
    double den = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3] - m * m;
    for (int r = 0; r < 4; ++r) {
        P[r][r] += m;
        for (int c = 0; c < 4; ++c) P[r][c] *= I / den;
    }
}

/* Dirac spinors in the spin-z basis xi_0 = (1,0), xi_1 = (0,1):
 * u = (sqrt(E+m) xi ; (sigma.p) xi / sqrt(E+m)),
 * v = ((sigma.p) eta / sqrt(E+m) ; sqrt(E+m) eta). */
static void sigma_dot_p(const double *p, int s, cplx out[2])
{
    /* (sigma.p) acting on basis vector s */
    cplx px = p[1], py = p[2], pz = p[3];
    if (s == 0) { out[0] = pz; out[1] = px + I * py; }
    else        { out[0] = px - I * py; out[1] = -pz; }
}

static void spinor_u(const double *p, double m, int s, cplx u[4])
{
    double n = sqrt(p[0] + m);
    cplx sp[2]; sigma_dot_p(p, s, sp);
    u[0] = s == 0 ? n : 0; u[1] = s == 1 ? n : 0;
    u[2] = sp[0] / n; u[3] = sp[1] / n;
}

static void spinor_v(const double *p, double m, int s, cplx v[4])
{
    double n = sqrt(p[0] + m);
    cplx sp[2]; sigma_dot_p(p, s, sp);
    v[0] = sp[0] / n; v[1] = sp[1] / n;
    v[2] = s == 0 ? n : 0; v[3] = s == 1 ? n : 0;
}

/* psi-bar = psi^dagger gamma^0 */
static void bar(const cplx psi[4], cplx out[4])
{
    out[0] = conj(psi[0]); out[1] = conj(psi[1]);
    out[2] = -conj(psi[2]); out[3] = -conj(psi[3]);
}

/* linear polarisations of a massless vector with three-momentum along p */
static void lin_pol(const double *p, int l, cplx eps[4])
{
    double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double n[3] = { p[1] / pa, p[2] / pa, p[3] / pa };
    double a[3] = { 0, 0, 1 };
    if (fabs(n[2]) > 0.9) { a[0] = 1; a[2] = 0; }
    double e1[3] = { a[1] * n[2] - a[2] * n[1], a[2] * n[0] - a[0] * n[2], a[0] * n[1] - a[1] * n[0] };
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] /= l1;
    double e2[3] = { n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0] };
    const double *e = l == 0 ? e1 : e2;
    eps[0] = 0; eps[1] = e[0]; eps[2] = e[1]; eps[3] = e[2];
}

/* ---------------------------------------------------------------- closed forms */

/* e+ e- -> mu+ mu- through photon and Z (massless fermions), spin averaged:
 * |M|^2 = (e^4/4) [ (|A_LL|^2+|A_RR|^2)(1+c)^2 + (|A_LR|^2+|A_RL|^2)(1-c)^2 ],
 * A_ij = Q_e Q_mu + g_i g_j s / ((s - MZ^2 + i MZ GZ) sW^2 cW^2),
 * g_L = T3 - Q sW^2, g_R = -Q sW^2, c = cos(angle e- , mu-);  MW from the
 * G_F scheme.  Momenta: e-, e+, mu-, mu+. */
double or_me2_ee_mumu_closed(const or_params *P, const double *p)
{
    double alpha = 1.0 / P->alpha_em_inv;
    double mz2 = P->mz * P->mz;
    double mw2 = 0.5 * mz2 + sqrt(0.25 * mz2 * mz2 - M_PI * alpha * mz2 / (sqrt(2.0) * P->gf));
    double sw2 = 1.0 - mw2 / mz2, cw2 = 1.0 - sw2;
    double e4 = (4.0 * M_PI * alpha) * (4.0 * M_PI * alpha);
    const double *p1 = p, *p2 = p + 4, *p3 = p + 8;
    double s = (p1[0] + p2[0]) * (p1[0] + p2[0]) - (p1[1] + p2[1]) * (p1[1] + p2[1])
             - (p1[2] + p2[2]) * (p1[2] + p2[2]) - (p1[3] + p2[3]) * (p1[3] + p2[3]);
    double a1 = sqrt(p1[1] * p1[1] + p1[2] * p1[2] + p1[3] * p1[3]);
    double a3 = sqrt(p3[1] * p3[1] + p3[2] * p3[2] + p3[3] * p3[3]);
    double c = (p1[1] * p3[1] + p1[2] * p3[2] + p1[3] * p3[3]) / (a1 * a3);
    double Q = -1.0, T3 = -0.5;
    double gL = T3 - Q * sw2, gR = -Q * sw2;
    cplx chi = s / ((s - mz2 + I * P->mz * P->wz) * sw2 * cw2);
    cplx ALL = Q * Q + gL * gL * chi, ARR = Q * Q + gR * gR * chi;
    cplx ALR = Q * Q + gL * gR * chi, ARL = Q * Q + gR * gL * chi;
    double same = creal(ALL * conj(ALL)) + creal(ARR * conj(ARR));
    double oppo = creal(ALR * conj(ALR)) + creal(ARL * conj(ARL));
    return 0.25 * e4 * (same * (1 + c) * (1 + c) + oppo * (1 - c) * (1 - c));
}

static double mdot_r(const double *a, const double *b)
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* g g -> Q Qbar, averaged (Combridge 1979):
 * g^4 (1/(6 t1 t2) - 3/8) (t1^2 + t2^2 + rho - rho^2/(4 t1 t2)),
 * t1 = 2 p1.p3 / s, t2 = 2 p2.p3 / s, rho = 4 m^2 / s. */
double or_me2_gg_tt_closed(double mt, double gs, const double *p)
{
    const double *p1 = p, *p2 = p + 4, *p3 = p + 8;
    double s = 2.0 * mdot_r(p1, p2);
    double t1 = 2.0 * mdot_r(p1, p3) / s, t2 = 2.0 * mdot_r(p2, p3) / s;
    double rho = 4.0 * mt * mt / s;
    double g4 = gs * gs * gs * gs;
    return g4 * (1.0 / (6.0 * t1 * t2) - 3.0 / 8.0) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4.0 * t1 * t2));
}

/* q qbar -> Q Qbar, averaged: g^4 (4/9) (t1^2 + t2^2 + rho/2). */
double or_me2_uu_tt_closed(double mt, double gs, const double *p)
{
    const double *p1 = p, *p2 = p + 4, *p3 = p + 8;
    double s = 2.0 * mdot_r(p1, p2);
    double t1 = 2.0 * mdot_r(p1, p3) / s, t2 = 2.0 * mdot_r(p2, p3) / s;
    double rho = 4.0 * mt * mt / s;
    double g4 = gs * gs * gs * gs;
    return g4 * (4.0 / 9.0) * (t1 * t1 + t2 * t2 + 0.5 * rho);
}

/* ---------------------------------------------------------------- colour */

/* T^a = lambda^a / 2 with the Gell-Mann matrices lambda^1..lambda^8 */
static void gellmann(int a, cplx T[3][3])
{
    memset(T, 0, sizeof(cplx) * 9);
    switch (a) {
    case 0: T[0][1] = 1; T[1][0] = 1; break;
    case 1: T[0][1] = -I; T[1][0] = I; break;
    case 2: T[0][0] = 1; T[1][1] = -1; break;
    case 3: T[0][2] = 1; T[2][0] = 1; break;
    case 4: T[0][2] = -I; T[2][0] = I; break;
    case 5: T[1][2] = 1; T[2][1] = 1; break;
    case 6: T[1][2] = -I; T[2][1] = I; break;
    case 7: T[0][0] = 1.0 / sqrt(3.0); T[1][1] = 1.0 / sqrt(3.0); T[2][2] = -2.0 / sqrt(3.0); break;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] *= 0.5;
}

void or_gellmann_T(int a, double *out)
{
    cplx T[3][3];
    gellmann(a, T);
    for (int i = 0; i < 9; ++i) { out[2 * i] = creal(T[i / 3][i % 3]); out[2 * i + 1] = cimag(T[i / 3][i % 3]); }
}

static void mat3_mul(cplx A[3][3], cplx B[3][3], cplx C[3][3])
{
    cplx t[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            t[i][j] = 0;
            for (int l = 0; l < 3; ++l) t[i][j] += A[i][l] * B[l][j];
        }
    memcpy(C, t, sizeof(t));
}

/* lexicographic permutations of 0..k-1 */
static int perms(int k, int out[][8])
{
    int a[8], n = 0;
    for (int i = 0; i < k; ++i) a[i] = i;
    for (;;) {
        memcpy(out[n++], a, sizeof(int) * 8);
        int i = k - 2;
        while (i >= 0 && a[i] > a[i + 1]) --i;
        if (i < 0) break;
        int j = k - 1;
        while (a[j] < a[i]) --j;
        int t = a[i]; a[i] = a[j]; a[j] = t;
        for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    }
    return n;
}

/* C[s][t] = sum over gluon colours a_1..a_k and quark indices i,j of
 * conj((T^{a_s1} ... T^{a_sk})_ij) (T^{a_t1} ... T^{a_tk})_ij, by brute force.
 * Up to four gluons the 8^k colour assignments are summed one after the other;
 * for five (32768 assignments, 120 x 120 entries) they are split into 64 fixed
 * consecutive chunks, each summed in order (the chunks over threads), and the
 * chunk sums added in chunk order: the result does not depend on the number of
 * threads. */
#define MAXPERM 120
static void colour_chunk(int k, int np, int (*P)[8], cplx T[8][3][3], int a0, int a1, double *Cp)
{
    cplx (*S)[3][3] = malloc(sizeof(cplx[3][3]) * MAXPERM);
    for (int as = a0; as < a1; ++as) {
        int col[8], r = as;
        for (int i = 0; i < k; ++i) { col[i] = r % 8; r /= 8; }
        for (int s = 0; s < np; ++s) {
            cplx M[3][3];
            memcpy(M, T[col[P[s][0]]], sizeof(M));
            for (int i = 1; i < k; ++i) mat3_mul(M, T[col[P[s][i]]], M);
            memcpy(S[s], M, sizeof(M));
        }
        for (int s = 0; s < np; ++s)
            for (int t = 0; t < np; ++t) {
                cplx acc = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) acc += conj(S[s][i][j]) * S[t][i][j];
                Cp[s * np + t] += creal(acc);
            }
    }
    free(S);
}

void or_colour_matrix(int k, double *C)
{
    static int P[40320][8];
    int np = perms(k, P);
    cplx T[8][3][3];
    for (int a = 0; a < 8; ++a) gellmann(a, T[a]);
    for (int i = 0; i < np * np; ++i) C[i] = 0.0;
    int n_assign = 1;
    for (int i = 0; i < k; ++i) n_assign *= 8;
    if (k <= 4) {
        colour_chunk(k, np, P, T, 0, n_assign, C);
        return;
    }
    enum { NCHUNK = 64 };
    double *part = calloc((size_t)NCHUNK * np * np, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < NCHUNK; ++c)
        colour_chunk(k, np, P, T, (int)((long)n_assign * c / NCHUNK), (int)((long)n_assign * (c + 1) / NCHUNK),
                     part + (size_t)c * np * np);
    for (int c = 0; c < NCHUNK; ++c)
        for (int i = 0; i < np * np; ++i) C[i] += part[(size_t)c * np * np + i];
    free(part);
}

/* ---------------------------------------------------------------- Berends-Giele */

#define MAXG 6

/* colour-ordered three-gluon contraction V^rho(k1,k2,k3=-(k1+k2); J1, J2) */
static void v3(const double *k1, const double *k2, const cplx *J1, const cplx *J2, cplx *out)
{
    double k3[4], a[4], b[4], c[4];
    for (int m = 0; m < 4; ++m) {
        k3[m] = -(k1[m] + k2[m]);
        a[m] = k1[m] - k2[m];
        b[m] = k2[m] - k3[m];
        c[m] = k3[m] - k1[m];
    }
    cplx bc[4] = { b[0], b[1], b[2], b[3] }, cc[4] = { c[0], c[1], c[2], c[3] };
    cplx j12 = mdot(J1, J2), bj1 = mdot(bc, J1), cj2 = mdot(cc, J2);
    for (int m = 0; m < 4; ++m) out[m] = j12 * a[m] + J2[m] * bj1 + J1[m] * cj2;
}

/* Partial amplitude A(t, g_perm[0] .. g_perm[k-1], tbar).  Currents of
 * consecutive gluons obey
 *   J(i..j) = (1/P^2) [ -g sum_m V3(J(i..m), J(m+1..j))
 *                       + g^2 sum_{m<n} (2 (J1.J3) J2 - (J1.J2) J3 - (J2.J3) J1) ],
 * and the quark line is closed by summing over how the ordered gluons split
 * into consecutive blocks, each block attached by i g J-slash, with quark
 * propagators between the blocks (momentum p3 minus the gluon momenta
 * absorbed so far). */
void or_bg_partial(int k, const double *kg, const double *eps, const double *p3, const double *p4,
                   double m, double gs, int s3, int s4, const int *perm, double *amp_re_im)
{
    gamma_init();
    cplx J[MAXG][MAXG][4];
    double P[MAXG][MAXG][4];
    for (int i = 0; i < k; ++i) {
        for (int mu = 0; mu < 4; ++mu) {
            J[i][i][mu] = eps[8 * perm[i] + 2 * mu] + I * eps[8 * perm[i] + 2 * mu + 1];
            P[i][i][mu] = kg[4 * perm[i] + mu];
        }
    }
    for (int len = 2; len <= k; ++len)
        for (int i = 0; i + len - 1 < k; ++i) {
            int j = i + len - 1;
            for (int mu = 0; mu < 4; ++mu) P[i][j][mu] = P[i][i][mu] + P[i + 1][j][mu];
            double p2 = mdot_r(P[i][j], P[i][j]);
            cplx acc[4] = { 0, 0, 0, 0 }, t[4];
            for (int mm = i; mm < j; ++mm) {
                v3(P[i][mm], P[mm + 1][j], J[i][mm], J[mm + 1][j], t);
                for (int mu = 0; mu < 4; ++mu) acc[mu] += -gs * t[mu];
            }
            for (int mm = i; mm < j; ++mm)
                for (int nn = mm + 1; nn < j; ++nn) {
                    const cplx *J1 = J[i][mm], *J2 = J[mm + 1][nn], *J3 = J[nn + 1][j];
                    cplx d13 = mdot(J1, J3), d12 = mdot(J1, J2), d23 = mdot(J2, J3);
                    for (int mu = 0; mu < 4; ++mu)
                        acc[mu] += gs * gs * (2.0 * d13 * J2[mu] - d12 * J3[mu] - d23 * J1[mu]);
                }
            for (int mu = 0; mu < 4; ++mu) J[i][j][mu] = acc[mu] / p2;
        }

    cplx u3[4], ub3[4], v4[4];
    spinor_u(p3, m, s3, u3);
    bar(u3, ub3);
    spinor_v(p4, m, s4, v4);

    cplx U[MAXG][4];          /* U[j]: row spinor after the first j ordered gluons (with propagator) */
    memcpy(U[0], ub3, sizeof(ub3));
    double q[4] = { p3[0], p3[1], p3[2], p3[3] };
    for (int j = 1; j < k; ++j) {
        for (int mu = 0; mu < 4; ++mu) q[mu] -= P[j - 1][j - 1][mu];
        cplx acc[4] = { 0, 0, 0, 0 };
        for (int l = 0; l < j; ++l) {
            cplx S[4][4], r[4];
            slash(J[l][j - 1], S);
            row_times(U[l], S, r);
            for (int c = 0; c < 4; ++c) acc[c] += I * gs * r[c];
        }
        cplx Pr[4][4];
        quark_prop(q, m, Pr);
        row_times(acc, Pr, U[j]);
    }
    cplx amp = 0;
    for (int l = 0; l < k; ++l) {
        cplx S[4][4], r[4];
        slash(J[l][k - 1], S);
        row_times(U[l], S, r);
        amp += I * gs * row_col(r, v4);
    }
    amp_re_im[0] = creal(amp);
    amp_re_im[1] = cimag(amp);
}

/* Sum over spins, linear polarisations and colours of |M|^2 for
 * g..g -> t tbar g..g.  p_all: n_in_gluons incoming gluons, then t, tbar,
 * then the outgoing gluons; gluon momenta enter the recursion as incoming
 * (outgoing ones with a minus sign). */
double or_me2_bg(int k, const double *p_all, int n_in_gluons, double m, double gs)
{
    static double *Cm[7];
    static volatile int c_ready[7] = {0};
    if (k < 1 || k > 5) return 0.0;
    if (!c_ready[k]) {
#pragma omp critical(or_colour_init)
        {
            if (!c_ready[k]) {
                int n = 1;
                for (int i = 2; i <= k; ++i) n *= i;
                double *c = malloc(sizeof(double) * n * n);
                or_colour_matrix(k, c);
                Cm[k] = c;
                __sync_synchronize();
                c_ready[k] = 1;
            }
        }
    }
    int P[MAXPERM][8];
    int np = perms(k, P);
    double kg[MAXG * 4];
    const double *p3 = p_all + 4 * n_in_gluons, *p4 = p_all + 4 * (n_in_gluons + 1);
    const double *gp[MAXG];
    for (int i = 0; i < n_in_gluons; ++i) gp[i] = p_all + 4 * i;
    for (int i = n_in_gluons; i < k; ++i) gp[i] = p_all + 4 * (i + 2);
    for (int i = 0; i < k; ++i)
        for (int mu = 0; mu < 4; ++mu) kg[4 * i + mu] = (i < n_in_gluons ? 1.0 : -1.0) * gp[i][mu];

    double total = 0.0;
    int n_pol = 1 << k;
    for (int pol = 0; pol < n_pol; ++pol) {
        double eps[MAXG * 8];
        for (int i = 0; i < k; ++i) {
            cplx e[4];
            lin_pol(gp[i], (pol >> i) & 1, e);
            for (int mu = 0; mu < 4; ++mu) { eps[8 * i + 2 * mu] = creal(e[mu]); eps[8 * i + 2 * mu + 1] = cimag(e[mu]); }
        }
        for (int s3 = 0; s3 < 2; ++s3)
            for (int s4 = 0; s4 < 2; ++s4) {
                cplx A[MAXPERM];
                for (int s = 0; s < np; ++s) {
                    double a[2];
                    or_bg_partial(k, kg, eps, p3, p4, m, gs, s3, s4, P[s], a);
                    A[s] = a[0] + I * a[1];
                }
                double sum = 0.0;
                for (int s = 0; s < np; ++s)
                    for (int t = 0; t < np; ++t)
                        sum += creal(conj(A[s]) * Cm[k][s * np + t] * A[t]);
                total += sum;
            }
    }
    return total;
}

/* ---------------------------------------------------------------- two quark lines */

/* f^{abc} = -2 i Tr([T^a, T^b] T^c) */
static double fabc(cplx T[8][3][3], int a, int b, int c)
{
    cplx ab[3][3], ba[3][3], m[3][3];
    mat3_mul(T[a], T[b], ab);
    mat3_mul(T[b], T[a], ba);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m[i][j] = ab[i][j] - ba[i][j];
    mat3_mul(m, T[c], m);
    return creal(-2.0 * I * (m[0][0] + m[1][1] + m[2][2]));
}

/* psibar gamma^mu psi as a contravariant four-vector */
static void fcurrent(const cplx *rowbar, const cplx *col, cplx *J)
{
    for (int mu = 0; mu < 4; ++mu) {
        cplx s = 0;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) s += rowbar[r] * GAM[mu][r][c] * col[c];
        J[mu] = s;
    }
}

/* u(p1) ubar(p2) -> t(p3) tbar(p4): one s-channel gluon diagram, colour
 * (T^c)_{i3 j4} (T^c)_{j2 i1} summed explicitly. */
double or_me2_uu_tt_diagram(double mt, double gs, const double *p)
{
    gamma_init();
    const double *p1 = p, *p2 = p + 4, *p3 = p + 8, *p4 = p + 12;
    cplx T[8][3][3];
    for (int a = 0; a < 8; ++a) gellmann(a, T[a]);
    double q[4];
    for (int mu = 0; mu < 4; ++mu) q[mu] = p1[mu] + p2[mu];
    double q2 = mdot_r(q, q);
    double total = 0.0;
    for (int s1 = 0; s1 < 2; ++s1) for (int s2 = 0; s2 < 2; ++s2)
    for (int s3 = 0; s3 < 2; ++s3) for (int s4 = 0; s4 < 2; ++s4) {
        cplx u1[4], v2[4], vb2[4], u3[4], ub3[4], v4[4], Ju[4], Jt[4];
        spinor_u(p1, 0.0, s1, u1);
        spinor_v(p2, 0.0, s2, v2); bar(v2, vb2);
        spinor_u(p3, mt, s3, u3); bar(u3, ub3);
        spinor_v(p4, mt, s4, v4);
        fcurrent(vb2, u1, Ju);
        fcurrent(ub3, v4, Jt);
        /* (i g)^2 (-i / q^2) Ju.Jt */
        cplx L = (I * gs) * (I * gs) * (-I / q2) * mdot(Ju, Jt);
        for (int i1 = 0; i1 < 3; ++i1) for (int j2 = 0; j2 < 3; ++j2)
        for (int i3 = 0; i3 < 3; ++i3) for (int j4 = 0; j4 < 3; ++j4) {
            cplx c = 0;
            for (int a = 0; a < 8; ++a) c += T[a][i3][j4] * T[a][j2][i1];
            cplx M = c * L;
            total += creal(M * conj(M));
        }
    }
    return total / 36.0;
}

/* u(p1) g(p2) -> t(p3) tbar(p4) u(p5): the five tree diagrams
 *  D1 gluon absorbed on the u line before the t tbar gluon is emitted,
 *  D2 after it, D3/D4 gluon on the t / tbar side of the heavy line,
 *  D5 through the three-gluon vertex;
 * the gluon polarisation is eps (nullable: then summed over linear
 * polarisations).  Returns the sum over spins and explicit colours of |M|^2. */
static double ug_ttu_sum(double mt, double gs, const double *p, const cplx *eps_fixed)
{
    gamma_init();
    const double *p1 = p, *p2 = p + 4, *p3 = p + 8, *p4 = p + 12, *p5 = p + 16;
    cplx T[8][3][3];
    for (int a = 0; a < 8; ++a) gellmann(a, T[a]);
    static double F[8][8][8];
    static int f_ready = 0;
    if (!f_ready) {
#pragma omp critical(or_f_init)
        {
            if (!f_ready) {
                for (int a = 0; a < 8; ++a) for (int b = 0; b < 8; ++b) for (int c = 0; c < 8; ++c)
                    F[a][b][c] = fabc(T, a, b, c);
                f_ready = 1;
            }
        }
    }
    /* colour factors X_D[i1][a][i3][j4][i5] */
    static cplx X[5][3][8][3][3][3];
    static int x_ready = 0;
    if (!x_ready) {
#pragma omp critical(or_x_init)
        {
            if (!x_ready) {
                for (int i1 = 0; i1 < 3; ++i1) for (int a = 0; a < 8; ++a)
                for (int i3 = 0; i3 < 3; ++i3) for (int j4 = 0; j4 < 3; ++j4) for (int i5 = 0; i5 < 3; ++i5) {
                    cplx x[5] = { 0, 0, 0, 0, 0 };
                    for (int c = 0; c < 8; ++c) {
                        cplx ca[3][3], ac[3][3];
                        mat3_mul(T[c], T[a], ca);
                        mat3_mul(T[a], T[c], ac);
                        x[0] += ca[i5][i1] * T[c][i3][j4];
                        x[1] += ac[i5][i1] * T[c][i3][j4];
                        x[2] += T[c][i5][i1] * ac[i3][j4];
                        x[3] += T[c][i5][i1] * ca[i3][j4];
                        for (int d = 0; d < 8; ++d) x[4] += F[c][a][d] * T[c][i5][i1] * T[d][i3][j4];
                    }
                    for (int D = 0; D < 5; ++D) X[D][i1][a][i3][j4][i5] = x[D];
                }
                x_ready = 1;
            }
        }
    }
    double qtt[4], qu[4], kA[4], kB[4], kC[4], pr1[4], pr2[4], pr3[4], pr4[4];
    for (int mu = 0; mu < 4; ++mu) {
        qtt[mu] = p3[mu] + p4[mu];            /* gluon into t tbar (D1, D2) */
        qu[mu] = p1[mu] - p5[mu];             /* gluon off the u line (D3, D4, D5) */
        pr1[mu] = p1[mu] + p2[mu];            /* D1 light propagator */
        pr2[mu] = p5[mu] - p2[mu];            /* D2 light propagator */
        pr3[mu] = p3[mu] - p2[mu];            /* D3 heavy propagator */
        pr4[mu] = p3[mu] - qu[mu];            /* D4 heavy propagator */
        kA[mu] = qu[mu]; kB[mu] = p2[mu]; kC[mu] = -qtt[mu];
    }
    double q2tt = mdot_r(qtt, qtt), q2u = mdot_r(qu, qu);
    cplx S1[4][4], S2[4][4], S3[4][4], S4[4][4];
    quark_prop(pr1, 0.0, S1);
    quark_prop(pr2, 0.0, S2);
    quark_prop(pr3, mt, S3);
    quark_prop(pr4, mt, S4);
    cplx ig = I * gs;
    double total = 0.0;
    int n_pol = eps_fixed ? 1 : 2;
    for (int pol = 0; pol < n_pol; ++pol) {
        cplx eps[4];
        if (eps_fixed) memcpy(eps, eps_fixed, sizeof(eps)); else lin_pol(p2, pol, eps);
        cplx Eps[4][4];
        slash(eps, Eps);
        for (int s1 = 0; s1 < 2; ++s1) for (int s3 = 0; s3 < 2; ++s3)
        for (int s4 = 0; s4 < 2; ++s4) for (int s5 = 0; s5 < 2; ++s5) {
            cplx u1[4], u3[4], ub3[4], v4[4], u5[4], ub5[4];
            spinor_u(p1, 0.0, s1, u1);
            spinor_u(p3, mt, s3, u3); bar(u3, ub3);
            spinor_v(p4, mt, s4, v4);
            spinor_u(p5, 0.0, s5, u5); bar(u5, ub5);
            cplx L[5] = { 0, 0, 0, 0, 0 };
            cplx Jt[4], Ju[4];
            fcurrent(ub3, v4, Jt);
            fcurrent(ub5, u1, Ju);
            for (int mu = 0; mu < 4; ++mu) {
                double g = mu == 0 ? 1.0 : -1.0;   /* lower the index of gamma^mu */
                cplx Gm[4][4];
                for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) Gm[r][c] = GAM[mu][r][c];
                cplx r1[4], r2[4];
                /* D1: ubar5 (ig gamma^mu) S1 (ig epsslash) u1 * (-i/q2tt) * (ig Jt_mu) */
                row_times(ub5, Gm, r1); row_times(r1, S1, r1); row_times(r1, Eps, r1);
                L[0] += ig * ig * row_col(r1, u1) * (-I / q2tt) * ig * g * Jt[mu];
                /* D2: ubar5 (ig epsslash) S2 (ig gamma^mu) u1 */
                row_times(ub5, Eps, r2); row_times(r2, S2, r2); row_times(r2, Gm, r2);
                L[1] += ig * ig * row_col(r2, u1) * (-I / q2tt) * ig * g * Jt[mu];
                /* D3: ubar3 (ig epsslash) S3 (ig gamma^mu) v4 * (-i/q2u) * (ig Ju_mu) */
                row_times(ub3, Eps, r1); row_times(r1, S3, r1); row_times(r1, Gm, r1);
                L[2] += ig * ig * row_col(r1, v4) * (-I / q2u) * ig * g * Ju[mu];
                /* D4: ubar3 (ig gamma^mu) S4 (ig epsslash) v4 */
                row_times(ub3, Gm, r2); row_times(r2, S4, r2); row_times(r2, Eps, r2);
                L[3] += ig * ig * row_col(r2, v4) * (-I / q2u) * ig * g * Ju[mu];
            }
            /* D5: (ig Ju)_mu (-i/kA^2) g V^{mu nu rho}(kA,kB,kC) eps_nu (-i/kC^2) (ig Jt)_rho */
            {
                double a[4], b[4], c[4];
                for (int mu = 0; mu < 4; ++mu) { a[mu] = kA[mu] - kB[mu]; b[mu] = kB[mu] - kC[mu]; c[mu] = kC[mu] - kA[mu]; }
                cplx ac[4] = { a[0], a[1], a[2], a[3] }, bc[4] = { b[0], b[1], b[2], b[3] }, cc[4] = { c[0], c[1], c[2], c[3] };
                cplx V = mdot(Ju, eps) * mdot(ac, Jt) + mdot(eps, Jt) * mdot(bc, Ju) + mdot(Jt, Ju) * mdot(cc, eps);
                L[4] = ig * ig * gs * (-I / q2u) * (-I / q2tt) * V;
            }
            for (int i1 = 0; i1 < 3; ++i1) for (int a = 0; a < 8; ++a)
            for (int i3 = 0; i3 < 3; ++i3) for (int j4 = 0; j4 < 3; ++j4) for (int i5 = 0; i5 < 3; ++i5) {
                cplx M = 0;
                for (int D = 0; D < 5; ++D) M += X[D][i1][a][i3][j4][i5] * L[D];
                total += creal(M * conj(M));
            }
        }
    }
    return total;
}

double or_me2_ug_ttu(double mt, double gs, const double *p)
{
    return ug_ttu_sum(mt, gs, p, NULL) / 96.0;
}

double or_amp2_ug_ttu_ward(double mt, double gs, const double *p)
{
    cplx k[4] = { p[4], p[5], p[6], p[7] };
    return ug_ttu_sum(mt, gs, p, k);
}

/* ---------------------------------------------------------------- dispatch */

int or_proc_info_get(int proc, or_proc_info *o)
{
    switch (proc) {
    case OR_EE_MUMU: *o = (or_proc_info){ 4, 2, 2, 16, 0, 0.25, 1.0 }; return 0;
    case OR_GG_TT:   *o = (or_proc_info){ 4, 2, 10, 16, 2, 1.0 / 256.0, 1.0 }; return 0;
    case OR_UU_TT:   *o = (or_proc_info){ 4, 2, 10, 16, 2, 1.0 / 36.0, 1.0 }; return 0;
    case OR_GG_TTG:  *o = (or_proc_info){ 5, 3, 14, 32, 3, 1.0 / 256.0, 1.0 }; return 0;
    case OR_UG_TTU:  *o = (or_proc_info){ 5, 3, 14, 32, 3, 1.0 / 96.0, 1.0 }; return 0;
    case OR_GG_TTGG: *o = (or_proc_info){ 6, 4, 18, 64, 4, 1.0 / 256.0, 0.5 }; return 0;
    case OR_GG_TTGGG: *o = (or_proc_info){ 7, 5, 22, 128, 5, 1.0 / 256.0, 1.0 / 6.0 }; return 0;
    }
    return 1;
}

double or_me2(int proc, const or_params *P, const double *p)
{
    double gs = sqrt(4.0 * M_PI * P->alpha_s);
    switch (proc) {
    case OR_EE_MUMU: return or_me2_ee_mumu_closed(P, p);
    case OR_GG_TT:   return or_me2_bg(2, p, 2, P->mt, gs) / 256.0;
    case OR_UU_TT:   return or_me2_uu_tt_closed(P->mt, gs, p);
    case OR_GG_TTG:  return or_me2_bg(3, p, 2, P->mt, gs) / 256.0;
    case OR_UG_TTU:  return or_me2_ug_ttu(P->mt, gs, p);
    case OR_GG_TTGG: return or_me2_bg(4, p, 2, P->mt, gs) / 256.0 * 0.5;
    case OR_GG_TTGGG: return or_me2_bg(5, p, 2, P->mt, gs) / 256.0 / 6.0;
    }
    return 0.0;
}

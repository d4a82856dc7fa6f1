/*
 * Plain FP64 CPU oracle for the leading-order Monte Carlo integrand of
 * "Towards the automation of Monte Carlo simulation on GPU for particle
 * physics processes" (Carrazza, Cruz-Martinez, Rossi, Zaro; arXiv:2105.10529).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only tests/, the smoke
 * check and the CPU-baseline leg of bench.py may load it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Pipeline order follows Sec. 2.1 of the paper (random numbers -> phase-space
 * kinematics -> matrix element -> histogram accumulation), with the
 * integrator, PDF interpolation, phase-space generator with fiducial cuts and
 * the squared matrix element as the four ingredients listed in Sec. 1.
 *
 * Parity status per function (details in each source file):
 *   philox / uniforms ....... pinned (independent library Philox, bijection)
 *   vegas map / refine ...... pinned (identity grid, closed-form rebinning)
 *   parton map .............. pinned (closed-form luminosity-area integral)
 *   rambo ................... pinned (massless volume, massive 2-body beta/8pi,
 *                             3-body massive volume by 1-D quadrature)
 *   cuts, scale ............. pinned (hand-built momenta)
 *   pdf bicubic ............. pinned (exact on quadratics, node values)
 *   me2 e+e- -> mu+mu- ...... closed form; pinned (QED limit, total sigma)
 *   me2 q qbar -> t tbar .... closed form; pinned (sigma-hat closed form)
 *   me2 gg -> t tbar (+g..) . Berends-Giele, up to three final gluons; pinned
 *                             (Combridge closed form, Ward identity, Lorentz
 *                             invariance, Bose symmetry, massless MHV ratios,
 *                             collinear factorisation chains k -> k - 1,
 *                             explicit colour sums)
 *   me2 u g -> t tbar u ..... explicit Feynman diagrams, explicit colour;
 *                             pinned (Ward identity, Lorentz invariance; the
 *                             same diagram machinery reproduces the u ubar ->
 *                             t tbar closed form)
 *   colour matrices ......... brute force over Gell-Mann matrices; pinned
 *                             (Casimir diagonal, SU(3) identities)
 */
#ifndef MF_ORACLE_H
#define MF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Process numbering (same meaning as the library's enum, defined here on its own). */
enum { OR_EE_MUMU = 0, OR_GG_TT = 1, OR_UU_TT = 2, OR_GG_TTG = 3, OR_UG_TTU = 4, OR_GG_TTGG = 5, OR_GG_TTGGG = 6 };

typedef struct {
    double sqrt_s;        /* collider (or e+e-) energy, GeV                        */
    double mt;            /* top mass, GeV                                         */
    double alpha_s;       /* fixed strong coupling                                 */
    double mz, wz;        /* Z mass and width, GeV                                 */
    double alpha_em_inv;  /* 1/alpha_em                                            */
    double gf;            /* Fermi constant, GeV^-2                                */
    double pt_min;        /* cut on final light partons, GeV (<=0 disables)        */
    double eta_max;       /* cut on |eta| of final light partons (<=0 disables)    */
    double dr_min;        /* Delta R between final gluons (<=0 disables)           */
    uint64_t seed;        /* Philox key                                             */
    uint32_t channel;     /* channel id folded into the Philox counter              */
    int n_bins;           /* VEGAS bins per dimension                               */
    double alpha;         /* VEGAS damping exponent                                 */
} or_params;

/* Per-process static data. */
typedef struct {
    int n_ext;           /* external particles (incoming first)                 */
    int n_final;         /* final-state particles                               */
    int dim;             /* VEGAS dimension                                     */
    int n_hel;           /* helicity combinations                               */
    int as_power;        /* power k of alpha_s in |M|^2                         */
    double avg;          /* initial spin x colour average                       */
    double sym;          /* identical final-state symmetry factor               */
} or_proc_info;

int or_proc_info_get(int proc, or_proc_info *out);

/* Philox4x32-10 (Salmon et al., SC'11) and the per-event uniform stream: the random
 * numbers that start the paper's event pipeline (Sec. 2.1) */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t a, uint32_t b);
void or_uniforms(uint64_t seed, uint64_t event, uint32_t iteration, uint32_t channel,
                 int dim, double *u);

/* VEGAS (Lepage 1978; the paper's integrator, Sec. 1): map, grid refinement and the
 * combination of iterations */
void or_vegas_init(double *grid, int dim, int nb);
double or_vegas_map(const double *grid, int dim, int nb, const double *u, double *x, uint8_t *bins);
void or_vegas_refine(const double *hist, double *grid, int dim, int nb, double alpha);
void or_vegas_combine(int n_iter, const double *I, const double *var,
                      double *mean, double *err, double *chi2dof);

/* parton-luminosity map from two uniforms to x1, x2 (a choice of this library; the
 * paper does not give one) */
void or_parton_map(double x0, double v, double tau0, double *x1, double *x2, double *jac);

/* RAMBO (Kleiss, Stirling, Ellis 1986) with the massive rescaling; output momenta
 * (E,px,py,pz) in the partonic rest frame */
int or_rambo(int n, double sqrt_shat, const double *masses, const double *u, double *p, double *weight);
double or_rambo_massless_volume(int n, double shat);

/* fiducial cuts and factorisation scale (Sec. 2.1: phase space with cuts) */
int or_cuts(int proc, const or_params *P, const double *plab /* n_ext x 4 */);
double or_muf2(int proc, const or_params *P, const double *p /* n_ext x 4 */);

/* log-bicubic PDF interpolation (the PDF stage of Sec. 1, LHAPDF6 scheme).  grid: n_flav x nx x nq values of x f(x,Q^2) on
 * ln-uniform nodes x in [x_min,1], Q^2 in [q2_min,q2_max]. */
typedef struct {
    const double *xf; int n_flav, nx, nq;
    double x_min, q2_min, q2_max;
} or_pdf;
double or_pdf_xf(const or_pdf *pdf, int flav, double x, double q2);

/* squared matrix elements (Sec. 2.2), spin/colour averaged, including the
 * identical-particle factor; momenta n_ext x 4, incoming first. */
double or_me2(int proc, const or_params *P, const double *p);
double or_me2_ee_mumu_closed(const or_params *P, const double *p);
double or_me2_gg_tt_closed(double mt, double gs, const double *p);
double or_me2_uu_tt_closed(double mt, double gs, const double *p);
/* Berends-Giele: gluons with momenta kg (incoming convention, k x 4),
 * polarisation vectors eps (k x 4 complex as re,im pairs), t (p3), tbar (p4);
 * spins s3,s4 in {0,1}; perm: colour ordering.  Returns the partial amplitude. */
void or_bg_partial(int k, const double *kg, const double *eps, const double *p3, const double *p4,
                   double m, double gs, int s3, int s4, const int *perm, double *amp_re_im);
double or_me2_bg(int k, const double *p_all, int n_in_gluons, double m, double gs);
/* colour matrix C[s][t] = sum_colours conj((T^s)_ij) (T^t)_ij over orderings of k gluons
 * (orderings enumerated lexicographically), by brute force over Gell-Mann matrices;
 * k <= 5 (120 orderings). */
void or_colour_matrix(int k, double *C);
/* Gell-Mann generators T^a = lambda^a/2, a=0..7: 3x3 complex as re,im pairs */
void or_gellmann_T(int a, double *T);
/* explicit Feynman diagrams with explicit colour indices: u g -> t tbar u, and
 * u ubar -> t tbar through the same machinery (pinned by its closed form) */
double or_me2_ug_ttu(double mt, double gs, const double *p);
double or_me2_uu_tt_diagram(double mt, double gs, const double *p);
/* u g -> t tbar u with the gluon polarisation replaced by its momentum: sum over
 * spins and colours of |M|^2, which gauge invariance sets to zero (Ward test) */
double or_amp2_ug_ttu_ward(double mt, double gs, const double *p);

/* the whole per-event integrand (Sec. 2.1): random numbers to event weight */
typedef struct {
    double u[32], x[32];
    uint8_t bins[32];
    double jac_vegas, x1, x2, shat, jac_parton, w_ps;
    double p[7][4];     /* partonic rest frame */
    double plab[7][4];  /* lab frame */
    int mask;
    double muf2, f1, f2, me2;
    double w;           /* event weight f*J (pb), before the 1/N of the estimator */
} or_event_out;

int or_event(int proc, const or_params *P, const or_pdf *pdf, const double *grid,
             uint64_t event, uint32_t iteration, const int *mask_override, or_event_out *o);
/* or_event for n listed events, threads over events (n_threads <= 0: all) */
int or_events(int proc, const or_params *P, const or_pdf *pdf, const double *grid, const uint64_t *events,
              int64_t n, uint32_t iteration, or_event_out *out, int n_threads);

/* one VEGAS pass over events [0,n) at fixed grid: sums of w and w^2 (w includes 1/n)
 * and the histogram hist[d][b] += w^2.  mask_in (nullable) freezes cut masks,
 * mask_out (nullable) records them. */
int or_pass(int proc, const or_params *P, const or_pdf *pdf, const double *grid, int64_t n,
            uint32_t iteration, const uint8_t *mask_in, uint8_t *mask_out,
            double *sum_w, double *sum_w2, double *hist, int64_t *n_pass, int n_threads);
/* observable histogram (p_T of the first final-state particle), see or_integrand.c */
int or_obs_bin(double px, double py, int nobs, double lo, double hi);
int or_pass_obs(int proc, const or_params *P, const or_pdf *pdf, const double *grid, int64_t n,
                uint32_t iteration, int nobs, double lo, double hi, double *sum_w, double *sum_w2,
                double *obs, int n_threads);

typedef struct {
    double sigma, error, chi2dof;
    int64_t n_pass;
} or_result;

/* full integration: n_iter passes, refine between them; grid_io (nullable) receives the
 * final grid; per_iter (nullable) receives I_k, var_k pairs. */
int or_integrate(int proc, const or_params *P, const or_pdf *pdf, int64_t n, int n_iter,
                 double *grid_io, double *per_iter, or_result *res, int n_threads);
/* the same with the observable histogram: obs_hist, obs_err [nobs + 2] combined over the
 * iterations, obs_iter (nullable) [n_iter][nobs + 2][2] per-iteration (sum w/N, variance) */
int or_integrate_obs(int proc, const or_params *P, const or_pdf *pdf, int64_t n, int n_iter,
                     int nobs, double lo, double hi, double *obs_hist, double *obs_err, double *obs_iter,
                     or_result *res, int n_threads);

#ifdef __cplusplus
}
#endif
#endif

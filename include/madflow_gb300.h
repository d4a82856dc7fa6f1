/*
 * madflow_gb300 -- C ABI of the GB300 (sm_103a) leading-order Monte Carlo
 * integrand of arXiv:2105.10529 ("Towards the automation of Monte Carlo
 * simulation on GPU for particle physics processes", Carrazza, Cruz-Martinez,
 * Rossi, Zaro).
 *
 * The paper (Sec. 1, Sec. 2.1) states the problem as: integrate a process
 * over phase space with a VEGAS integrator that draws random numbers, builds
 * the phase-space kinematics with fiducial cuts, interpolates PDFs, evaluates
 * the squared matrix element of Sec. 2.2 and accumulates histograms, with
 * every step on the GPU and results kept in GPU memory (Sec. 3.1).  The two
 * user calls are therefore
 *     integrate(process, sqrt_s, cuts, n_events, n_iter) -> sigma, error
 *     evaluate(process, momenta)                         -> |M|^2
 * plus the single-pass and inspection calls that the tests and the
 * benchmark use.
 *
 * Conventions of every call:
 *  - Return value: MF_OK (0) or an mf_status error code.  No C++ exception
 *    crosses the ABI.  mf_last_error() gives a one-line reason.
 *  - Pointers named *_dev are CUDA device pointers owned by the caller;
 *    pointers named *_host are host pointers owned by the caller.  The
 *    library owns only the buffers inside mf_ctx.
 *  - All device work runs on the stream given to mf_create (NULL = legacy
 *    default stream).  Calls that return host results synchronise that
 *    stream before returning; calls that only write device buffers do not.
 *  - Momenta are (E, px, py, pz) in GeV, float64, laid out [event][particle][4]
 *    with the incoming particles first, in the process order listed below.
 *  - Cross sections are in pb.
 */
#ifndef MADFLOW_GB300_H
#define MADFLOW_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define MF_ABI_VERSION 1

/* Processes (particle order of the momenta):
 *   MF_EE_MUMU  e-(1) e+(2) -> mu-(3) mu+(4), photon + Z, massless
 *   MF_GG_TT    g(1) g(2) -> t(3) tbar(4)
 *   MF_UU_TT    u(1) ubar(2) -> t(3) tbar(4)
 *   MF_GG_TTG   g(1) g(2) -> t(3) tbar(4) g(5)
 *   MF_UG_TTU   u(1) g(2) -> t(3) tbar(4) u(5)
 *   MF_GG_TTGG  g(1) g(2) -> t(3) tbar(4) g(5) g(6)
 *   MF_GG_TTGGG g(1) g(2) -> t(3) tbar(4) g(5) g(6) g(7)  (the multi-leg
 *               extension of Sec. 4: its matrix element is a warp-level
 *               Berends-Giele recursion; no derivatives, not in batches)      */
enum mf_process { MF_EE_MUMU = 0, MF_GG_TT = 1, MF_UU_TT = 2, MF_GG_TTG = 3, MF_UG_TTU = 4, MF_GG_TTGG = 5,
                  MF_GG_TTGGG = 6 };

/* Arithmetic of the integrand: MF_FP64 everywhere in FP64; MF_MIXED
 * evaluates wavefunctions, vertices and the colour sum in FP32, computes the
 * phase space, Jacobians, PDFs, propagator denominators and the spinor and
 * polarisation bases in double-float arithmetic (a value as the sum of two
 * floats, about 48 bits, on the FP32 pipes; the VEGAS bins and cut decisions
 * are those of the FP64 path), and keeps FP64 for event weights and all
 * accumulations.  mf_evaluate and the derivative calls take FP64 momenta and
 * form the per-event pieces in FP64, except the g g -> t tbar g g record of
 * the recycled recursion, formed in double-float. */
enum mf_precision { MF_FP64 = 0, MF_MIXED = 1 };

enum mf_status {
    MF_OK = 0,
    MF_ERR_ARG = 1,          /* invalid argument (null pointer, size out of range, unknown process) */
    MF_ERR_CUDA = 2,         /* a CUDA runtime call failed; the reason is in mf_last_error           */
    MF_ERR_TIMEOUT = 3,      /* a bounded device wait ran out                                        */
    MF_ERR_NUMERIC = 4,      /* more non-finite event weights than allowed (they are zeroed)         */
    MF_ERR_UNSUPPORTED = 5   /* process or option not built into this library                        */
};

/* Physics and integrator settings (GeV units).  mf_default_config fills the
 * values of the synthetic workloads: m_t = 173, alpha_s = 0.118 (fixed),
 * M_Z = 91.188, Gamma_Z = 2.441404, 1/alpha = 132.507, G_F = 1.16639e-5,
 * pT > 30, |eta| < 2.5, Delta R > 0.4 on final light partons, 50 bins,
 * alpha = 1.5, seed 0, channel 0, MF_MIXED. */
typedef struct mf_config {
    double mt;            /* top mass                                              */
    double alpha_s;       /* strong coupling, fixed                                */
    double mz, wz;        /* Z mass and width                                      */
    double alpha_em_inv;  /* 1 / alpha_em                                          */
    double gf;            /* Fermi constant (GeV^-2); sets M_W and sin^2(theta_W)  */
    double pt_min;        /* light-parton pT cut (<= 0 disables)                   */
    double eta_max;       /* light-parton |eta| cut (<= 0 disables)                */
    double dr_min;        /* Delta R cut between final gluons (<= 0 disables)      */
    unsigned long long seed;  /* Philox key                                        */
    unsigned int channel;     /* channel id in the Philox counter (0..2^24-1)      */
    int n_bins;           /* VEGAS bins per dimension, 2..64                        */
    double alpha;         /* VEGAS damping exponent                                */
    int precision;        /* mf_precision                                          */
} mf_config;

typedef struct mf_result {
    double sigma_pb;          /* inverse-variance weighted mean over iterations     */
    double error_pb;          /* its standard error                                 */
    double chi2_dof;          /* chi^2 of the iteration estimates per d.o.f.        */
    long long n_events_total; /* events evaluated                                   */
    long long n_pass;         /* events passing the cuts                            */
    long long n_nan;          /* non-finite weights set to zero                     */
    int n_iter;
    /* with want_grads: d sigma / d m_t [pb/GeV] and its Monte Carlo error, and
     * d sigma / d alpha_s [pb], from one derivative pass at the final grid
     * (fresh random numbers); 0 otherwise */
    double dsigma_dmt, dsigma_dmt_error, dsigma_dalphas;
} mf_result;

/* Fiducial cuts on the final light partons (Sec. 1: phase space with cuts):
 * pT > pt_min [GeV], |eta| < eta_max, Delta R between every pair of final
 * gluons > dr_min.
 * A value <= 0 (or an infinite eta_max) disables that cut. */
typedef struct mf_cuts {
    double pt_min, eta_max, dr_min;
} mf_cuts;

/* Per-event outputs of mf_vegas_pass (device pointers, each nullable):
 * u, x: [n][dim] uniforms and VEGAS-mapped points; bins: [n][dim] bin
 * indices; w: [n] event weight f J in pb (before the 1/N of the estimator);
 * mask: [n] cut mask; me2: [n] averaged |M|^2 (0 where the cuts fail);
 * momenta: [n][n_ext][4] partonic-frame momenta. */
typedef struct mf_event_arrays {
    double *u, *x;
    unsigned char *bins;
    double *w;
    unsigned char *mask;
    double *me2;
    double *momenta;
} mf_event_arrays;

int mf_default_config(mf_config *cfg);

/* Number of external particles and the VEGAS dimension of a process
 * (D = 2 for MF_EE_MUMU, 2 + 4 n_final otherwise).  MF_ERR_ARG for an
 * unknown process. */
int mf_process_info(int process, int *n_ext, int *dim);

/* Create a context on the current CUDA device.  pdf_grid_host: x f(x,Q^2)
 * on ln-uniform nodes, layout [flavour][ix][iq] with flavours 0 gluon,
 * 1 u, 2 ubar (n_flav >= 1; the gluon processes read flavour 0), copied to
 * the device.  stream: a cudaStream_t or NULL.  On success *out owns device
 * buffers sized for every built process (about 100 MB on a 152-SM GPU:
 * per-CTA partial sums, the heavy integrand's kinematics store and the
 * per-event records of schedules 3 and 4; the batch calls add their own on
 * first use); release with mf_destroy. */
int mf_create(struct mf_ctx **out, const mf_config *cfg, const double *pdf_grid_host, int n_flav, int nx, int nq,
              double x_min, double q2_min, double q2_max, void *stream);
void mf_destroy(struct mf_ctx *ctx);
const char *mf_last_error(const struct mf_ctx *ctx);
int mf_set_precision(struct mf_ctx *ctx, int precision);
/* Integrand schedule for the heavy processes (gg -> t tbar g, gg -> t tbar g g):
 * 0 = warps run freely through the helicity sum, 1 = a CTA barrier after every
 * helicity keeps the CTA's warps on the same instructions,
 * 2 = as 1, and for g g -> t tbar g g in MF_MIXED the colour sum of every
 * helicity (24 x 24 colour matrix, Sec. 2.2) runs on the tensor cores as one
 * (128 events x 24) x (24 x 24) contraction per 128 threads (tcgen05, bf16 split of the
 * colour-flow amplitudes, FP32 accumulation in tensor memory); elsewhere 2 acts
 * as 1.  3 = the warp-per-event schedule of g g -> t tbar g g in MF_MIXED (no
 * counterpart in the paper, whose kernels give one thread per event): one warp per
 * event, its 32 lanes evaluating the 32 helicities of the parity-halved sum of
 * Sec. 2.2 at once, the colour sum on the tensor cores as in 2, and the event's
 * sum over its lanes by a fixed shuffle tree.  The warp shares one copy of the
 * event's helicity-independent pieces, so the kernel needs far less shared memory
 * and the SM's L1 keeps more of the matrix element's local memory.  The helicity
 * split and the other processes run 3 as 2.
 * 4 (the default) = for g g -> t tbar g g in MF_MIXED, one warp per event with the
 * helicity-recycled Berends-Giele recursion (the same |M|^2 as Sec. 2.2's helicity
 * loop, re-associated; no counterpart in the paper): every off-shell current is
 * evaluated once per combination of the helicities it depends on, the colour-ordered
 * partial amplitudes of the 32 configurations follow from five complex contractions
 * each, and the colour sum runs on the tensor cores as in 3.  It needs the context's
 * record region (one CTA per SM); the helicity split runs it as 2 and the other
 * processes as 3.
 * Schedules 0 and 1 give identical results; 2, 3 and 4 differ from them and from
 * each other by FP32 rounding.  MF_ERR_ARG for other values. */
int mf_set_schedule(struct mf_ctx *ctx, int sched);
/* Observable histogram (Sec. 2.1: the pipeline ends in histogram accumulation;
 * Sec. 3, Fig. 2: the leading-order cross section differential in p_T): the
 * transverse momentum of the first final-state particle (the top quark in the
 * top-pair processes, the muon in e+ e- -> mu+ mu-), sqrt(px^2 + py^2) in FP64,
 * in n_bins (1 .. 100) uniform bins on [lo, hi).  Bin j = 0 holds p_T < lo
 * (and a non-finite p_T), j = n_bins + 1 holds p_T >= hi, else
 * j = 1 + floor((p_T - lo) n_bins / (hi - lo)). */
typedef struct mf_obs {
    int n_bins;
    double lo, hi;
} mf_obs;
/* Enables (spec with n_bins >= 1) or disables (NULL or n_bins = 0) the
 * histogram for the following mf_integrate calls (not the batch or pass
 * calls).  Every iteration fills sum w/N per bin from the same weights as
 * the integral; the iterations combine with the integral's inverse-variance
 * weights, so the n_bins + 2 bins add up to sigma.  Allocates about 10 MB on
 * first use.  MF_ERR_ARG for a bad spec (n_bins outside 0..100, hi <= lo,
 * non-finite edges). */
int mf_set_observable(struct mf_ctx *ctx, const mf_obs *spec);
/* The histogram of the last mf_integrate since mf_set_observable (host
 * buffers, caller-owned, each nullable): hist_host [n_bins + 2] in pb per bin
 * (divide by the bin width for d sigma / d p_T), err_host [n_bins + 2] their
 * Monte Carlo errors, iter_host [n_iter][n_bins + 2][2] each iteration's
 * (sum w/N, variance) per bin.  MF_ERR_ARG when there is none. */
int mf_get_observable(struct mf_ctx *ctx, double *hist_host, double *err_host, double *iter_host);

/* Helicity split of the heavy integrand (no counterpart in the paper, whose
 * kernels give one thread per event): parts = 1 (the default), one thread
 * sums every helicity of its event; parts = 2, two threads of a CTA (t and
 * t + half the CTA, in different warps) share an event, each summing every
 * other one of the helicities the matrix element evaluates (Sec. 2.2's
 * helicity sum split in two), and the pair adds its halves; a CTA then
 * holds half as many events at a time.  Applies to
 * g g -> t tbar g and g g -> t tbar g g in MF_MIXED under schedules 1, 2 and 3
 * (with 3 it runs schedule 2's kernel), in mf_vegas_pass without per-event
 * outputs and in mf_integrate; elsewhere it acts as 1.  Results differ from parts = 1 by FP32 rounding only.
 * MF_ERR_ARG for other values. */
int mf_set_helicity_split(struct mf_ctx *ctx, int parts);

/* Helicity sampling (the paper's matrix element sums every helicity
 * configuration, Sec. 2.2; sampling them is a variance-for-cost trade of the
 * Monte Carlo that keeps its expectation): n_samples = 0 (the default) sums
 * them all; n_samples = 1, 2, 4, ..., 32 makes each event of g g -> t tbar g g g
 * evaluate n_samples of the 64 parity-halved configurations instead, one drawn
 * uniformly from each of n_samples equal strata of consecutive configurations
 * (configuration 2j + 1, j = 0 .. 63, stands for the pair {2j + 1, 126 - 2j}),
 * weighted by the stratum size 64 / n_samples.  The per-event |M|^2 is then an
 * unbiased estimate of the summed one, and the cross section's expectation is
 * unchanged while its variance grows.  The draws are reproducible: stratum s
 * of event e takes bits [s b, (s + 1) b) (b = log2(64 / n_samples)) of
 * Philox4x32-10 (Salmon et al. 2011) at counter (e lo, e hi, iteration,
 * channel << 8 | 0xFF), a counter block no VEGAS dimension uses, with the key
 * (seed lo ^ 0x68656C69 ^ stream, seed hi); `stream` selects independent draws
 * over the same events.  n_samples = 64 is the full sum.  Applies to
 * mf_integrate, mf_integrate_grid and mf_vegas_pass (its per-event |M|^2 is
 * the estimate); mf_evaluate, mf_helicity_profile, the derivative calls, the
 * batch calls and mf_vegas_pass_static always sum every configuration, and
 * so do the other processes.  MF_ERR_ARG for other values. */
int mf_set_helicity_sampling(struct mf_ctx *ctx, int n_samples, unsigned int stream);

/* Synchronises the context's stream and reports whether a bounded device-side
 * wait ran out since the last check (MF_ERR_TIMEOUT; the flag is cleared) or
 * not (MF_OK).  mf_integrate makes the same check before returning. */
int mf_device_status(struct mf_ctx *ctx);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * warp waits on an mbarrier phase that nothing completes, with at most
 * `iterations` (1 .. 2^20) polls, the same bounded wait the tensor-core colour
 * sum uses; the expiry raises the context's device error flag.  Returns what
 * mf_device_status then returns: MF_ERR_TIMEOUT when the mechanism works.
 * The context stays usable.  Synchronises. */
int mf_selftest_wait(struct mf_ctx *ctx, unsigned int iterations);
/* Replace the PDF grid (same shape as at creation) by a host copy. */
int mf_set_pdf(struct mf_ctx *ctx, const double *pdf_grid_host);

/* integrate (Sec. 2.1): n_iter VEGAS iterations of n_events each on a
 * uniform starting grid, the grid refined after every iteration but the
 * last; all iterations enter the weighted mean.  cuts (host, nullable): the
 * fiducial cuts of this call, NULL for those of the configuration.
 * n_events >= 2, 1 <= n_iter <= 1000.  want_grads != 0: one more pass of
 * n_events at the final grid gives out->dsigma_dmt (with its error) and
 * out->dsigma_dalphas (as mf_vegas_pass_grad; MF_ERR_UNSUPPORTED where that
 * has no kernel).  iter_host (nullable): [n_iter][2] estimate and variance
 * per iteration; grid_host (nullable): [dim][n_bins+1] final grid.
 * The iterations (integrand, end-of-pass reduction and refinement, and the
 * observable's reduction) are captured once as a CUDA graph on a private
 * stream, ordered after the work queued on the context's stream; a later
 * call with the same process, sizes, cuts, couplings, schedule and
 * observable replays it.  The context keeps the graphs of its 16 most
 * recently used parameter sets, so channels integrated in turn are each
 * replayed.  Synchronises. */
int mf_integrate(struct mf_ctx *ctx, int process, double sqrt_s, const mf_cuts *cuts, long long n_events, int n_iter,
                 int want_grads, mf_result *out_host, double *iter_host, double *grid_host);

/* integrate from a caller grid (no counterpart in the paper: it resumes an
 * adaptation, e.g. one started by mf_vegas_pass / mf_vegas_refine): as
 * mf_integrate, but the first iteration uses grid_in_host [dim][n_bins+1]
 * (host, caller-owned, copied) instead of the uniform grid, and iteration j
 * draws its random numbers from Philox iteration first_iteration + j (the
 * derivative pass from first_iteration + n_iter).  MF_ERR_ARG when
 * grid_in_host is NULL.  Like mf_integrate, its iterations are captured once
 * as a CUDA graph and replayed.  Synchronises. */
int mf_integrate_grid(struct mf_ctx *ctx, int process, double sqrt_s, const mf_cuts *cuts, long long n_events,
                      int n_iter, unsigned int first_iteration, const double *grid_in_host, int want_grads,
                      mf_result *out_host, double *iter_host, double *grid_host);

/* One VEGAS pass over events [ev_offset, ev_offset + n_events) of Philox
 * iteration `iteration` at a caller grid (grid_dev: [dim][n_bins+1]).
 * sums_dev: [2 + dim n_bins] receives sum w, sum w^2 and the histogram
 * of w^2 (w includes the 1/n_events of the estimator).  mask_in_dev
 * (nullable, [n_events]) freezes the cut masks.  ev (nullable) requests the
 * per-event outputs (device arrays, caller-owned; a NULL member is skipped):
 * u, x [n_events][dim], bins [n_events][dim], w, mask, me2 [n_events],
 * momenta [n_events][n_ext][4] in the partonic rest frame.  Under schedules 3
 * and 4 and the helicity split the pass with outputs runs the very kernel that runs
 * without them (the stores are a run-time choice), so its outputs are those
 * of the timed configuration.  Does not synchronise. */
int mf_vegas_pass(struct mf_ctx *ctx, int process, double sqrt_s, const double *grid_dev, long long n_events,
                  long long ev_offset, unsigned int iteration, const unsigned char *mask_in_dev, double *sums_dev,
                  const mf_event_arrays *ev);

/* VEGAS grid refinement (Sec. 1, the VegasFlow integrator; Lepage 1978)
 * from the sums of one or more passes: sums_dev [2 + dim n_bins] as
 * written by mf_vegas_pass (several ranks' sums may be combined first: the
 * refinement depends only on the shape of each dimension's histogram),
 * grid_dev [dim][n_bins+1] updated in place; a dimension whose histogram is
 * all zero keeps its edges.  dim <= 22, 2 <= n_bins <= 64, alpha >= 0.
 * Does not synchronise. */
int mf_vegas_refine(struct mf_ctx *ctx, int dim, int n_bins, double alpha, const double *sums_dev, double *grid_dev);

/* One VEGAS pass like mf_vegas_pass, for callers that cannot allocate GPU
 * memory (no context is created and nothing is allocated).  The paper has
 * no counterpart: this exists for hosts that own all device memory and
 * forbid allocation in their callbacks, or that must not let a call
 * synchronise the device as cudaMalloc may.
 * Inputs: cfg (host), pdf_dev [n_flav][nx][nq] and grid_dev [dim][n_bins+1]
 * (device, caller-owned, same meaning as for mf_create / mf_vegas_pass).
 * Output: sums_dev [2 + dim n_bins] (device): sum w, sum w^2, histogram.
 * Kernel: integrand schedule 0 (one event per thread, colour sum on the FMA
 * pipes) whatever the precision; for g g -> t tbar g g in MF_MIXED its sums
 * therefore differ from a context's default schedule 4 by FP32 rounding
 * (a few 1e-6 relative) and it runs slower.
 * Scratch: a fixed 4 MiB array inside the library (the per-CTA partial
 * sums and two counters), held by every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address; make that first call before any stream capture.  Every call
 * shares the array and overwrites it, so calls whose work overlaps on the GPU
 * (other streams, other host threads) race: serialise them.  Sizes whose
 * partial sums do not fit (2 + dim n_bins doubles per CTA) return MF_ERR_ARG;
 * other errors as for mf_vegas_pass.  stream: cudaStream_t or NULL.  Does not
 * synchronise. */
int mf_vegas_pass_static(int process, const mf_config *cfg, double sqrt_s, const double *pdf_dev, int n_flav, int nx,
                         int nq, double x_min, double q2_min, double q2_max, const double *grid_dev, long long n_events,
                         long long ev_offset, unsigned int iteration, double *sums_dev, void *stream);

/* Replace m_t and alpha_s of the context (both > 0; MF_ERR_ARG otherwise). */
int mf_set_couplings(struct mf_ctx *ctx, double mt, double alpha_s);

/* Derivative pass of the estimator sigma_hat = (1/N) sum_e w_e at a fixed
 * grid (grid_dev [dim][n_bins+1]), events [ev_offset, ev_offset + n_events)
 * of Philox iteration `iteration`, with every cut mask fixed at the base point
 * (or given by mask_in_dev [n_events], nullable): the pathwise derivative
 * of the Monte Carlo estimate.  Forward mode: each event's weight and its
 * m_t derivative come out of one evaluation of the whole integrand (parton
 * map, RAMBO with its mass rescaling, scale, PDFs, matrix element),
 * recomputed from the random numbers and stored nowhere.
 * out_dev [4] (device): sigma_hat, d sigma_hat / d m_t, sum_e (dw_e/dm_t / N)^2
 * (for the MC error of the derivative) and d sigma_hat / d alpha_s.
 * Top-pair processes only (MF_ERR_UNSUPPORTED for e+ e- -> mu+ mu-); for
 * g g -> t tbar g g only the MF_MIXED derivative is built.  Does not
 * synchronise. */
int mf_vegas_pass_grad(struct mf_ctx *ctx, int process, double sqrt_s, const double *grid_dev, long long n_events,
                       long long ev_offset, unsigned int iteration, const unsigned char *mask_in_dev, double *out_dev);

/* evaluate (Sec. 2.2): spin- and colour-averaged |M|^2 (identical-particle
 * factor included) of n phase-space points.  momenta_dev: [n][n_ext][4]
 * (E, px, py, pz), incoming first; me2_dev: [n] (nullable when dme2_dp_dev
 * is given).  dme2_dp_dev (nullable): [n][n_ext][4] derivatives of |M|^2 with
 * respect to every momentum component, the components taken as independent
 * variables of the library's formula (top-pair processes only,
 * MF_ERR_UNSUPPORTED otherwise).  For the gluon processes (g g -> t tbar plus
 * 0 to 3 gluons, FP64 and MF_MIXED) a reverse sweep of the Berends-Giele
 * recursion: per helicity the currents are recomputed, the adjoints run
 * back through the colour sum, the closures, the recursion and the external
 * states, and one tangent per component through the per-event invariants
 * contracts them; me2_dev then holds that recursion's |M|^2 (equal to the
 * value path's on shell, to rounding).  For u ubar -> t tbar and u g -> t
 * tbar u one forward tangent per component.  Device pointers, caller-owned.
 * Does not synchronise. */
int mf_evaluate(struct mf_ctx *ctx, int process, const double *momenta_dev, long long n, double *me2_dev,
                double *dme2_dp_dev);

/* Helicity profile (the measurement behind the helicity filtering; the
 * paper's generated matrix element sums helicities in a loop, Sec. 2.2):
 * for n phase-space points momenta_dev [n][n_ext][4] (as mf_evaluate), out_dev
 * [n][2^n_ext] receives the averaged |M_h|^2 of every helicity configuration
 * h (bit i of h: helicity of external particle i, set = +1), so that each row
 * adds up to mf_evaluate's |M|^2.  The configurations that helicity
 * conservation on a massless fermion line forbids come out exactly zero; the
 * integrand and mf_evaluate skip them (e+ e- -> mu+ mu-: 12 of 16, u ubar ->
 * t tbar: 8 of 16, u g -> t tbar u: 16 of 32).  For the gluon processes
 * the parity mirror h ^ (2^n_ext - 1) has the same value (the integrand
 * evaluates one of each pair and doubles it).  In the context's precision;
 * device pointers, caller-owned; n = 0 is a no-op.  Does not synchronise. */
int mf_helicity_profile(struct mf_ctx *ctx, int process, const double *momenta_dev, long long n, double *out_dev);

/* Batched channels: several partonic subprocesses of one hadronic process
 * (p p -> t tbar + jets), each integrated on its own VEGAS grid, the sum
 * being the hadronic cross section.  The paper integrates one process at a
 * time (Sec. 2.1, the integrate(process, ...) call); batching them has no
 * counterpart there.  n_ch (1..8) channels, processes[i] one of the top-pair
 * processes (MF_GG_TT, MF_GG_TTG, MF_GG_TTGG, MF_UU_TT, MF_UG_TTU; a process
 * may repeat), n_events[i] >= 2 events per iteration.  Channel i draws its
 * random numbers with Philox channel id cfg.channel + i.
 * Every iteration hands out (channel, tile) work items, most expensive
 * channel first, to persistent CTAs through a device counter; each tile
 * writes its own row of partial sums and a channel's rows are reduced in
 * tile order, so the result does not depend on which CTA ran which tile.
 * Schedule (mf_set_batch_schedule, mf_autotune_batch): 0 = one persistent
 * launch for all channels; 1 = the g g -> t tbar g and t tbar g g channels
 * in the persistent launch at high priority and the cheaper channels as
 * their own integrand kernels at low priority, which fill the SMs as the
 * expensive work runs out; 2 = every channel as
 * its own integrand kernel, the g g -> t tbar g(g) ones at high priority (in
 * mode 2 these run a single-process pass's kernel, not persistent tiles);
 * 3 = the kernels of mode 2 one after another on the iteration's stream,
 * each filling the GPU.  In modes 1 and 2 every channel that runs as its own
 * kernel has its own stream, forked from the iteration's start and joined
 * before its reductions, so that the channels overlap on the GPU.  All
 * iterations
 * (launches, reductions, refinements) are captured once as a CUDA graph on a
 * private stream and replayed while the channel list, sizes, sqrt_s, n_iter,
 * couplings and schedule stay the same.  The schedule changes how sums are
 * grouped (results agree to rounding), the CTA count and timing do not.
 * cuts (host, nullable): as mf_integrate.  want_grads != 0: after the
 * iterations one derivative pass per channel at its final grid (Philox
 * iteration n_iter, as mf_batch_grad) fills the dsigma_* fields, the total's
 * being the channel sums (errors in quadrature).
 * Outputs (host): per_ch_host [n_ch] results as mf_integrate;
 * total_host: sigma = sum of the channels' sigma, error = their errors in
 * quadrature, chi2_dof = 0, counts summed; grids_host (nullable)
 * [n_ch][18][n_bins+1] final grids (rows past the channel's dimension are not
 * written).  MF_MIXED contexts only (MF_ERR_UNSUPPORTED otherwise).
 * Orders itself after work already queued on the context's stream and
 * synchronises before returning. */
int mf_integrate_batch(struct mf_ctx *ctx, int n_ch, const int *processes, const long long *n_events, double sqrt_s,
                       const mf_cuts *cuts, int n_iter, int want_grads, struct mf_result *per_ch_host,
                       struct mf_result *total_host, double *grids_host);

/* One pass of a batch of channels at caller grids, with optional per-event
 * outputs: the inspection call of mf_integrate_batch, as mf_vegas_pass is of
 * mf_integrate (no counterpart in the paper).  Runs the kernels of the
 * current batch schedule (mf_set_batch_schedule; the persistent kernel in
 * modes 0 and 1) once, without refinement, on events [0, n_events[i]) of
 * Philox iteration `iteration` and channel cfg.channel + i, at the
 * configuration's cuts.  grids_dev (device) [n_ch][18][n_bins+1]: each
 * channel's grid in its first dim rows; sums_dev (device)
 * [n_ch][2 + 18 n_bins]: each channel's pass sums as mf_vegas_pass (first
 * 2 + dim n_bins entries written).  ev_host (host, nullable) [n_ch]: per
 * channel the per-event device arrays of mf_vegas_pass (NULL members
 * skipped), written by the same kernels that run without them.
 * Other arguments and errors as mf_integrate_batch.  Orders itself after
 * work already queued on the context's stream; synchronises. */
int mf_batch_pass(struct mf_ctx *ctx, int n_ch, const int *processes, const long long *n_events, double sqrt_s,
                  const double *grids_dev, unsigned int iteration, double *sums_dev, const mf_event_arrays *ev_host);

/* d sigma_total / d m_t of a batch: one derivative pass per channel (as
 * mf_vegas_pass_grad, mixed precision) at the final grids left by the last
 * mf_integrate_batch call, which must have had the same channel list
 * (MF_ERR_ARG otherwise).  Channel i uses Philox channel cfg.channel + i and
 * iteration `iteration` (take one not used in training for an independent
 * estimate), events [0, n_events[i]), cuts as mf_integrate (use the same as
 * the integration).  out_host [n_ch + 1][4]: per channel,
 * then the sum over channels: sigma_hat, d sigma_hat/d m_t, its Monte Carlo
 * error (the channels' errors in quadrature for the sum), d sigma_hat/d
 * alpha_s.  Synchronises. */
int mf_batch_grad(struct mf_ctx *ctx, int n_ch, const int *processes, const long long *n_events, double sqrt_s,
                  const mf_cuts *cuts, unsigned int iteration, double *out_host);

/* Sets the mf_integrate_batch schedule explicitly (no counterpart in the
 * paper): mode 0/1/2/3 (one launch / split / per-channel kernels / the same
 * in turn, see mf_integrate_batch), sched 0/1 (helicity barrier off/on in the
 * g g -> t tbar g(g) matrix elements; in modes 2 and 3 also 2, the integrand
 * schedule with the tensor-core colour sum, 3, the warp-per-event
 * schedule, and 4, the helicity-recycled recursion, as mf_set_schedule),
 * tile_heavy and tile_light in [32, 2^26] events per work item for the
 * g g -> t tbar g(g) channels and for the others (in modes 1 and 2 the cheaper
 * channels' kernels get one CTA per tile_light events; in modes 2 and 3 the
 * g g -> t tbar g(g) kernels at most one CTA per tile_heavy events, up to as
 * many as fit), ctas_per_sm in
 * [0, 16] (0 = as many as fit; values above that are clamped), hsplit 1 or 2
 * (helicity split of the g g -> t tbar g(g) channels as mf_set_helicity_split;
 * 2 needs sched 1; modes 0 and 1 only).  MF_ERR_ARG outside these ranges.  Defaults: 0, 1, 4096,
 * 4096, 0, 1. */
int mf_set_batch_schedule(struct mf_ctx *ctx, int mode, int sched, long long tile_heavy, long long tile_light,
                          int ctas_per_sm, int hsplit);

/* Launch-schedule autotuner for mf_integrate_batch (no counterpart in the
 * paper).  Times one iteration of the given channels and sizes at uniform
 * grids for every mode {0, 1} x (helicity barrier, helicity split) {(0, 1),
 * (1, 1), (1, 2)} x tile_heavy {1024, 2048, 4096} x tile_light {2048, 4096},
 * mode 2 x sched {1, 2, 3, 4} x tile_heavy {512, 4096} x tile_light
 * {256, 2048, 4096}, and mode 3 x sched 4 x tile_heavy {512, 4096} x
 * tile_light {256, 2048} (CTAs per SM as fit; 64 candidates; each run once
 * untimed first, so that no candidate pays for its kernels' first launch)
 * and keeps the fastest for later
 * mf_integrate_batch calls on this context.  choice_host [6] (nullable)
 * receives (mode, sched, tile_heavy, tile_light, ctas_per_sm, hsplit), the
 * arguments of mf_set_batch_schedule.  Arguments as mf_integrate_batch; the cuts are the
 * configuration's.  Synchronises. */
int mf_autotune_batch(struct mf_ctx *ctx, int n_ch, const int *processes, const long long *n_events, double sqrt_s,
                      int *choice_host);

/* FMA throughput of the current device (no counterpart in the paper): the ALU
 * peak that the matrix-element kernels, bound by the FMA pipes, are measured
 * against.  precision MF_MIXED measures FP32, MF_FP64 FP64: 8 CTAs of 256
 * threads per SM, each thread running 8 independent multiply-add chains,
 * timed with CUDA events on stream (cudaStream_t or NULL), best of 3 launches
 * of about 8 ms after one warm-up.  *tflops_host (host, caller-owned): the
 * rate in TFLOP/s (an FMA counts 2).  The result depends on the SM clock at
 * the time of the call.  Needs no context; synchronises the stream.
 * MF_ERR_ARG for a null pointer or another precision. */
int mf_measure_fma_peak(int precision, void *stream, double *tflops_host);

/* Self-test of the double-float arithmetic (a value as the unevaluated sum of
 * two floats, about 48 bits) in which the mixed-precision path computes its
 * kinematics (Sec. 2.1: phase space, parton map, PDFs; no counterpart in the
 * paper, whose kinematics run in FP64).  y_dev[i] = f(x_dev[i]) for
 * i < n, the argument rounded to the nearest double-float and the result
 * converted to double; f one of MF_DF_EXP (e^x, |x| < 87), MF_DF_LOG (ln x,
 * x > 0), MF_DF_SQRT, MF_DF_SINPI (sin(pi x)), MF_DF_COSPI (cos(pi x)),
 * MF_DF_RECIP (1/x), MF_DF_SQUARE (x x).  x_dev, y_dev: device arrays of n
 * doubles, caller-owned.  Runs on stream (cudaStream_t or NULL) and
 * synchronises it.  Needs no context.  MF_ERR_ARG for another f, n < 0 or a
 * null array with n > 0; MF_ERR_CUDA on a launch failure. */
enum { MF_DF_EXP = 0, MF_DF_LOG = 1, MF_DF_SQRT = 2, MF_DF_SINPI = 3, MF_DF_COSPI = 4, MF_DF_RECIP = 5,
       MF_DF_SQUARE = 6 };
int mf_selftest_df(int fn, const double *x_dev, long long n, double *y_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif

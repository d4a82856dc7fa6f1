// C ABI of the library (declared in include/madflow_gb300.h).
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mf_ctx.h"

using namespace mf;



namespace mf {
// ------------------------------------------------------------------ end of a pass

// VEGAS grid refinement of one dimension from its histogram h of (f J)^2
// (Lepage 1978): neighbour smoothing, normalisation, damping
// ((r-1)/ln r)^alpha, then edges moved so that every new bin holds the same
// share of the damped weights.  A dimension with an empty histogram keeps
// its grid.
__device__ void refine_dim(const double* h, double* e, int nb, double alpha)
{
    double tot = 0.0;
    for (int i = 0; i < nb; ++i) tot += h[i];
    if (!(tot > 0.0)) return;
    double s[MAX_BINS], w[MAX_BINS], ne[MAX_BINS + 1];
    s[0] = (7.0 * h[0] + h[1]) / 8.0;
    for (int i = 1; i < nb - 1; ++i) s[i] = (h[i - 1] + 6.0 * h[i] + h[i + 1]) / 8.0;
    s[nb - 1] = (h[nb - 2] + 7.0 * h[nb - 1]) / 8.0;
    double sum = 0.0;
    for (int i = 0; i < nb; ++i) sum += s[i];
    double wsum = 0.0;
    for (int i = 0; i < nb; ++i) {
        const double r = s[i] / sum;
        w[i] = (r > 0.0 && r < 1.0) ? pow((r - 1.0) / log(r), alpha) : (r >= 1.0 ? 1.0 : 0.0);
        wsum += w[i];
    }
    const double delta = wsum / (double)nb;
    ne[0] = 0.0; ne[nb] = 1.0;
    double acc = 0.0;
    int j = 0;
    for (int k = 1; k < nb; ++k) {
        const double target = (double)k * delta;
        while (j < nb - 1 && acc + w[j] < target) { acc += w[j]; ++j; }
        double frac = w[j] > 0.0 ? (target - acc) / w[j] : 0.0;
        frac = frac > 1.0 ? 1.0 : frac;
        ne[k] = e[j] + frac * (e[j + 1] - e[j]);
    }
    for (int k = 0; k <= nb; ++k) e[k] = ne[k];
}

// Sums the per-CTA partials in CTA order, stores (I_k, var_k) for the
// iteration and, when asked, refines the grid.  One CTA; column c of the
// partials is summed by thread c, dimension d is refined by thread d.
__global__ void finish_pass_kernel(const double* partials, int nblk, int D, int nb, long long n, double alpha,
                                   int refine, double* grid, double* iter_stats, double* sums_out)
{
    extern __shared__ double sh[];     // [2 + D nb] sums
    const int ncol = 2 + D * nb;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * ncol + c];
        sh[c] = s;
        if (sums_out) sums_out[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0 && iter_stats) {
        const double I = sh[0], I2 = sh[1];
        iter_stats[0] = I;
        iter_stats[1] = ((double)n * I2 - I * I) / (double)(n - 1);
    }
    if (refine && (int)threadIdx.x < D) refine_dim(sh + 2 + threadIdx.x * nb, grid + threadIdx.x * (nb + 1), nb, alpha);
}

// Self-test of the bounded device waits: every thread waits on an mbarrier
// phase that nothing completes, with the given iteration limit, and the
// expiry raises the context's error flag (as in the tensor-core colour sum).
__global__ void wait_selftest_kernel(unsigned* err, unsigned limit)
{
    __shared__ unsigned long long mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    if (!mbar_wait(&mbar, 0, limit)) atomicExch(err, 1u);
}

// Observable of one pass: bin j of the per-CTA rows summed in CTA order by thread j,
// stored as (I_j, var_j) with the integral's variance estimate (n sum (w/N)^2 - I^2)/(n - 1)
__global__ void obs_reduce_kernel(const double* rows, int nblk, int nbins2, long long n, double* out)
{
    for (int j = threadIdx.x; j < nbins2; j += blockDim.x) {
        double I = 0.0, I2 = 0.0;
        for (int b = 0; b < nblk; ++b) {
            I += rows[(size_t)b * 2 * nbins2 + 2 * j];
            I2 += rows[(size_t)b * 2 * nbins2 + 2 * j + 1];
        }
        out[2 * j] = I;
        out[2 * j + 1] = ((double)n * I2 - I * I) / (double)(n - 1);
    }
}

// refinement from already reduced pass sums [2 + D nb]
__global__ void refine_kernel(const double* sums, int D, int nb, double alpha, double* grid)
{
    if ((int)threadIdx.x < D) refine_dim(sums + 2 + threadIdx.x * nb, grid + threadIdx.x * (nb + 1), nb, alpha);
}

}  // namespace mf

namespace {

constexpr int MAX_ITER = 1000;
constexpr double PI = 3.14159265358979323846;

const ProcOps* proc_ops(int p)
{
    switch (p) {
    case MF_EE_MUMU: return ops_ee_mumu();
    case MF_GG_TT: return ops_gg_tt();
    case MF_GG_TTG: return ops_gg_ttg();
    case MF_GG_TTGG: return ops_gg_ttgg();
    case MF_UU_TT: return ops_uu_tt();
    case MF_UG_TTU: return ops_ug_ttu();
    case MF_GG_TTGGG: return ops_gg_ttggg();
    default: return nullptr;
    }
}

const GradOpsTable* grad_ops(int p)
{
    switch (p) {
    case MF_GG_TT: return grad_gg_tt();
    case MF_GG_TTG: return grad_gg_ttg();
    case MF_GG_TTGG: return grad_gg_ttgg();
    case MF_UU_TT: return grad_uu_tt();
    case MF_UG_TTU: return grad_ug_ttu();
    case MF_GG_TTGGG: return grad_gg_ttggg();
    default: return nullptr;
    }
}

int fail(mf_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

#define MF_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, MF_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// fills the process-independent and process-dependent kernel parameters
int make_params(mf_ctx* c, int process, const ProcOps* ops, double sqrt_s, KParams& kp, const mf_cuts* cuts = nullptr)
{
    const mf_config& g = c->cfg;
    const int need_flav = process == MF_UU_TT ? 3 : (process == MF_UG_TTU ? 2 : 1);
    if (process != MF_EE_MUMU && c->n_flav < need_flav)
        return fail(c, MF_ERR_ARG, "the PDF grid lacks a flavour this process needs");
    std::memset(&kp, 0, sizeof(kp));
    kp.sqrt_s = sqrt_s;
    kp.S = sqrt_s * sqrt_s;
    kp.mt = g.mt;
    kp.gs = std::sqrt(4.0 * PI * g.alpha_s);
    const int nf = ops->NEXT - 2;
    // massless n-body volume without its shat^(n-2): (2 pi)^(4-3n) (pi/2)^(n-1) / ((n-1)! (n-2)!)
    kp.vol_const = std::pow(2.0 * PI, 4.0 - 3.0 * nf) * std::pow(PI / 2.0, nf - 1) / (factorial(nf - 1) * factorial(nf - 2));
    if (process != MF_EE_MUMU) {
        const double tau0 = 4.0 * g.mt * g.mt / kp.S;
        if (!(tau0 > 0.0 && tau0 < 1.0)) return fail(c, MF_ERR_ARG, "sqrt_s below the t tbar threshold");
        kp.ln_tau0 = std::log(tau0);
    }
    // fiducial cuts of this call, else those of the configuration
    const double pt_min = cuts ? cuts->pt_min : g.pt_min, eta_max = cuts ? cuts->eta_max : g.eta_max;
    const double dr_min = cuts ? cuts->dr_min : g.dr_min;
    kp.pt_min2 = pt_min > 0.0 ? pt_min * pt_min : 0.0;
    kp.sinh_eta = eta_max > 0.0 && std::isfinite(eta_max) ? std::sinh(eta_max) : 0.0;
    kp.dr_min2 = dr_min > 0.0 ? dr_min * dr_min : 0.0;
    {
        const double a = 1.0 / g.alpha_em_inv, mz2 = g.mz * g.mz;
        const double mw2 = 0.5 * mz2 + std::sqrt(0.25 * mz2 * mz2 - PI * a * mz2 / (std::sqrt(2.0) * g.gf));
        kp.ew.sw2 = 1.0 - mw2 / mz2;
        kp.ew.cw2 = 1.0 - kp.ew.sw2;
        kp.ew.e2 = 4.0 * PI * a;
        kp.ew.mz = g.mz;
        kp.ew.wz = g.wz;
    }
    kp.key = make_uint2((uint32_t)g.seed, (uint32_t)(g.seed >> 32));
    kp.channel = g.channel;
    kp.nb = g.n_bins;
    kp.pdfg.nx = c->nx;
    kp.pdfg.nq = c->nq;
    kp.pdfg.lx0 = std::log(c->x_min);
    kp.pdfg.hx = (0.0 - kp.pdfg.lx0) / (double)(c->nx - 1);
    kp.pdfg.lq0 = std::log(c->q2_min);
    kp.pdfg.lq1 = std::log(c->q2_max);
    kp.pdfg.hq = (kp.pdfg.lq1 - kp.pdfg.lq0) / (double)(c->nq - 1);
    kp.pdfg.ihx = 1.0 / kp.pdfg.hx;
    kp.pdfg.ihq = 1.0 / kp.pdfg.hq;
    kp.pdf = c->d_pdf;
    kp.pdf_df = c->d_pdf_df;
    kp.ln_muf2_fixed = std::log(g.mt * g.mt);
    fill_kin_df(kp.kd, kp.S, kp.ln_tau0, kp.mt, kp.gs, kp.vol_const, kp.ln_muf2_fixed, kp.pdfg);
    kp.partials = c->d_partials;
    kp.counters = c->d_counters;
    kp.dev_err = c->d_err;
    kp.kin = c->d_kin;
    kp.kin_bins = c->d_kin_bins;
    kp.kin_ctas = c->kin_ctas;
    kp.inv_rec = c->d_inv;
    kp.inv_ctas = c->inv_ctas;
    // sampling as many configurations as the sum has is the sum itself
    if (c->hel_samples > 0 && c->hel_samples < ops->hel_sample_max) {
        kp.hel_samples = c->hel_samples;
        kp.hel_stream = c->hel_stream;
    }
    return MF_OK;
}

// reads and clears the device error flag (the stream must be synchronised)
bool take_device_error(mf_ctx* c)
{
    unsigned h = 0;
    if (cudaMemcpy(&h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
    if (h) cudaMemset(c->d_err, 0, sizeof(unsigned));
    return h != 0;
}

int pick_blocks(mf_ctx* c, const ProcOps* ops, size_t sm, int prec, int* nblk)
{
    int per_sm = 0;
    MF_CUDA(c, ops->occupancy(prec, sm, &per_sm));
    if (per_sm < 1) return fail(c, MF_ERR_CUDA, "integrand kernel does not fit on an SM");
    if (ops->sched_ctas) {
        const int k = ops->sched_ctas(prec, c->sched, c->hsplit);
        if (k > 0) per_sm = k;
    }
    int n = per_sm * c->n_sm;
    if (n > c->max_blocks) n = c->max_blocks;
    *nblk = n;
    return MF_OK;
}

}  // namespace

int mf_fail(mf_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }
int mf_make_params(mf_ctx* c, int process, const ProcOps* ops, double sqrt_s, KParams& kp, const mf_cuts* cuts)
{
    return make_params(c, process, ops, sqrt_s, kp, cuts);
}
const ProcOps* mf_proc_ops(int process) { return proc_ops(process); }
const GradOpsTable* mf_grad_ops(int process) { return grad_ops(process); }

extern "C" {

int mf_default_config(mf_config* cfg)
{
    if (!cfg) return MF_ERR_ARG;
    cfg->mt = 173.0;
    cfg->alpha_s = 0.118;
    cfg->mz = 91.188;
    cfg->wz = 2.441404;
    cfg->alpha_em_inv = 132.507;
    cfg->gf = 1.16639e-5;
    cfg->pt_min = 30.0;
    cfg->eta_max = 2.5;
    cfg->dr_min = 0.4;
    cfg->seed = 0;
    cfg->channel = 0;
    cfg->n_bins = 50;
    cfg->alpha = 1.5;
    cfg->precision = MF_MIXED;
    return MF_OK;
}

int mf_process_info(int process, int* n_ext, int* dim)
{
    const ProcOps* o = proc_ops(process);
    if (!o) return MF_ERR_ARG;
    if (n_ext) *n_ext = o->NEXT;
    if (dim) *dim = o->D;
    return MF_OK;
}

int mf_create(mf_ctx** out, const mf_config* cfg, const double* pdf_grid_host, int n_flav, int nx, int nq,
              double x_min, double q2_min, double q2_max, void* stream)
{
    if (!out || !cfg || !pdf_grid_host) return MF_ERR_ARG;
    *out = nullptr;
    if (n_flav < 1 || n_flav > 3 || nx < 4 || nq < 4 || nx * nq > 8192) return MF_ERR_ARG;
    if (!(x_min > 0.0 && x_min < 1.0 && q2_min > 0.0 && q2_max > q2_min)) return MF_ERR_ARG;
    if (cfg->n_bins < 2 || cfg->n_bins > MAX_BINS || cfg->channel >= (1u << 24)) return MF_ERR_ARG;
    if (cfg->precision != MF_FP64 && cfg->precision != MF_MIXED) return MF_ERR_ARG;
    mf_ctx* c = new (std::nothrow) mf_ctx;
    if (!c) return MF_ERR_ARG;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)stream;
    c->n_flav = n_flav; c->nx = nx; c->nq = nq;
    c->x_min = x_min; c->q2_min = q2_min; c->q2_max = q2_max;
    auto bail = [&](int code) { mf_destroy(c); return code; };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(MF_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) return bail(MF_ERR_CUDA);
    c->max_blocks = c->n_sm * 32;
    const size_t npdf = (size_t)n_flav * nx * nq;
    const size_t ncol = 2 + (size_t)MAX_DIM * MAX_BINS;
    if (cudaMalloc(&c->d_pdf, npdf * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_pdf_df, npdf * sizeof(Df)) != cudaSuccess ||
        cudaMalloc(&c->d_grid, (size_t)MAX_DIM * (MAX_BINS + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_partials, (size_t)c->max_blocks * ncol * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_iter, (size_t)MAX_ITER * 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_sums, ncol * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_counters, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(unsigned)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(unsigned)) != cudaSuccess)
        return bail(MF_ERR_CUDA);
    // global kinematics store of the heavy integrand: up to 4 CTAs per SM of 256 queued events
    c->kin_ctas = 4 * c->n_sm;
    if (cudaMalloc(&c->d_kin, (size_t)c->kin_ctas * (KIN_NEXT_MAX * 4 + 1) * KIN_CAP_UNIT * sizeof(double)) !=
            cudaSuccess ||
        cudaMalloc(&c->d_kin_bins, (size_t)c->kin_ctas * MAX_DIM * KIN_CAP_UNIT) != cudaSuccess)
        return bail(MF_ERR_CUDA);
    // records of the warp-per-event schedule: one CTA per SM of LH_TPB queued events
    c->inv_ctas = c->n_sm;
    if (cudaMalloc(&c->d_inv, (size_t)c->inv_ctas * LH_INV_WORDS_MAX * LH_TPB * sizeof(float)) != cudaSuccess)
        return bail(MF_ERR_CUDA);
    if (cudaMemcpy(c->d_pdf, pdf_grid_host, npdf * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(MF_ERR_CUDA);
    {
        const std::vector<Df> pdf_df = split_df(pdf_grid_host, npdf);
        if (cudaMemcpy(c->d_pdf_df, pdf_df.data(), npdf * sizeof(Df), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(MF_ERR_CUDA);
    }
    for (int p : { MF_EE_MUMU, MF_GG_TT, MF_GG_TTG, MF_GG_TTGG, MF_UU_TT, MF_UG_TTU, MF_GG_TTGGG }) {
        const ProcOps* o = proc_ops(p);
        if (o->prepare(o->smem(1, MAX_BINS, nx * nq, true), o->smem(0, MAX_BINS, nx * nq, true)) != cudaSuccess)
            return bail(MF_ERR_CUDA);
    }
    *out = c;
    return MF_OK;
}

void mf_destroy(mf_ctx* c)
{
    if (!c) return;
    if (c->cap_stream) cudaStreamSynchronize(c->cap_stream);
    cudaFree(c->d_pdf);
    cudaFree(c->d_pdf_df);
    cudaFree(c->d_grid);
    cudaFree(c->d_partials);
    cudaFree(c->d_iter);
    cudaFree(c->d_sums);
    cudaFree(c->d_counters);
    cudaFree(c->d_err);
    cudaFree(c->d_kin);
    cudaFree(c->d_kin_bins);
    cudaFree(c->d_inv);
    cudaFree(c->d_obs_partials);
    cudaFree(c->d_obs_iter);
    cudaFree(c->d_kps);
    cudaFree(c->d_tiles);
    cudaFree(c->d_bgrids);
    cudaFree(c->d_biter);
    cudaFree(c->d_bsums);
    cudaFree(c->d_bcount);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->int_stream) cudaStreamSynchronize(c->int_stream);
    for (auto& kg : c->int_graphs) cudaGraphExecDestroy(kg.second);
    if (c->int_ev) cudaEventDestroy(c->int_ev);
    if (c->int_stream) cudaStreamDestroy(c->int_stream);
    if (c->ev_user) cudaEventDestroy(c->ev_user);
    if (c->ev_cap) cudaEventDestroy(c->ev_cap);
    for (int k = 0; k < mf::MAX_CH; ++k) {
        if (c->ev_side[k]) cudaEventDestroy(c->ev_side[k]);
        if (c->cap_side[k]) cudaStreamDestroy(c->cap_side[k]);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char* mf_last_error(const mf_ctx* c) { return c ? c->err.c_str() : "null context"; }

int mf_selftest_wait(mf_ctx* c, unsigned int iterations)
{
    if (!c || iterations < 1 || iterations > (1u << 20)) return MF_ERR_ARG;
    wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->d_err, iterations);
    MF_CUDA(c, cudaGetLastError());
    return mf_device_status(c);
}

int mf_device_status(mf_ctx* c)
{
    if (!c) return MF_ERR_ARG;
    MF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (take_device_error(c)) return fail(c, MF_ERR_TIMEOUT, "a bounded device wait ran out");
    return MF_OK;
}

int mf_set_precision(mf_ctx* c, int precision)
{
    if (!c || (precision != MF_FP64 && precision != MF_MIXED)) return MF_ERR_ARG;
    c->cfg.precision = precision;
    return MF_OK;
}

int mf_set_schedule(mf_ctx* c, int sched)
{
    if (!c || sched < 0 || sched > 4) return MF_ERR_ARG;
    c->sched = sched;
    return MF_OK;
}

int mf_set_observable(mf_ctx* c, const mf_obs* spec)
{
    if (!c) return MF_ERR_ARG;
    c->obs_iters = 0;
    if (!spec || spec->n_bins == 0) {
        c->obs_n = 0;
        return MF_OK;
    }
    if (spec->n_bins < 1 || spec->n_bins > MAX_OBS_BINS || !std::isfinite(spec->lo) || !std::isfinite(spec->hi) ||
        !(spec->hi > spec->lo))
        return fail(c, MF_ERR_ARG, "mf_set_observable: bad histogram");
    if (!c->d_obs_partials) {
        MF_CUDA(c, cudaMalloc(&c->d_obs_partials, sizeof(double) * (size_t)c->max_blocks * 2 * (MAX_OBS_BINS + 2)));
        MF_CUDA(c, cudaMalloc(&c->d_obs_iter, sizeof(double) * (size_t)MAX_ITER * 2 * (MAX_OBS_BINS + 2)));
    }
    c->obs_n = spec->n_bins;
    c->obs_lo = spec->lo;
    c->obs_hi = spec->hi;
    c->obs_inv_w = (double)spec->n_bins / (spec->hi - spec->lo);
    return MF_OK;
}

int mf_get_observable(mf_ctx* c, double* hist_host, double* err_host, double* iter_host)
{
    if (!c) return MF_ERR_ARG;
    if (c->obs_n == 0 || c->obs_iters == 0)
        return fail(c, MF_ERR_ARG, "mf_get_observable: no histogram since mf_set_observable");
    const size_t n2 = (size_t)c->obs_n + 2;
    if (hist_host) std::memcpy(hist_host, c->obs_hist.data(), n2 * sizeof(double));
    if (err_host) std::memcpy(err_host, c->obs_err.data(), n2 * sizeof(double));
    if (iter_host) std::memcpy(iter_host, c->obs_iter_host.data(), (size_t)c->obs_iters * 2 * n2 * sizeof(double));
    return MF_OK;
}

int mf_set_helicity_split(mf_ctx* c, int parts)
{
    if (!c || (parts != 1 && parts != 2)) return MF_ERR_ARG;
    c->hsplit = parts;
    return MF_OK;
}

int mf_set_helicity_sampling(mf_ctx* c, int n_samples, unsigned int stream)
{
    if (!c || n_samples < 0 || n_samples > 64 || (n_samples & (n_samples - 1))) return MF_ERR_ARG;
    c->hel_samples = n_samples;
    c->hel_stream = stream;
    return MF_OK;
}

int mf_set_pdf(mf_ctx* c, const double* pdf_grid_host)
{
    if (!c || !pdf_grid_host) return MF_ERR_ARG;
    const size_t npdf = (size_t)c->n_flav * c->nx * c->nq;
    MF_CUDA(c, cudaMemcpyAsync(c->d_pdf, pdf_grid_host, npdf * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // the double-float copy from pageable memory: the call returns once the host buffer is staged
    const std::vector<Df> pdf_df = split_df(pdf_grid_host, npdf);
    MF_CUDA(c, cudaMemcpyAsync(c->d_pdf_df, pdf_df.data(), npdf * sizeof(Df), cudaMemcpyHostToDevice, c->stream));
    return MF_OK;
}

int mf_vegas_pass(mf_ctx* c, int process, double sqrt_s, const double* grid_dev, long long n_events,
                  long long ev_offset, unsigned int iteration, const unsigned char* mask_in_dev, double* sums_dev,
                  const mf_event_arrays* ev)
{
    if (!c) return MF_ERR_ARG;
    const ProcOps* ops = proc_ops(process);
    if (!ops) return fail(c, MF_ERR_ARG, "unknown process");
    if (!grid_dev || !sums_dev || n_events < 1 || ev_offset < 0 || !(sqrt_s > 0.0))
        return fail(c, MF_ERR_ARG, "mf_vegas_pass: bad argument");
    KParams kp;
    int rc = make_params(c, process, ops, sqrt_s, kp);
    if (rc) return rc;
    kp.iteration = iteration;
    kp.n_events = n_events;
    kp.ev_offset = ev_offset;
    kp.inv_n = 1.0 / (double)n_events;
    kp.grid = grid_dev;
    kp.mask_in = mask_in_dev;
    const bool write = ev != nullptr;
    if (ev) {
        kp.ev_u = ev->u; kp.ev_x = ev->x; kp.ev_bins = ev->bins; kp.ev_w = ev->w;
        kp.ev_mask = ev->mask; kp.ev_me2 = ev->me2; kp.ev_p = ev->momenta;
        kp.ev_out = 1;
    }
    const size_t sm = ops->smem(c->cfg.precision, c->cfg.n_bins, c->nx * c->nq, false);
    int nblk = 0;
    rc = pick_blocks(c, ops, sm, c->cfg.precision, &nblk);
    if (rc) return rc;
    MF_CUDA(c, cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), c->stream));
    MF_CUDA(c, ops->integrand(c->cfg.precision, write, c->sched, c->hsplit, kp, nblk, sm, c->stream));
    const int ncol = 2 + ops->D * c->cfg.n_bins;
    finish_pass_kernel<<<1, 1024, ncol * sizeof(double), c->stream>>>(c->d_partials, nblk, ops->D, c->cfg.n_bins,
                                                                     n_events, c->cfg.alpha, 0, nullptr, nullptr,
                                                                     sums_dev);
    MF_CUDA(c, cudaGetLastError());
    return MF_OK;
}

int mf_vegas_refine(mf_ctx* c, int dim, int n_bins, double alpha, const double* sums_dev, double* grid_dev)
{
    if (!c) return MF_ERR_ARG;
    if (dim < 1 || dim > MAX_DIM || n_bins < 2 || n_bins > MAX_BINS || !sums_dev || !grid_dev || !(alpha >= 0.0))
        return fail(c, MF_ERR_ARG, "mf_vegas_refine: bad argument");
    refine_kernel<<<1, 32, 0, c->stream>>>(sums_dev, dim, n_bins, alpha, grid_dev);
    MF_CUDA(c, cudaGetLastError());
    return MF_OK;
}

}  // extern "C"

namespace {

// the launch parameters that a captured iteration graph bakes in
std::string integrate_key(const KParams& kp, int prec, int sched, int hsplit, int nblk, size_t sm, int n_iter,
                          unsigned first_it, int obs_n)
{
    KParams k = kp;
    k.iteration = 0;
    std::string key(reinterpret_cast<const char*>(&k), sizeof(k));
    const long long tail[8] = { prec, sched, hsplit, nblk, (long long)sm, n_iter, (long long)first_it, obs_n };
    key.append(reinterpret_cast<const char*>(tail), sizeof(tail));
    return key;
}

// n_iter VEGAS iterations (Philox iterations first_it, first_it + 1, ...) from the grid
// grid_in_host (nullable: uniform); see mf_integrate and mf_integrate_grid
int integrate_impl(mf_ctx* c, int process, double sqrt_s, const mf_cuts* cuts, long long n_events, int n_iter,
                   unsigned first_it, const double* grid_in_host, int want_grads, mf_result* out, double* iter_host,
                   double* grid_host)
{
    const ProcOps* ops = proc_ops(process);
    if (!ops) return fail(c, MF_ERR_ARG, "unknown process");
    if (!out || n_events < 2 || n_iter < 1 || n_iter > MAX_ITER || !(sqrt_s > 0.0))
        return fail(c, MF_ERR_ARG, "mf_integrate: bad argument");
    const GradOpsTable* gops = nullptr;
    if (want_grads) {
        gops = grad_ops(process);
        if (!gops || !gops->has_pass) return fail(c, MF_ERR_UNSUPPORTED, "no derivative pass for this process");
        if (c->cfg.precision == MF_FP64 && !gops->has_fp64)
            return fail(c, MF_ERR_UNSUPPORTED, "FP64 derivative of this process not built; use MF_MIXED");
    }
    KParams kp;
    int rc = make_params(c, process, ops, sqrt_s, kp, cuts);
    if (rc) return rc;
    const int D = ops->D, nb = c->cfg.n_bins;
    kp.n_events = n_events;
    kp.ev_offset = 0;
    kp.inv_n = 1.0 / (double)n_events;
    kp.grid = c->d_grid;
    const bool obs = c->obs_n > 0;
    const int nobs2 = c->obs_n + 2;
    if (obs) {
        kp.nobs = c->obs_n;
        kp.obs_lo = c->obs_lo;
        kp.obs_inv_w = c->obs_inv_w;
        kp.obs_partials = c->d_obs_partials;
    }
    const size_t sm = ops->smem(c->cfg.precision, nb, c->nx * c->nq, obs);
    int nblk = 0;
    rc = pick_blocks(c, ops, sm, c->cfg.precision, &nblk);
    if (rc) return rc;
    // private stream for capture and replay, ordered after the caller's stream
    if (!c->int_stream) {
        MF_CUDA(c, cudaStreamCreateWithFlags(&c->int_stream, cudaStreamNonBlocking));
        MF_CUDA(c, cudaEventCreateWithFlags(&c->int_ev, cudaEventDisableTiming));
    }
    cudaStream_t s = c->int_stream;
    MF_CUDA(c, cudaEventRecord(c->int_ev, c->stream));
    MF_CUDA(c, cudaStreamWaitEvent(s, c->int_ev, 0));
    std::vector<double> g0((size_t)D * (nb + 1));
    if (grid_in_host) {
        std::memcpy(g0.data(), grid_in_host, g0.size() * sizeof(double));
    } else {
        for (int d = 0; d < D; ++d)
            for (int i = 0; i <= nb; ++i) g0[(size_t)d * (nb + 1) + i] = (double)i / (double)nb;
    }
    MF_CUDA(c, cudaMemcpyAsync(c->d_grid, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    MF_CUDA(c, cudaMemsetAsync(c->d_counters, 0, 2 * sizeof(unsigned long long), s));
    const int ncol = 2 + D * nb;
    // the iterations: captured once, replayed while the parameters stay the same
    const std::string key = integrate_key(kp, c->cfg.precision, c->sched, c->hsplit, nblk, sm, n_iter, first_it,
                                          obs ? c->obs_n : 0);
    cudaGraphExec_t exec = nullptr;
    for (size_t i = 0; i < c->int_graphs.size(); ++i)
        if (c->int_graphs[i].first == key) {
            // a hit moves to the most recently used end
            auto kg = c->int_graphs[i];
            c->int_graphs.erase(c->int_graphs.begin() + (long)i);
            c->int_graphs.push_back(kg);
            exec = kg.second;
            break;
        }
    if (!exec) {
        if (c->int_graphs.size() >= mf_ctx::INT_GRAPHS) {
            cudaGraphExecDestroy(c->int_graphs.front().second);
            c->int_graphs.erase(c->int_graphs.begin());
        }
        cudaGraph_t g = nullptr;
        MF_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int erc = MF_OK;
        for (int it = 0; it < n_iter && erc == MF_OK; ++it) {
            kp.iteration = first_it + (uint32_t)it;
            if (ops->integrand(c->cfg.precision, false, c->sched, c->hsplit, kp, nblk, sm, s) != cudaSuccess) {
                erc = fail(c, MF_ERR_CUDA, "integrand launch");
                break;
            }
            finish_pass_kernel<<<1, 1024, ncol * sizeof(double), s>>>(c->d_partials, nblk, D, nb, n_events, c->cfg.alpha,
                                                                     it < n_iter - 1, c->d_grid, c->d_iter + 2 * it,
                                                                     nullptr);
            if (obs)
                obs_reduce_kernel<<<1, 128, 0, s>>>(c->d_obs_partials, nblk, nobs2, n_events,
                                                    c->d_obs_iter + (size_t)it * 2 * nobs2);
        }
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (erc) { if (g) cudaGraphDestroy(g); return erc; }
        if (ce != cudaSuccess) return fail(c, MF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiateWithFlags(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(c, MF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        c->int_graphs.emplace_back(key, exec);
    }
    MF_CUDA(c, cudaGraphLaunch(exec, s));
    if (want_grads) {
        // one derivative pass at the final grid on fresh random numbers (Philox iteration first_it + n_iter)
        KParams kg = kp;
        kg.iteration = first_it + (uint32_t)n_iter;
        kg.mask_in = nullptr;
        const long long want = (n_events + 127) / 128, cap = (long long)c->n_sm * gops->ctas_per_sm;
        const int gblk = (int)(want < cap ? want : cap);
        MF_CUDA(c, gops->grad(c->cfg.precision, kg, gblk, c->d_partials, gops->k_as, c->cfg.alpha_s, s));
        finish_pass_kernel<<<1, 32, 4 * sizeof(double), s>>>(c->d_partials, gblk, 1, 2, n_events, 0.0, 0, nullptr,
                                                             nullptr, c->d_sums);
        MF_CUDA(c, cudaGetLastError());
    }
    double gsum[4] = { 0.0, 0.0, 0.0, 0.0 };
    if (want_grads) MF_CUDA(c, cudaMemcpyAsync(gsum, c->d_sums, sizeof(gsum), cudaMemcpyDeviceToHost, s));
    std::vector<double> iters((size_t)2 * n_iter);
    unsigned long long cnt[2];
    MF_CUDA(c, cudaMemcpyAsync(iters.data(), c->d_iter, iters.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    MF_CUDA(c, cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    if (grid_host)
        MF_CUDA(c, cudaMemcpyAsync(grid_host, c->d_grid, (size_t)D * (nb + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (obs) {
        c->obs_iter_host.resize((size_t)n_iter * 2 * nobs2);
        MF_CUDA(c, cudaMemcpyAsync(c->obs_iter_host.data(), c->d_obs_iter, c->obs_iter_host.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
    }
    MF_CUDA(c, cudaStreamSynchronize(s));
    if (take_device_error(c)) return fail(c, MF_ERR_TIMEOUT, "a bounded device wait ran out");
    double sw = 0.0, swi = 0.0;
    for (int k = 0; k < n_iter; ++k) {
        const double wk = 1.0 / iters[2 * k + 1];
        sw += wk;
        swi += wk * iters[2 * k];
    }
    const double mean = swi / sw;
    double chi2 = 0.0;
    for (int k = 0; k < n_iter; ++k) chi2 += (iters[2 * k] - mean) * (iters[2 * k] - mean) / iters[2 * k + 1];
    out->sigma_pb = mean;
    out->error_pb = std::sqrt(1.0 / sw);
    if (obs) {
        // every bin combines its iterations with the integral's weights lambda_k = (1/var_k) / sum_j (1/var_j),
        // so that the bins add up to the combined cross section
        c->obs_hist.assign(nobs2, 0.0);
        c->obs_err.assign(nobs2, 0.0);
        for (int k = 0; k < n_iter; ++k) {
            const double lam = (1.0 / iters[2 * k + 1]) / sw;
            const double* r = c->obs_iter_host.data() + (size_t)k * 2 * nobs2;
            for (int j = 0; j < nobs2; ++j) {
                c->obs_hist[j] += lam * r[2 * j];
                c->obs_err[j] += lam * lam * r[2 * j + 1];
            }
        }
        for (int j = 0; j < nobs2; ++j) c->obs_err[j] = std::sqrt(c->obs_err[j] > 0.0 ? c->obs_err[j] : 0.0);
        c->obs_iters = n_iter;
    }
    out->chi2_dof = n_iter > 1 ? chi2 / (n_iter - 1) : 0.0;
    out->n_events_total = n_events * (long long)n_iter;
    out->n_pass = (long long)cnt[0];
    out->n_nan = (long long)cnt[1];
    out->n_iter = n_iter;
    out->dsigma_dmt = out->dsigma_dmt_error = out->dsigma_dalphas = 0.0;
    if (want_grads) {
        const double nd = (double)n_events, var = (nd * gsum[2] - gsum[1] * gsum[1]) / (nd - 1.0);
        out->dsigma_dmt = gsum[1];
        out->dsigma_dmt_error = std::sqrt(var > 0.0 ? var : 0.0);
        out->dsigma_dalphas = gsum[3];
    }
    if (iter_host) std::memcpy(iter_host, iters.data(), iters.size() * sizeof(double));
    if (cnt[1] > (unsigned long long)(n_events * (long long)n_iter) / 1000)
        return fail(c, MF_ERR_NUMERIC, "more than 0.1% of the event weights were not finite");
    return MF_OK;
}

}  // namespace

extern "C" {

int mf_integrate(mf_ctx* c, int process, double sqrt_s, const mf_cuts* cuts, long long n_events, int n_iter,
                 int want_grads, mf_result* out, double* iter_host, double* grid_host)
{
    if (!c) return MF_ERR_ARG;
    return integrate_impl(c, process, sqrt_s, cuts, n_events, n_iter, 0u, nullptr, want_grads, out, iter_host,
                          grid_host);
}

int mf_integrate_grid(mf_ctx* c, int process, double sqrt_s, const mf_cuts* cuts, long long n_events, int n_iter,
                      unsigned int first_iteration, const double* grid_in_host, int want_grads, mf_result* out,
                      double* iter_host, double* grid_host)
{
    if (!c) return MF_ERR_ARG;
    if (!grid_in_host) return fail(c, MF_ERR_ARG, "mf_integrate_grid: no starting grid");
    return integrate_impl(c, process, sqrt_s, cuts, n_events, n_iter, first_iteration, grid_in_host, want_grads,
                          out, iter_host, grid_host);
}

int mf_set_couplings(mf_ctx* c, double mt, double alpha_s)
{
    if (!c || !(mt > 0.0) || !(alpha_s > 0.0)) return MF_ERR_ARG;
    c->cfg.mt = mt;
    c->cfg.alpha_s = alpha_s;
    return MF_OK;
}

int mf_vegas_pass_grad(mf_ctx* c, int process, double sqrt_s, const double* grid_dev, long long n_events,
                       long long ev_offset, unsigned int iteration, const unsigned char* mask_in_dev, double* out_dev)
{
    if (!c) return MF_ERR_ARG;
    const ProcOps* ops = proc_ops(process);
    const GradOpsTable* g = grad_ops(process);
    if (!ops || !g || !g->has_pass) return fail(c, MF_ERR_UNSUPPORTED, "no derivative pass for this process");
    if (c->cfg.precision == MF_FP64 && !g->has_fp64)
        return fail(c, MF_ERR_UNSUPPORTED, "FP64 derivative of this process not built; use MF_MIXED");
    if (!grid_dev || !out_dev || n_events < 1 || ev_offset < 0 || !(sqrt_s > 0.0))
        return fail(c, MF_ERR_ARG, "mf_vegas_pass_grad: bad argument");
    KParams kp;
    int rc = make_params(c, process, ops, sqrt_s, kp);
    if (rc) return rc;
    kp.iteration = iteration;
    kp.n_events = n_events;
    kp.ev_offset = ev_offset;
    kp.inv_n = 1.0 / (double)n_events;
    kp.grid = grid_dev;
    kp.mask_in = mask_in_dev;
    long long want = (n_events + 127) / 128;
    const long long cap = (long long)c->n_sm * g->ctas_per_sm;
    const int nblk = (int)(want < cap ? want : cap);
    MF_CUDA(c, g->grad(c->cfg.precision, kp, nblk, c->d_partials, g->k_as, c->cfg.alpha_s, c->stream));
    finish_pass_kernel<<<1, 32, 4 * sizeof(double), c->stream>>>(c->d_partials, nblk, 1, 2, n_events, 0.0, 0, nullptr,
                                                                 nullptr, out_dev);
    MF_CUDA(c, cudaGetLastError());
    return MF_OK;
}

int mf_helicity_profile(mf_ctx* c, int process, const double* momenta_dev, long long n, double* out_dev)
{
    if (!c) return MF_ERR_ARG;
    const ProcOps* ops = proc_ops(process);
    if (!ops || !ops->profile) return fail(c, MF_ERR_ARG, "unknown process");
    if (n == 0) return MF_OK;
    if (!momenta_dev || !out_dev || n < 0) return fail(c, MF_ERR_ARG, "mf_helicity_profile: bad argument");
    KParams kp;
    int rc = make_params(c, process, ops, 1.0e4, kp);
    if (rc) return rc;
    const long long nb = (n + 63) / 64, cap = (long long)c->n_sm * 16;
    const int nblk = (int)(nb < cap ? nb : cap);
    MF_CUDA(c, ops->profile(c->cfg.precision, momenta_dev, n, out_dev, kp.mt, kp.gs, kp.ew, nblk, c->stream));
    return MF_OK;
}

int mf_evaluate(mf_ctx* c, int process, const double* momenta_dev, long long n, double* me2_dev, double* dme2_dp_dev)
{
    if (!c) return MF_ERR_ARG;
    const ProcOps* ops = proc_ops(process);
    if (!ops) return fail(c, MF_ERR_ARG, "unknown process");
    if (dme2_dp_dev) {
        // |M|^2 and its momentum derivatives in one kernel (forward mode, one tangent per component)
        const GradOpsTable* g = grad_ops(process);
        if (!g) return fail(c, MF_ERR_UNSUPPORTED, "no derivative for this process");
        if (c->cfg.precision == MF_FP64 && !g->has_fp64_evaluate)
            return fail(c, MF_ERR_UNSUPPORTED, "FP64 derivative of this process not built; use MF_MIXED");
        if (n == 0) return MF_OK;
        if (!momenta_dev || n < 0) return fail(c, MF_ERR_ARG, "mf_evaluate: bad argument");
        const double gs = std::sqrt(4.0 * PI * c->cfg.alpha_s);
        const long long nb = (n + 127) / 128, cap = (long long)c->n_sm * 8;
        const int nblk = (int)(nb < cap ? nb : cap);
        MF_CUDA(c, g->evaluate_grad(c->cfg.precision, momenta_dev, n, me2_dev, dme2_dp_dev, c->cfg.mt, gs, nblk,
                                    c->stream));
        return MF_OK;
    }
    if (n == 0) return MF_OK;
    if (!momenta_dev || !me2_dev || n < 0) return fail(c, MF_ERR_ARG, "mf_evaluate: bad argument");
    KParams kp;
    int rc = make_params(c, process, ops, 1.0e4, kp);
    if (rc) return rc;
    long long nb = (n + 127) / 128;
    const long long cap = (long long)c->n_sm * 16;
    const int nblk = (int)(nb < cap ? nb : cap);
    MF_CUDA(c, ops->evaluate(c->cfg.precision, momenta_dev, n, me2_dev, kp.mt, kp.gs, kp.ew, nblk, c->stream));
    return MF_OK;
}

}  // extern "C"

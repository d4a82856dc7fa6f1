// Allocation-free VEGAS pass (declared in include/madflow_gb300.h as
// mf_vegas_pass_static).
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// framework which owns all device memory and forbids allocation in its
// callbacks, code on a path that must not synchronise the device (a
// cudaMalloc may), or a long-running service that pre-plans its memory and
// treats any allocation after start-up as a failure.  For them this entry
// point runs the same fused integrand kernel and the same end-of-pass
// reduction as mf_vegas_pass without an mf_ctx: the caller passes the PDF
// grid, the VEGAS grid and the output sums as device pointers, and the
// kernel's scratch (the per-CTA partial sums and two counters) lives in the
// fixed array below, which every GPU that loads this library holds until the
// process exits.  Nothing here allocates: no cudaMalloc, no cudaFree, no
// library routine that allocates.
#include <cuda_runtime.h>
#include <atomic>
#include <cmath>
#include <cstring>

#include "mf_dispatch.cuh"
#include "../../include/madflow_gb300.h"

namespace mf {
// defined with the other end-of-pass kernels in mf_capi.cu
__global__ void finish_pass_kernel(const double* partials, int nblk, int D, int nb, long long n, double alpha,
                                   int refine, double* grid, double* iter_stats, double* sums_out);
}

namespace {

using namespace mf;

// 4 MiB of scratch: two counters, then [blocks][2 + dim n_bins] partial sums.
constexpr size_t kScratchDoubles = 512 * 1024;
static __device__ __align__(256) double g_pass_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
// per-device state, filled by the first call on that device (host threads may race
// on the first call; every one of them stores the same address)
std::atomic<double*> g_scratch_ptr[kMaxDevices] = {};

const ProcOps* ops_for(int p)
{
    switch (p) {
    case MF_EE_MUMU: return ops_ee_mumu();
    case MF_GG_TT: return ops_gg_tt();
    case MF_GG_TTG: return ops_gg_ttg();
    case MF_GG_TTGG: return ops_gg_ttgg();
    case MF_UU_TT: return ops_uu_tt();
    case MF_UG_TTU: return ops_ug_ttu();
    default: return nullptr;
    }
}

double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// Device address of the scratch array on the current device.  In host code
// the symbol g_pass_scratch is only a host-side stand-in, so the address
// comes from cudaGetSymbolAddress, taken once per device with that device
// current.
int scratch_on_current_device(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MF_ERR_CUDA;
    double* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pass_scratch) != cudaSuccess || !p) return MF_ERR_CUDA;
        ptr = static_cast<double*>(p);
        g_scratch_ptr[dev].store(ptr, std::memory_order_release);
    }
    *out = ptr;
    return MF_OK;
}

}  // namespace

extern "C" int mf_vegas_pass_static(int process, const mf_config* cfg, double sqrt_s, const double* pdf_dev, int n_flav,
                                    int nx, int nq, double x_min, double q2_min, double q2_max, const double* grid_dev,
                                    long long n_events, long long ev_offset, unsigned int iteration, double* sums_dev,
                                    void* stream)
{
    const ProcOps* ops = ops_for(process);
    if (!ops) return MF_ERR_ARG;
    if (!cfg || !pdf_dev || !grid_dev || !sums_dev || n_events < 1 || ev_offset < 0 || !(sqrt_s > 0.0)) return MF_ERR_ARG;
    if (n_flav < 1 || n_flav > 3 || nx < 4 || nq < 4 || nx * nq > 8192) return MF_ERR_ARG;
    if (!(x_min > 0.0 && x_min < 1.0 && q2_min > 0.0 && q2_max > q2_min)) return MF_ERR_ARG;
    if (cfg->n_bins < 2 || cfg->n_bins > MAX_BINS || cfg->channel >= (1u << 24)) return MF_ERR_ARG;
    if (cfg->precision != MF_FP64 && cfg->precision != MF_MIXED) return MF_ERR_ARG;
    const int need_flav = process == MF_UU_TT ? 3 : (process == MF_UG_TTU ? 2 : 1);
    if (process != MF_EE_MUMU && n_flav < need_flav) return MF_ERR_ARG;
    const int D = ops->D, nb = cfg->n_bins;
    const size_t ncol = 2 + (size_t)D * nb;
    // the scratch must hold at least one CTA's partials beyond the counters
    if (2 + ncol > kScratchDoubles) return MF_ERR_ARG;

    double* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != MF_OK) return MF_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MF_ERR_CUDA;
    const size_t sm = ops->smem(cfg->precision, nb, nx * nq, false);
    // allow this process's kernels the largest shared-memory size any argument set can need,
    // the observable region included: the same sizes mf_create sets, so a call here never
    // lowers the limit that a context's passes with the observable histogram rely on
    if (ops->prepare(ops->smem(1, MAX_BINS, 8192, true), ops->smem(0, MAX_BINS, 8192, true)) != cudaSuccess)
        return MF_ERR_CUDA;
    int n_sm = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MF_ERR_CUDA;
    if (ops->occupancy(cfg->precision, sm, &per_sm) != cudaSuccess || per_sm < 1) return MF_ERR_CUDA;
    const long long cap = (long long)((kScratchDoubles - 2) / ncol);
    long long nblk = (long long)per_sm * n_sm;
    if (nblk > cap) nblk = cap;

    const double PI = 3.14159265358979323846;
    KParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.sqrt_s = sqrt_s;
    kp.S = sqrt_s * sqrt_s;
    kp.mt = cfg->mt;
    kp.gs = std::sqrt(4.0 * PI * cfg->alpha_s);
    const int nf = ops->NEXT - 2;
    kp.vol_const = std::pow(2.0 * PI, 4.0 - 3.0 * nf) * std::pow(PI / 2.0, nf - 1) / (factorial(nf - 1) * factorial(nf - 2));
    if (process != MF_EE_MUMU) {
        const double tau0 = 4.0 * cfg->mt * cfg->mt / kp.S;
        if (!(tau0 > 0.0 && tau0 < 1.0)) return MF_ERR_ARG;
        kp.ln_tau0 = std::log(tau0);
    }
    kp.pt_min2 = cfg->pt_min > 0.0 ? cfg->pt_min * cfg->pt_min : 0.0;
    // an infinite eta_max disables the cut, as in a context's passes
    kp.sinh_eta = cfg->eta_max > 0.0 && std::isfinite(cfg->eta_max) ? std::sinh(cfg->eta_max) : 0.0;
    kp.dr_min2 = cfg->dr_min > 0.0 ? cfg->dr_min * cfg->dr_min : 0.0;
    {
        const double a = 1.0 / cfg->alpha_em_inv, mz2 = cfg->mz * cfg->mz;
        const double mw2 = 0.5 * mz2 + std::sqrt(0.25 * mz2 * mz2 - PI * a * mz2 / (std::sqrt(2.0) * cfg->gf));
        kp.ew.sw2 = 1.0 - mw2 / mz2;
        kp.ew.cw2 = 1.0 - kp.ew.sw2;
        kp.ew.e2 = 4.0 * PI * a;
        kp.ew.mz = cfg->mz;
        kp.ew.wz = cfg->wz;
    }
    kp.key = make_uint2((uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32));
    kp.channel = cfg->channel;
    kp.iteration = iteration;
    kp.nb = nb;
    kp.n_events = n_events;
    kp.ev_offset = ev_offset;
    kp.inv_n = 1.0 / (double)n_events;
    kp.pdfg.nx = nx;
    kp.pdfg.nq = nq;
    kp.pdfg.lx0 = std::log(x_min);
    kp.pdfg.hx = (0.0 - kp.pdfg.lx0) / (double)(nx - 1);
    kp.pdfg.lq0 = std::log(q2_min);
    kp.pdfg.lq1 = std::log(q2_max);
    kp.pdfg.hq = (kp.pdfg.lq1 - kp.pdfg.lq0) / (double)(nq - 1);
    kp.pdfg.ihx = 1.0 / kp.pdfg.hx;
    kp.pdfg.ihq = 1.0 / kp.pdfg.hq;
    kp.pdf = pdf_dev;
    kp.pdf_df = nullptr;   // no copy without an allocation: the mixed kinematics convert each node
    kp.ln_muf2_fixed = std::log(cfg->mt * cfg->mt);
    fill_kin_df(kp.kd, kp.S, kp.ln_tau0, kp.mt, kp.gs, kp.vol_const, kp.ln_muf2_fixed, kp.pdfg);
    kp.grid = grid_dev;
    // layout of the shared scratch: [0..1] counters, then the partial sums
    kp.counters = reinterpret_cast<unsigned long long*>(scratch);
    kp.partials = scratch + 2;

    cudaStream_t s = (cudaStream_t)stream;
    // the counters start at zero on every call; the partials are fully overwritten by the kernel
    if (cudaMemsetAsync(scratch, 0, 2 * sizeof(double), s) != cudaSuccess) return MF_ERR_CUDA;
    // schedule 0: one event per thread with the FMA colour sum (the warp-per-event schedule
    // needs a per-CTA record region that only a context owns)
    if (ops->integrand(cfg->precision, false, 0, 1, kp, (int)nblk, sm, s) != cudaSuccess) return MF_ERR_CUDA;
    finish_pass_kernel<<<1, 1024, ncol * sizeof(double), s>>>(kp.partials, (int)nblk, D, nb, n_events, cfg->alpha, 0,
                                                              nullptr, nullptr, sums_dev);
    if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
    return MF_OK;
}

// Batched channels in one persistent launch, with the VEGAS iterations
// captured as a CUDA graph and the launch schedule picked by a small
// autotuner (declared in include/madflow_gb300.h: mf_integrate_batch,
// mf_autotune_batch).
//
// The work is a list of (channel, tile) pairs: tile t of channel c holds
// events [t T, (t+1) T) of that channel.  Persistent CTAs take tiles from a
// device counter (an atomic increment: no CTA ever waits for another), run
// the channel's own integrand on them with the channel's own VEGAS grid and
// Philox channel id, and write one set of partial sums per tile.  The
// end-of-pass reduction sums the tiles of each channel in tile order, so the
// result does not depend on which CTA ran which tile.
#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mf_batch.cuh"
#include "mf_ctx.h"
#include "generated/me_gg_tt.cuh"
#include "generated/me_gg_ttg.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/me_uu_tt.cuh"
#include "generated/me_ug_ttu.cuh"

namespace mf {
__global__ void finish_pass_kernel(const double* partials, int nblk, int D, int nb, long long n, double alpha,
                                   int refine, double* grid, double* iter_stats, double* sums_out);

constexpr int BATCH_TPB = 128;
using PGgTt = ProcTops<Me_gg_tt>;
using PGgTtg = ProcTops<Me_gg_ttg>;
using PGgTtgg = ProcTops<Me_gg_ttgg>;
using PUuTt = ProcTops<Me_uu_tt, 1, 2>;
using PUgTtu = ProcTops<Me_ug_ttu, 1, 0>;

template <bool SYNC>
__global__ void __launch_bounds__(BATCH_TPB) batch_kernel(BatchParams bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KParams s_kp;
    __shared__ long long s_tile;
    const int tid = threadIdx.x;
    const long long total = bp.tile_begin[bp.n_ch];
    for (;;) {
        if (tid == 0) s_tile = (long long)atomicAdd(bp.tile_counter, 1ull);
        __syncthreads();
        const long long t = s_tile;
        if (t >= total) break;
        int c = 0;
        while (c + 1 < bp.n_ch && t >= bp.tile_begin[c + 1]) ++c;
        if (tid == 0) {
            s_kp = bp.kps[c];
            s_kp.iteration = bp.iteration;
        }
        __syncthreads();
        const long long lt = t - bp.tile_begin[c];
        const long long e0 = lt * bp.tile_events;
        const long long e1 = e0 + bp.tile_events < s_kp.n_events ? e0 + bp.tile_events : s_kp.n_events;
        switch (bp.proc[c]) {
        case MF_GG_TT:
            integrand_light<PGgTt, float, BATCH_TPB, false>(s_kp, smem_raw, e0, BATCH_TPB, e1,
                                                            bp.tile_out[c] + lt * (2 + PGgTt::D * s_kp.nb));
            break;
        case MF_UU_TT:
            integrand_light<PUuTt, float, BATCH_TPB, false>(s_kp, smem_raw, e0, BATCH_TPB, e1,
                                                            bp.tile_out[c] + lt * (2 + PUuTt::D * s_kp.nb));
            break;
        case MF_UG_TTU:
            integrand_light<PUgTtu, float, BATCH_TPB, false>(s_kp, smem_raw, e0, BATCH_TPB, e1,
                                                             bp.tile_out[c] + lt * (2 + PUgTtu::D * s_kp.nb));
            break;
        case MF_GG_TTG:
            integrand_heavy<PGgTtg, float, BATCH_TPB, false, SYNC>(s_kp, smem_raw, e0, BATCH_TPB, e1,
                                                                   bp.tile_out[c] + lt * (2 + PGgTtg::D * s_kp.nb));
            break;
        case MF_GG_TTGG:
            integrand_heavy<PGgTtgg, float, BATCH_TPB, false, SYNC>(s_kp, smem_raw, e0, BATCH_TPB, e1,
                                                                    bp.tile_out[c] + lt * (2 + PGgTtgg::D * s_kp.nb));
            break;
        default:
            break;
        }
        __syncthreads();   // shared memory is reused by the next tile
    }
}

}  // namespace mf

using namespace mf;

namespace {

size_t batch_smem(int nb, int npv)
{
    size_t m = 0;
    m = std::max(m, SmemLayout<PGgTt, float, BATCH_TPB>::bytes(nb, npv));
    m = std::max(m, SmemLayout<PUuTt, float, BATCH_TPB>::bytes(nb, npv));
    m = std::max(m, SmemLayout<PUgTtu, float, BATCH_TPB>::bytes(nb, npv));
    m = std::max(m, SmemLayout<PGgTtg, float, BATCH_TPB>::bytes(nb, npv));
    m = std::max(m, SmemLayout<PGgTtgg, float, BATCH_TPB>::bytes(nb, npv));
    return m;
}

#define MF_BCUDA(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return mf_fail(ctx, MF_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

int ensure_batch_buffers(mf_ctx* c, size_t tile_doubles)
{
    if (!c->cap_stream) {
        MF_BCUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        MF_BCUDA(c, cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming));
        MF_BCUDA(c, cudaEventCreateWithFlags(&c->ev_cap, cudaEventDisableTiming));
        MF_BCUDA(c, cudaMalloc(&c->d_kps, sizeof(KParams) * MAX_CH));
        MF_BCUDA(c, cudaMalloc(&c->d_bgrids, sizeof(double) * MAX_CH * MAX_DIM * (MAX_BINS + 1)));
        MF_BCUDA(c, cudaMalloc(&c->d_biter, sizeof(double) * MAX_CH * 1000 * 2));
        MF_BCUDA(c, cudaMalloc(&c->d_bsums, sizeof(double) * MAX_CH * (2 + MAX_DIM * MAX_BINS)));
        MF_BCUDA(c, cudaMalloc(&c->d_bcount, sizeof(unsigned long long) * (2 * MAX_CH + 1)));
        const size_t sm = batch_smem(MAX_BINS, 8192);
        MF_BCUDA(c, cudaFuncSetAttribute((const void*)batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        MF_BCUDA(c, cudaFuncSetAttribute((const void*)batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    }
    if (tile_doubles > c->tiles_cap) {
        cudaFree(c->d_tiles);
        c->d_tiles = nullptr;
        c->tiles_cap = 0;
        MF_BCUDA(c, cudaMalloc(&c->d_tiles, sizeof(double) * tile_doubles));
        c->tiles_cap = tile_doubles;
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_key.clear(); }
    }
    return MF_OK;
}

struct Plan {
    int n_ch = 0;
    int proc[MAX_CH];
    long long n[MAX_CH];
    int dim[MAX_CH];
    long long tiles[MAX_CH];
    BatchParams bp;
    std::vector<KParams> kps;
    int nblk = 0;
    size_t sm = 0;
    int sched = 1;
};

int make_plan(mf_ctx* c, int n_ch, const int* procs, const long long* n_events, double sqrt_s, long long tile,
              int sched, int bps, Plan& pl)
{
    if (n_ch < 1 || n_ch > MAX_CH || !procs || !n_events) return mf_fail(c, MF_ERR_ARG, "batch: bad channel list");
    if (c->cfg.precision != MF_MIXED) return mf_fail(c, MF_ERR_UNSUPPORTED, "batch: only the mixed precision is built");
    pl.n_ch = n_ch;
    pl.sched = sched;
    pl.kps.resize(n_ch);
    const int nb = c->cfg.n_bins;
    size_t tile_doubles = 0;
    for (int i = 0; i < n_ch; ++i) {
        const ProcOps* ops = mf_proc_ops(procs[i]);
        if (!ops || procs[i] == MF_EE_MUMU) return mf_fail(c, MF_ERR_ARG, "batch: channels must be hadronic top processes");
        if (n_events[i] < 2) return mf_fail(c, MF_ERR_ARG, "batch: every channel needs at least 2 events");
        pl.proc[i] = procs[i];
        pl.n[i] = n_events[i];
        pl.dim[i] = ops->D;
        pl.tiles[i] = (n_events[i] + tile - 1) / tile;
        tile_doubles += (size_t)pl.tiles[i] * (2 + ops->D * nb);
    }
    int rc = ensure_batch_buffers(c, tile_doubles);
    if (rc) return rc;
    std::memset(&pl.bp, 0, sizeof(pl.bp));
    pl.bp.kps = c->d_kps;
    pl.bp.n_ch = n_ch;
    pl.bp.tile_events = tile;
    pl.bp.tile_counter = c->d_bcount + 2 * MAX_CH;
    size_t off = 0;
    long long tb = 0;
    for (int i = 0; i < n_ch; ++i) {
        KParams& kp = pl.kps[i];
        rc = mf_make_params(c, procs[i], mf_proc_ops(procs[i]), sqrt_s, kp);
        if (rc) return rc;
        kp.channel = c->cfg.channel + (uint32_t)i;
        kp.n_events = n_events[i];
        kp.ev_offset = 0;
        kp.inv_n = 1.0 / (double)n_events[i];
        kp.grid = c->d_bgrids + (size_t)i * MAX_DIM * (MAX_BINS + 1);
        kp.counters = c->d_bcount + 2 * i;
        kp.partials = nullptr;
        pl.bp.proc[i] = procs[i];
        pl.bp.tile_begin[i] = tb;
        pl.bp.tile_out[i] = c->d_tiles + off;
        tb += pl.tiles[i];
        off += (size_t)pl.tiles[i] * (2 + pl.dim[i] * nb);
    }
    pl.bp.tile_begin[n_ch] = tb;
    pl.sm = batch_smem(nb, c->nx * c->nq);
    int per_sm = 0;
    MF_BCUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sched ? (const void*)batch_kernel<true>
                                                                               : (const void*)batch_kernel<false>,
                                                               BATCH_TPB, pl.sm));
    if (per_sm < 1) return mf_fail(c, MF_ERR_CUDA, "batch kernel does not fit on an SM");
    if (bps > 0 && bps < per_sm) per_sm = bps;
    pl.nblk = per_sm * c->n_sm;
    return MF_OK;
}

// the uniform starting grids of every channel and the counters
int reset_batch(mf_ctx* c, const Plan& pl, cudaStream_t s)
{
    const int nb = c->cfg.n_bins;
    std::vector<double> g((size_t)MAX_CH * MAX_DIM * (MAX_BINS + 1), 0.0);
    for (int i = 0; i < pl.n_ch; ++i)
        for (int d = 0; d < pl.dim[i]; ++d)
            for (int k = 0; k <= nb; ++k)
                g[(size_t)i * MAX_DIM * (MAX_BINS + 1) + (size_t)d * (nb + 1) + k] = (double)k / (double)nb;
    MF_BCUDA(c, cudaMemcpyAsync(c->d_bgrids, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    MF_BCUDA(c, cudaMemcpyAsync(c->d_kps, pl.kps.data(), sizeof(KParams) * pl.n_ch, cudaMemcpyHostToDevice, s));
    MF_BCUDA(c, cudaMemsetAsync(c->d_bcount, 0, sizeof(unsigned long long) * 2 * MAX_CH, s));
    // the pageable staging above must complete before the host vector goes away
    MF_BCUDA(c, cudaStreamSynchronize(s));
    return MF_OK;
}

// one iteration: the persistent launch, then per channel the tile reduction and the refinement
int enqueue_iteration(mf_ctx* c, Plan& pl, int it, int n_iter, cudaStream_t s)
{
    const int nb = c->cfg.n_bins;
    MF_BCUDA(c, cudaMemsetAsync(pl.bp.tile_counter, 0, sizeof(unsigned long long), s));
    pl.bp.iteration = (unsigned)it;
    if (pl.sched) batch_kernel<true><<<pl.nblk, BATCH_TPB, pl.sm, s>>>(pl.bp);
    else batch_kernel<false><<<pl.nblk, BATCH_TPB, pl.sm, s>>>(pl.bp);
    MF_BCUDA(c, cudaGetLastError());
    for (int i = 0; i < pl.n_ch; ++i) {
        const int ncol = 2 + pl.dim[i] * nb;
        finish_pass_kernel<<<1, 1024, ncol * sizeof(double), s>>>(
            pl.bp.tile_out[i], (int)pl.tiles[i], pl.dim[i], nb, pl.n[i], c->cfg.alpha, it < n_iter - 1,
            c->d_bgrids + (size_t)i * MAX_DIM * (MAX_BINS + 1), c->d_biter + ((size_t)i * 1000 + it) * 2,
            c->d_bsums + (size_t)i * (2 + MAX_DIM * MAX_BINS));
        MF_BCUDA(c, cudaGetLastError());
    }
    return MF_OK;
}

std::string plan_key(const mf_ctx* c, const Plan& pl, int n_iter, double sqrt_s)
{
    std::string k = std::to_string(n_iter) + "|" + std::to_string(sqrt_s) + "|" + std::to_string(pl.sched) + "|" +
                    std::to_string(pl.bp.tile_events) + "|" + std::to_string(pl.nblk) + "|" +
                    std::to_string(c->cfg.n_bins) + "|" + std::to_string(c->cfg.alpha) + "|" + std::to_string((unsigned long long)c->d_tiles);
    for (int i = 0; i < pl.n_ch; ++i) k += "|" + std::to_string(pl.proc[i]) + ":" + std::to_string(pl.n[i]);
    return k;
}

void combine(const double* it, int n_iter, double& mean, double& err, double& chi2dof)
{
    double sw = 0.0, swi = 0.0;
    for (int k = 0; k < n_iter; ++k) {
        const double wk = 1.0 / it[2 * k + 1];
        sw += wk;
        swi += wk * it[2 * k];
    }
    mean = swi / sw;
    err = std::sqrt(1.0 / sw);
    double chi2 = 0.0;
    for (int k = 0; k < n_iter; ++k) chi2 += (it[2 * k] - mean) * (it[2 * k] - mean) / it[2 * k + 1];
    chi2dof = n_iter > 1 ? chi2 / (n_iter - 1) : 0.0;
}

}  // namespace

extern "C" {

int mf_integrate_batch(mf_ctx* c, int n_ch, const int* processes, const long long* n_events, double sqrt_s,
                       int n_iter, mf_result* per_ch_host, mf_result* total_host, double* grids_host)
{
    if (!c) return MF_ERR_ARG;
    if (n_iter < 1 || n_iter > 1000 || !per_ch_host || !total_host || !(sqrt_s > 0.0))
        return mf_fail(c, MF_ERR_ARG, "mf_integrate_batch: bad argument");
    Plan pl;
    int rc = make_plan(c, n_ch, processes, n_events, sqrt_s, c->b_tile, c->b_sched, c->b_bps, pl);
    if (rc) return rc;
    // order against the caller's stream, then work on the private capture stream
    MF_BCUDA(c, cudaEventRecord(c->ev_user, c->stream));
    MF_BCUDA(c, cudaStreamWaitEvent(c->cap_stream, c->ev_user, 0));
    rc = reset_batch(c, pl, c->cap_stream);
    if (rc) return rc;
    const std::string key = plan_key(c, pl, n_iter, sqrt_s);
    if (!c->graph || c->graph_key != key) {
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
        cudaGraph_t g = nullptr;
        MF_BCUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        int erc = MF_OK;
        for (int it = 0; it < n_iter && erc == MF_OK; ++it) erc = enqueue_iteration(c, pl, it, n_iter, c->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
        if (erc) { if (g) cudaGraphDestroy(g); return erc; }
        if (ce != cudaSuccess) return mf_fail(c, MF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { c->graph = nullptr; return mf_fail(c, MF_ERR_CUDA, "graph instantiate failed"); }
        c->graph_key = key;
    }
    MF_BCUDA(c, cudaGraphLaunch(c->graph, c->cap_stream));
    std::vector<double> it((size_t)MAX_CH * 1000 * 2);
    std::vector<unsigned long long> cnt(2 * MAX_CH);
    MF_BCUDA(c, cudaMemcpyAsync(it.data(), c->d_biter, it.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cap_stream));
    MF_BCUDA(c, cudaMemcpyAsync(cnt.data(), c->d_bcount, cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                c->cap_stream));
    const int nb = c->cfg.n_bins;
    if (grids_host)
        for (int i = 0; i < n_ch; ++i)
            MF_BCUDA(c, cudaMemcpyAsync(grids_host + (size_t)i * MAX_DIM * (nb + 1),
                                        c->d_bgrids + (size_t)i * MAX_DIM * (MAX_BINS + 1),
                                        sizeof(double) * pl.dim[i] * (nb + 1), cudaMemcpyDeviceToHost, c->cap_stream));
    MF_BCUDA(c, cudaStreamSynchronize(c->cap_stream));
    c->b_last_nch = n_ch;
    for (int i = 0; i < n_ch; ++i) c->b_last_proc[i] = processes[i];
    double tot = 0.0, var = 0.0;
    long long ne = 0, np = 0, nn = 0;
    for (int i = 0; i < n_ch; ++i) {
        mf_result& r = per_ch_host[i];
        combine(&it[(size_t)i * 1000 * 2], n_iter, r.sigma_pb, r.error_pb, r.chi2_dof);
        r.n_events_total = n_events[i] * (long long)n_iter;
        r.n_pass = (long long)cnt[2 * i];
        r.n_nan = (long long)cnt[2 * i + 1];
        r.n_iter = n_iter;
        tot += r.sigma_pb;
        var += r.error_pb * r.error_pb;
        ne += r.n_events_total; np += r.n_pass; nn += r.n_nan;
    }
    total_host->sigma_pb = tot;
    total_host->error_pb = std::sqrt(var);
    total_host->chi2_dof = 0.0;
    total_host->n_events_total = ne;
    total_host->n_pass = np;
    total_host->n_nan = nn;
    total_host->n_iter = n_iter;
    return MF_OK;
}

int mf_batch_grad(mf_ctx* c, int n_ch, const int* processes, const long long* n_events, double sqrt_s,
                  unsigned int iteration, double* out_host)
{
    if (!c) return MF_ERR_ARG;
    if (n_ch < 1 || n_ch > MAX_CH || !processes || !n_events || !out_host || !(sqrt_s > 0.0))
        return mf_fail(c, MF_ERR_ARG, "mf_batch_grad: bad argument");
    if (c->cfg.precision != MF_MIXED) return mf_fail(c, MF_ERR_UNSUPPORTED, "batch: only the mixed precision is built");
    if (n_ch != c->b_last_nch || !std::equal(processes, processes + n_ch, c->b_last_proc))
        return mf_fail(c, MF_ERR_ARG, "mf_batch_grad: the channel list differs from the last mf_integrate_batch");
    for (int i = 0; i < n_ch; ++i)
        if (n_events[i] < 2) return mf_fail(c, MF_ERR_ARG, "mf_batch_grad: every channel needs at least 2 events");
    // per channel: sigma_hat, d sigma_hat/d m_t, sum (dw/N)^2, d sigma_hat/d alpha_s
    double* d_out = c->d_bsums;   // [n_ch][4]; d_bsums is free between batch calls
    MF_BCUDA(c, cudaEventRecord(c->ev_user, c->stream));
    MF_BCUDA(c, cudaStreamWaitEvent(c->cap_stream, c->ev_user, 0));
    for (int i = 0; i < n_ch; ++i) {
        const ProcOps* ops = mf_proc_ops(processes[i]);
        const GradOpsTable* g = mf_grad_ops(processes[i]);
        KParams kp;
        int rc = mf_make_params(c, processes[i], ops, sqrt_s, kp);
        if (rc) return rc;
        kp.channel = c->cfg.channel + (uint32_t)i;
        kp.iteration = iteration;
        kp.n_events = n_events[i];
        kp.ev_offset = 0;
        kp.inv_n = 1.0 / (double)n_events[i];
        kp.grid = c->d_bgrids + (size_t)i * MAX_DIM * (MAX_BINS + 1);
        kp.mask_in = nullptr;
        const long long want = (n_events[i] + 127) / 128, cap = (long long)c->n_sm * 8;
        const int nblk = (int)(want < cap ? want : cap);
        // the single-process partials buffer: this call is ordered after the caller's
        // stream and synchronises before returning, so nothing else uses it meanwhile
        double* part = c->d_partials;
        MF_BCUDA(c, g->grad(MF_MIXED, kp, nblk, part, g->k_as, c->cfg.alpha_s, c->cap_stream));
        finish_pass_kernel<<<1, 32, 4 * sizeof(double), c->cap_stream>>>(part, nblk, 1, 2, n_events[i], 0.0, 0, nullptr,
                                                                        nullptr, d_out + 4 * i);
        MF_BCUDA(c, cudaGetLastError());
    }
    std::vector<double> o(4 * (size_t)n_ch);
    MF_BCUDA(c, cudaMemcpyAsync(o.data(), d_out, o.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cap_stream));
    MF_BCUDA(c, cudaStreamSynchronize(c->cap_stream));
    double t[4] = { 0.0, 0.0, 0.0, 0.0 };
    for (int i = 0; i < n_ch; ++i) {
        const double n = (double)n_events[i], d = o[4 * i + 1], s2 = o[4 * i + 2];
        const double var = (n * s2 - d * d) / (n - 1.0);
        out_host[4 * i + 0] = o[4 * i + 0];
        out_host[4 * i + 1] = d;
        out_host[4 * i + 2] = std::sqrt(var > 0.0 ? var : 0.0);
        out_host[4 * i + 3] = o[4 * i + 3];
        t[0] += o[4 * i]; t[1] += d; t[2] += var > 0.0 ? var : 0.0; t[3] += o[4 * i + 3];
    }
    out_host[4 * n_ch + 0] = t[0];
    out_host[4 * n_ch + 1] = t[1];
    out_host[4 * n_ch + 2] = std::sqrt(t[2]);
    out_host[4 * n_ch + 3] = t[3];
    return MF_OK;
}

int mf_set_batch_schedule(mf_ctx* c, int sched, long long tile_events, int ctas_per_sm)
{
    if (!c) return MF_ERR_ARG;
    if ((sched != 0 && sched != 1) || tile_events < 32 || tile_events > (1LL << 26) || ctas_per_sm < 0 ||
        ctas_per_sm > 16)
        return mf_fail(c, MF_ERR_ARG, "mf_set_batch_schedule: bad argument");
    c->b_sched = sched;
    c->b_tile = tile_events;
    c->b_bps = ctas_per_sm;
    return MF_OK;
}

int mf_autotune_batch(mf_ctx* c, int n_ch, const int* processes, const long long* n_events, double sqrt_s,
                      int* choice_host)
{
    if (!c) return MF_ERR_ARG;
    if (!(sqrt_s > 0.0) || !n_events) return mf_fail(c, MF_ERR_ARG, "mf_autotune_batch: bad argument");
    // pilot: one pass over an eighth of every channel's events at the uniform grid
    std::vector<long long> pilot(n_ch > 0 && n_ch <= MAX_CH ? n_ch : 1);
    for (int i = 0; i < (int)pilot.size(); ++i) pilot[i] = std::max(2LL, n_events[i] / 8);
    const long long tiles[3] = { 2048, 4096, 16384 };
    float best = 1e30f;
    int best_s = c->b_sched, best_b = c->b_bps;
    long long best_t = c->b_tile;
    cudaEvent_t e0, e1;
    MF_BCUDA(c, cudaEventCreate(&e0));
    MF_BCUDA(c, cudaEventCreate(&e1));
    int rc = MF_OK;
    for (int sched = 0; sched <= 1 && rc == MF_OK; ++sched)
        for (long long tile : tiles)
            for (int bps = 1; bps <= 2 && rc == MF_OK; ++bps) {
                Plan pl;
                rc = make_plan(c, n_ch, processes, pilot.data(), sqrt_s, tile, sched, bps, pl);
                if (rc) break;
                rc = reset_batch(c, pl, c->cap_stream);
                if (rc) break;
                rc = enqueue_iteration(c, pl, 0, 1, c->cap_stream);   // warm-up
                if (rc) break;
                cudaEventRecord(e0, c->cap_stream);
                rc = enqueue_iteration(c, pl, 1, 2, c->cap_stream);
                if (rc) break;
                cudaEventRecord(e1, c->cap_stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = mf_fail(c, MF_ERR_CUDA, "autotune timing"); break; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; best_s = sched; best_t = tile; best_b = bps; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->b_sched = best_s;
    c->b_tile = best_t;
    c->b_bps = best_b;
    if (choice_host) { choice_host[0] = best_s; choice_host[1] = (int)best_t; choice_host[2] = best_b; }
    return MF_OK;
}

}  // extern "C"

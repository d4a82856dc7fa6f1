// Internal state of an mf_ctx and the helpers shared by the C ABI sources.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <utility>
#include <vector>

#include "mf_batch.cuh"
#include "mf_dispatch.cuh"
#include "../../include/madflow_gb300.h"

struct mf_ctx {
    mf_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0, n_sm = 0;
    int n_flav = 0, nx = 0, nq = 0;
    double x_min = 0, q2_min = 0, q2_max = 0;
    double* d_pdf = nullptr;
    mf::Df* d_pdf_df = nullptr;   // its double-float copy (the mixed-precision kinematics)
    double* d_grid = nullptr;        // [MAX_DIM][MAX_BINS+1]
    double* d_partials = nullptr;    // [max_blocks][2 + MAX_DIM MAX_BINS]
    double* d_iter = nullptr;        // [MAX_ITER][2]
    double* d_sums = nullptr;        // [2 + MAX_DIM MAX_BINS]
    unsigned long long* d_counters = nullptr;
    unsigned* d_err = nullptr;       // raised by a device wait that ran out
    double* d_kin = nullptr;         // kinematics of queued events (heavy integrand), per CTA
    uint8_t* d_kin_bins = nullptr;
    int kin_ctas = 0;
    float* d_inv = nullptr;          // per-event records of the warp-per-event schedule, per CTA
    int inv_ctas = 0;
    int max_blocks = 0;
    int sched = 4;                   // integrand schedule (see mf_set_schedule)
    int hsplit = 1;                  // lanes per event in the heavy integrand (see mf_set_helicity_split)
    int hel_samples = 0;             // sampled helicity configurations per event (mf_set_helicity_sampling)
    uint32_t hel_stream = 0;         // stream of the helicity draws
    // observable histogram (mf_set_observable): n bins from obs_lo, obs_inv_w = n / (hi - lo)
    int obs_n = 0;
    double obs_lo = 0.0, obs_hi = 0.0, obs_inv_w = 0.0;
    double* d_obs_partials = nullptr;   // [max_blocks][obs_n + 2][2]
    double* d_obs_iter = nullptr;       // [MAX_ITER][obs_n + 2][2]: per-bin (I, var) of each iteration
    int obs_iters = 0;                  // iterations behind obs_hist (0: none yet)
    std::vector<double> obs_hist, obs_err, obs_iter_host;
    std::string err;
    // batched channels: workspace, tuned schedule and the cached CUDA graph
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture and replay (high priority)
    // the channels that run as their own integrand kernels: one forked stream each, so that
    // they overlap (node priorities decide who goes first), joined back by their events
    cudaStream_t cap_side[mf::MAX_CH] = {};
    cudaEvent_t ev_side[mf::MAX_CH] = {};
    cudaEvent_t ev_user = nullptr, ev_cap = nullptr;
    mf::KParams* d_kps = nullptr;        // [MAX_CH]
    double* d_tiles = nullptr;           // tile partial sums of all channels
    size_t tiles_cap = 0;                // doubles
    double* d_bgrids = nullptr;          // [MAX_CH][MAX_DIM][MAX_BINS+1]
    double* d_biter = nullptr;           // [MAX_CH][1000][2]
    double* d_bsums = nullptr;           // [MAX_CH][2 + MAX_DIM MAX_BINS]
    unsigned long long* d_bcount = nullptr;   // [MAX_CH][2] counters, then the tile counter
    int b_mode = 0;                      // tuned: 0 one launch for all channels, 1 split (see mf_set_batch_schedule)
    int b_sched = 1, b_bps = 0;          // tuned: barrier schedule, CTAs per SM (0 = occupancy)
    long long b_tile_heavy = 4096;       // tuned: events per tile of the 2 -> 3 and 2 -> 4 gluon channels
    long long b_tile_light = 4096;       // tuned: events per tile of the other channels
    int b_hsplit = 1;                    // tuned: lanes per event of the 2 -> 3 and 2 -> 4 gluon channels
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    // mf_integrate: its iterations captured as CUDA graphs on a private stream, one per set of
    // launch parameters (the key), the INT_GRAPHS most recently used kept for replay (a caller
    // that integrates several channels in turn replays each one's graph)
    static constexpr size_t INT_GRAPHS = 16;
    cudaStream_t int_stream = nullptr;
    cudaEvent_t int_ev = nullptr;
    std::vector<std::pair<std::string, cudaGraphExec_t>> int_graphs;   // least recently used first
    int b_last_nch = 0;                  // channel list of the grids in d_bgrids
    int b_last_proc[mf::MAX_CH] = {};
};

int mf_fail(mf_ctx* c, int code, const std::string& msg);
int mf_make_params(mf_ctx* c, int process, const mf::ProcOps* ops, double sqrt_s, mf::KParams& kp,
                   const mf_cuts* cuts = nullptr);
const mf::ProcOps* mf_proc_ops(int process);
const mf::GradOpsTable* mf_grad_ops(int process);

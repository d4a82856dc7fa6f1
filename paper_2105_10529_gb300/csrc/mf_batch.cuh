// Batched channels: several partonic subprocesses with their own event
// counts and VEGAS grids in one persistent launch (the batched
// p p -> t tbar + jets set).
#pragma once
#include "mf_integrand.cuh"

namespace mf {

constexpr int MAX_CH = 8;
// rows per channel of the batch calls' caller-side grid and sum layouts ([n_ch][18][n_bins+1],
// [n_ch][2 + 18 n_bins]): the largest dimension of the batch's processes (g g -> t tbar g g)
constexpr int BATCH_DIM = 18;

// The work list of one persistent launch: slots (channels) in the order
// their tiles are handed out, most expensive events first.
struct BatchParams {
    const KParams* kps;                 // [n_slot] per-slot parameters (device memory)
    int proc[MAX_CH];                   // mf_process of each slot
    long long tile_begin[MAX_CH + 1];   // global tile index where each slot starts
    long long tile_events[MAX_CH];      // events per tile of each slot
    double* tile_out[MAX_CH];           // [tiles of the slot][2 + D nb] partial sums per tile
    int n_slot;
    unsigned long long* tile_counter;   // next tile to hand out (zeroed before the launch)
    unsigned int iteration;             // Philox iteration of this pass
};

}  // namespace mf

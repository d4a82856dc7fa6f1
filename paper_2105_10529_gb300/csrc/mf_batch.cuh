// Batched channels: several partonic subprocesses with their own event
// counts and VEGAS grids in one persistent launch (the batched
// p p -> t tbar + jets set).
#pragma once
#include "mf_integrand.cuh"

namespace mf {

constexpr int MAX_CH = 8;

struct BatchParams {
    const KParams* kps;                 // [n_ch] per-channel parameters (device memory)
    int proc[MAX_CH];                   // mf_process of each channel
    long long tile_begin[MAX_CH + 1];   // global tile index where each channel starts
    double* tile_out[MAX_CH];           // [tiles of the channel][2 + D nb] partial sums per tile
    int n_ch;
    long long tile_events;              // events per tile
    unsigned long long* tile_counter;   // next tile to hand out (zeroed before the launch)
    unsigned int iteration;             // Philox iteration of this pass
};

}  // namespace mf

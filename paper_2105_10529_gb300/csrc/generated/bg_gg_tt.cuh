// Generated by paper_2105_10529_gb300/gen/bg_tables.py -- do not edit.
// Berends-Giele tables of gg_tt: 2 gluons on a top line, 2 colour orderings,
// 3 stored gluon currents, 3 top-line currents.
#pragma once
#include <cstdint>
#include "mf_bg.cuh"
namespace mf {
namespace bg_gg_tt {
constexpr int K = 2;
constexpr int NPERM = 2;
constexpr int NJ = 3;     // stored gluon currents (ids: level by level)
constexpr int NU = 3;     // top-line currents (id 0: ubar)
constexpr double COLOUR_DEN = 3.0;
constexpr int JOFF1 = 0, NJ1 = 2;
constexpr int JOFF2 = 2, NJ2 = 1;
constexpr int UOFF1 = 1, NU1 = 2;
__device__ const uint8_t j2_mask[1] = {3};
__device__ const uint16_t j2_v3[1][1][2] = {0, 1};
__device__ const uint8_t j2_v3m[1][1][2] = {1, 2};
__device__ const uint8_t u1_mask[2] = {1, 2};
__device__ const uint16_t u1_terms[2][1][2] = {0, 0, 0, 1};
__device__ const uint16_t closure[2][2][2] = {0, 2, 1, 1, 0, 32770, 2, 0};
// C_{sigma tau} times COLOUR_DEN (integers), orderings lexicographic
__device__ const float colour[4] = {16, -2, -2, 16};
}  // namespace bg_gg_tt

// level drivers of the recursion of gg_tt (see mf_bg.cuh)
struct BgGen_gg_tt {
    static constexpr int K = 2, NPERM = 2, NJ = 3, NU = 3;
    static constexpr double COLOUR_DEN = 3.0;
    __device__ static const float* colour() { return bg_gg_tt::colour; }
    __device__ static const uint16_t* closure() { return &bg_gg_tt::closure[0][0][0]; }
    // gluon currents of 2 .. K gluons and top-line currents of 1 .. K-1 gluons from the
    // external states in w.J[0 .. K-1] and w.U[0]
    template <typename R, class W> __device__ static void forward(W& w, int lane)
    {
        namespace T = bg_gg_tt;
        for (int t = lane; t < T::NJ2 + T::NU1; t += 32) {
            if (t < T::NJ2) bg_gluon_current<R, 2, 0>(w, t, T::JOFF2, T::j2_mask, &T::j2_v3[0][0][0], &T::j2_v3m[0][0][0], nullptr);
            else bg_top_current<R, 1>(w, t - T::NJ2, T::UOFF1, T::u1_mask, &T::u1_terms[0][0][0]);
        }
        __syncwarp();
    }
    // the reverse sweep: adjoints of the currents (a.Jb, a.Ub, a.Vb from the closures)
    // and of the per-event invariants (into the lane's registers gi), level by level
    // downwards: top-line level m with gluon level m + 1 (each pushes only to lower levels)
    template <typename R, class W, class A, class I>
    __device__ static void reverse(const W& w, A& a, I& gi, int lane)
    {
        namespace T = bg_gg_tt;
        for (int t = lane; t < T::NJ2 + T::NU1; t += 32) {
            if (t < T::NJ2) bg_gluon_current_adj<R, 2, 0>(w, a, gi, t, T::JOFF2, T::j2_mask, &T::j2_v3[0][0][0], &T::j2_v3m[0][0][0], nullptr);
            else bg_top_current_adj<R, 1>(w, a, gi, t - T::NJ2, T::UOFF1, T::u1_mask, &T::u1_terms[0][0][0]);
        }
        __syncwarp();
    }
};
}  // namespace mf

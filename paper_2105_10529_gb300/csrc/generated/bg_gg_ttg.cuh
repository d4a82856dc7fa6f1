// Generated by paper_2105_10529_gb300/gen/bg_tables.py -- do not edit.
// Berends-Giele tables of gg_ttg: 3 gluons on a top line, 6 colour orderings,
// 9 stored gluon currents, 10 top-line currents.
#pragma once
#include <cstdint>
#include "mf_bg.cuh"
namespace mf {
namespace bg_gg_ttg {
constexpr int K = 3;
constexpr int NPERM = 6;
constexpr int NJ = 9;     // stored gluon currents (ids: level by level)
constexpr int NU = 10;     // top-line currents (id 0: ubar)
constexpr double COLOUR_DEN = 9.0;
constexpr int JOFF1 = 0, NJ1 = 3;
constexpr int JOFF2 = 3, NJ2 = 3;
constexpr int JOFF3 = 6, NJ3 = 3;
constexpr int UOFF1 = 1, NU1 = 3;
constexpr int UOFF2 = 4, NU2 = 6;
__device__ const uint8_t j2_mask[3] = {3, 5, 6};
__device__ const uint16_t j2_v3[3][1][2] = {0, 1, 0, 2, 1, 2};
__device__ const uint8_t j2_v3m[3][1][2] = {1, 2, 1, 4, 2, 4};
__device__ const uint8_t j3_mask[3] = {7, 7, 7};
__device__ const uint16_t j3_v3[3][2][2] = {0, 5, 3, 2, 0, 32773, 4, 1, 1, 4, 32771, 2};
__device__ const uint8_t j3_v3m[3][2][2] = {1, 6, 3, 4, 1, 6, 5, 2, 2, 5, 3, 4};
__device__ const uint16_t j3_v4[3][1][3] = {0, 1, 2, 0, 2, 1, 1, 0, 2};
__device__ const uint8_t u1_mask[3] = {1, 2, 4};
__device__ const uint16_t u1_terms[3][1][2] = {0, 0, 0, 1, 0, 2};
__device__ const uint8_t u2_mask[6] = {3, 5, 3, 6, 5, 6};
__device__ const uint16_t u2_terms[6][2][2] = {0, 3, 1, 1, 0, 4, 1, 2, 0, 32771, 2, 0, 0, 5, 2, 2, 0, 32772, 3, 0, 0, 32773, 3, 1};
__device__ const uint16_t closure[6][3][2] = {0, 6, 1, 5, 4, 2, 0, 7, 1, 32773, 5, 1, 0, 8, 2, 4, 6, 2, 0, 7, 2, 32772, 7, 0, 0, 8, 3, 3, 8, 1, 0, 6, 3, 32771, 9, 0};
// C_{sigma tau} times COLOUR_DEN (integers), orderings lexicographic
__device__ const float colour[36] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64};
}  // namespace bg_gg_ttg

// level drivers of the recursion of gg_ttg (see mf_bg.cuh)
struct BgGen_gg_ttg {
    static constexpr int K = 3, NPERM = 6, NJ = 9, NU = 10;
    static constexpr double COLOUR_DEN = 9.0;
    __device__ static const float* colour() { return bg_gg_ttg::colour; }
    __device__ static const uint16_t* closure() { return &bg_gg_ttg::closure[0][0][0]; }
    // gluon currents of 2 .. K gluons and top-line currents of 1 .. K-1 gluons from the
    // external states in w.J[0 .. K-1] and w.U[0]
    template <typename R, class W> __device__ static void forward(W& w, int lane)
    {
        namespace T = bg_gg_ttg;
        for (int t = lane; t < T::NJ2 + T::NU1; t += 32) {
            if (t < T::NJ2) bg_gluon_current<R, 2, 0>(w, t, T::JOFF2, T::j2_mask, &T::j2_v3[0][0][0], &T::j2_v3m[0][0][0], nullptr);
            else bg_top_current<R, 1>(w, t - T::NJ2, T::UOFF1, T::u1_mask, &T::u1_terms[0][0][0]);
        }
        __syncwarp();
        for (int t = lane; t < T::NJ3 + T::NU2; t += 32) {
            if (t < T::NJ3) bg_gluon_current<R, 3, 1>(w, t, T::JOFF3, T::j3_mask, &T::j3_v3[0][0][0], &T::j3_v3m[0][0][0], &T::j3_v4[0][0][0]);
            else bg_top_current<R, 2>(w, t - T::NJ3, T::UOFF2, T::u2_mask, &T::u2_terms[0][0][0]);
        }
        __syncwarp();
    }
    // the reverse sweep: adjoints of the currents (a.Jb, a.Ub, a.Vb from the closures)
    // and of the per-event invariants (into the lane's registers gi), level by level
    // downwards: top-line level m with gluon level m + 1 (each pushes only to lower levels)
    template <typename R, class W, class A, class I>
    __device__ static void reverse(const W& w, A& a, I& gi, int lane)
    {
        namespace T = bg_gg_ttg;
        for (int t = lane; t < T::NJ3 + T::NU2; t += 32) {
            if (t < T::NJ3) bg_gluon_current_adj<R, 3, 1>(w, a, gi, t, T::JOFF3, T::j3_mask, &T::j3_v3[0][0][0], &T::j3_v3m[0][0][0], &T::j3_v4[0][0][0]);
            else bg_top_current_adj<R, 2>(w, a, gi, t - T::NJ3, T::UOFF2, T::u2_mask, &T::u2_terms[0][0][0]);
        }
        __syncwarp();
        for (int t = lane; t < T::NJ2 + T::NU1; t += 32) {
            if (t < T::NJ2) bg_gluon_current_adj<R, 2, 0>(w, a, gi, t, T::JOFF2, T::j2_mask, &T::j2_v3[0][0][0], &T::j2_v3m[0][0][0], nullptr);
            else bg_top_current_adj<R, 1>(w, a, gi, t - T::NJ2, T::UOFF1, T::u1_mask, &T::u1_terms[0][0][0]);
        }
        __syncwarp();
    }
};
}  // namespace mf

// g g -> t tbar g g g (five gluons on the top line, 120 colour orderings,
// 128 helicity configurations): the multi-leg process of Sec. 4 of
// arXiv:2105.10529, evaluated by the warp-level Berends-Giele recursion of
// mf_bg.cuh with the tables of generated/bg_gg_ttggg.cuh.
#pragma once
#include <type_traits>
#include "mf_bg.cuh"
#include "generated/bg_gg_ttggg.cuh"

namespace mf {

struct Me_gg_ttggg {
    static constexpr int NEXT = 7;
    static constexpr int NHEL = 128;
    static constexpr int NGLUON = 5;
    static constexpr int NCOL = bg_gg_ttggg::NPERM;
    static constexpr double COLOUR_DEN = bg_gg_ttggg::COLOUR_DEN;
    static constexpr double AVG = 1.0 / 256.0;
    static constexpr double SYM = 1.0 / 6.0;          // three identical final gluons
    static constexpr bool TC_COLOUR = false;
    static constexpr bool BG = true;                  // warp-level recursion, no per-thread slot
    template <typename R> static constexpr size_t slot_bytes() { return 0; }
    template <typename R> using Warp = BgWarp<R, NGLUON, bg_gg_ttggg::NJ, bg_gg_ttggg::NU, bg_gg_ttggg::NPERM>;
    // shared memory of a CTA: the colour matrix (rows padded to an odd stride, so that the
    // lanes' rows fall in distinct banks), then one state per warp
    static constexpr int CROW = NCOL + 1;
    static __host__ __device__ constexpr size_t colour_bytes() { return sizeof(float) * NCOL * CROW; }
    template <typename R> static __host__ __device__ constexpr size_t warp_bytes() { return (sizeof(Warp<R>) + 15) & ~(size_t)15; }
    template <typename R> static __host__ __device__ constexpr size_t cta_bytes(int warps)
    {
        return colour_bytes() + (size_t)warps * warp_bytes<R>();
    }
    __device__ static const float* colour_table() { return bg_gg_ttggg::colour; }
    // copies the colour matrix into the CTA's region (every thread of the CTA calls)
    __device__ static void load_colour(float* cs)
    {
        for (int i = threadIdx.x; i < NCOL * NCOL; i += blockDim.x) cs[(i / NCOL) * CROW + i % NCOL] = __ldg(colour_table() + i);
    }

    // sum over helicities of sum_{sigma tau} A*_sigma C_{sigma tau} A_tau / COLOUR_DEN for one
    // event, by the whole warp (bg_warp_me2; couplings and averages: norm())
    template <typename R>
    __device__ static double warp_me2(Warp<R>& w, const float* cs, const double* pev, int stride, double mt,
                                      bool all_hel, double* hel_out, double hel_scale, int nsamp = 0,
                                      uint4 rnd = uint4{ 0u, 0u, 0u, 0u })
    {
        return bg_warp_me2<BgGen_gg_ttggg, R>(w, cs, CROW, pev, stride, mt, all_hel, hel_out, hel_scale, nsamp, rnd);
    }
    // couplings, averages and symmetry factor that turn warp_me2 into the averaged |M|^2
    __host__ __device__ static double norm(double gs)
    {
        double g = 1.0;
        for (int i = 0; i < NGLUON; ++i) g *= gs * gs;
        return g * AVG * SYM;
    }
};

// mf_evaluate and the helicity profile for the warp-level matrix element: one warp per point
template <typename R>
__global__ void __launch_bounds__(128) bg_evaluate_kernel(const double* __restrict__ mom, long long n, double* me2,
                                                          double* hel_out, double mt, double gs)
{
    using ME = Me_gg_ttggg;
    extern __shared__ __align__(128) unsigned char mf_bg_smem[];
    float* cs = reinterpret_cast<float*>(mf_bg_smem);
    ME::load_colour(cs);
    __syncthreads();
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto& w = *reinterpret_cast<typename ME::template Warp<R>*>(mf_bg_smem + ME::colour_bytes() + warp * ME::warp_bytes<R>());
    const double nrm = ME::norm(gs);
    for (long long e = (long long)blockIdx.x * nw + warp; e < n; e += (long long)gridDim.x * nw) {
        const double* pe = mom + e * ME::NEXT * 4;
        double* ho = hel_out ? hel_out + e * ME::NHEL : nullptr;
        const double v = ME::warp_me2<R>(w, cs, pe, 1, mt, ho != nullptr, ho, nrm / ME::COLOUR_DEN);
        if (me2 && (threadIdx.x & 31) == 0) me2[e] = v * nrm;
    }
}

}  // namespace mf

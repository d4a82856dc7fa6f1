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

    // sum over helicities of sum_{sigma tau} A*_sigma C_{sigma tau} A_tau for one event, by the
    // whole warp (couplings and averages not applied: multiply by norm()).  pev: the event's FP64
    // momenta, component 4 i + c (particle i: g, g, t, tbar, g, g, g) at pev[(4 i + c) stride].
    // all_hel: every configuration (else one of each parity pair, doubled); hel_out (nullable,
    // all_hel): each configuration's value, times hel_scale, written by lane 0.
    template <typename R>
    __device__ static double warp_me2(Warp<R>& w, const float* cs, const double* pev, int stride, double mt,
                                      bool all_hel, double* hel_out, double hel_scale)
    {
        using namespace bg_gg_ttggg;
        const int lane = threadIdx.x & 31;
        double p[NEXT][4];
        for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = pev[(size_t)f * stride];
        constexpr int gl_ext[K] = { 0, 1, 4, 5, 6 };
        {
            // subset momenta and inverse denominators (FP64), one subset per lane
            const int msk = lane;
            if (msk >= 1) {
                double P[4] = { 0.0, 0.0, 0.0, 0.0 };
                for (int i = 0; i < K; ++i)
                    if (msk >> i & 1) {
                        const double sg = i < 2 ? 1.0 : -1.0;
                        for (int c = 0; c < 4; ++c) P[c] += sg * p[gl_ext[i]][c];
                    }
                double q[4];
                for (int c = 0; c < 4; ++c) { w.P[msk][c] = R(P[c]); q[c] = p[2][c] - P[c]; w.Q[msk][c] = R(q[c]); }
                w.iP2[msk] = __popc(msk) >= 2 ? R(1.0 / mdot(P, P)) : R(0);
                w.iQ[msk] = R(1.0 / (mdot(q, q) - mt * mt));
            }
            if (lane < K) {
                double a[3], b[3];
                gluon_basis(p[gl_ext[lane]], a, b);
                for (int j = 0; j < 3; ++j) { w.e1[lane][j] = R(a[j]); w.e2[lane][j] = R(b[j]); }
            }
            if (lane == K) w.fb3 = fermion_basis<R>(p[2], mt);
            if (lane == K + 1) w.fb4 = fermion_basis<R>(p[3], mt);
            if (lane == K + 2) w.mt = R(mt);
        }
        __syncwarp();
        R total = R(0);
        const int h0 = all_hel ? 0 : 1, hstep = all_hel ? 1 : 2;
#pragma unroll 1
        for (int ih = h0; ih < NHEL; ih += hstep) {
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
            if (lane < K) w.J[lane] = ext_gluon(w.e1[lane], w.e2[lane], HEL(gl_ext[lane]), lane >= 2);
            else if (lane == K) w.U[0] = ext_ubar(w.fb3, HEL(2));
            else if (lane == K + 1) w.V = ext_v(w.fb4, HEL(3));
#undef HEL
            __syncwarp();
            for (int t = lane; t < NJ2 + NU1; t += 32) {
                if (t < NJ2) bg_gluon_current<R, 2, 0>(w, t, JOFF2, j2_mask, &j2_v3[0][0][0], &j2_v3m[0][0][0], nullptr);
                else bg_top_current<R, 1>(w, t - NJ2, UOFF1, u1_mask, &u1_terms[0][0][0]);
            }
            __syncwarp();
            for (int t = lane; t < NJ3 + NU2; t += 32) {
                if (t < NJ3) bg_gluon_current<R, 3, 1>(w, t, JOFF3, j3_mask, &j3_v3[0][0][0], &j3_v3m[0][0][0], &j3_v4[0][0][0]);
                else bg_top_current<R, 2>(w, t - NJ3, UOFF2, u2_mask, &u2_terms[0][0][0]);
            }
            __syncwarp();
            for (int t = lane; t < NJ4 + NU3; t += 32) {
                if (t < NJ4) bg_gluon_current<R, 4, 3>(w, t, JOFF4, j4_mask, &j4_v3[0][0][0], &j4_v3m[0][0][0], &j4_v4[0][0][0]);
                else bg_top_current<R, 3>(w, t - NJ4, UOFF3, u3_mask, &u3_terms[0][0][0]);
            }
            __syncwarp();
            for (int t = lane; t < NJ5 + NU4; t += 32) {
                if (t < NJ5) bg_gluon_current<R, 5, 6>(w, t, JOFF5, j5_mask, &j5_v3[0][0][0], &j5_v3m[0][0][0], &j5_v4[0][0][0]);
                else bg_top_current<R, 4>(w, t - NJ5, UOFF4, u4_mask, &u4_terms[0][0][0]);
            }
            __syncwarp();
            // partial amplitudes: the top line closed on v(p_tbar)
            for (int s = lane; s < NPERM; s += 32) {
                cx<R> a = mkc(R(0), R(0));
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int ui = __ldg(&closure[s][j][0]);
                    const uint16_t r = __ldg(&closure[s][j][1]);
                    const cx<R> t = ffv_amp(w.U[ui], w.V, w.J[ref_id(r)]);
                    const R sg = ref_sign<R>(r);
                    a.r = fma(sg, t.r, a.r);
                    a.i = fma(sg, t.i, a.i);
                }
                w.A[s] = a;
            }
            __syncwarp();
            // colour sum: lane rows sigma = lane, lane + 32, ...
            R part = R(0);
            for (int s = lane; s < NPERM; s += 32) {
                const float* row = cs + s * CROW;
                R yr = R(0), yi = R(0);
#pragma unroll 8
                for (int t = 0; t < NPERM; ++t) {
                    const R c = R(row[t]);
                    yr = fma(c, w.A[t].r, yr);
                    yi = fma(c, w.A[t].i, yi);
                }
                part = fma(w.A[s].r, yr, fma(w.A[s].i, yi, part));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (hel_out && lane == 0) hel_out[ih] = double(part) * hel_scale;
            total += part;
            __syncwarp();
        }
        return double(total) * (all_hel ? 1.0 : 2.0) / COLOUR_DEN;
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

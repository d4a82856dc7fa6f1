// The event kinematics of the mixed-precision path in double-float arithmetic (mf_df.cuh):
// the same steps as the FP64 kinematics of mf_device.cuh (VEGAS map, parton map, RAMBO,
// log-bicubic PDFs), carried on the FP32 pipes with about 48 bits.  Their decisions keep
// the FP64 path's outcome: the VEGAS bin is the one of the FP64 product u nb, reproduced
// exactly in integers, and the cut predicates take the lab-frame momenta as doubles.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include "mf_df.cuh"
#include "mf_device.cuh"

namespace mf {

// double-float copies of a pass's kinematic constants, filled by the host next to their FP64
// values (fill_kin_df)
struct KinDf {
    Df S, ln_tau0, mt, gs, vol_const, ln_muf2_fixed;
    Df lx0, hx, ihx, lq0, lq1, hq, ihq;   // the PDF grid's geometry
};

inline void fill_kin_df(KinDf& k, double S, double ln_tau0, double mt, double gs, double vol_const,
                        double ln_muf2_fixed, const PdfGeom& g)
{
    k.S = Df(S); k.ln_tau0 = Df(ln_tau0); k.mt = Df(mt); k.gs = Df(gs); k.vol_const = Df(vol_const);
    k.ln_muf2_fixed = Df(ln_muf2_fixed);
    k.lx0 = Df(g.lx0); k.hx = Df(g.hx); k.ihx = Df(g.ihx);
    k.lq0 = Df(g.lq0); k.lq1 = Df(g.lq1); k.hq = Df(g.hq); k.ihq = Df(g.ihq);
}

// the nearest double-floats of n doubles (the PDF grid's copy)
inline std::vector<Df> split_df(const double* a, size_t n)
{
    std::vector<Df> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = Df(a[i]);
    return v;
}

#ifdef __CUDACC__

// the 52-bit integers k of an event's uniforms u = (k + 1/2) 2^-52: the Philox words that
// event_uniforms turns into doubles
template <int D>
__device__ __forceinline__ void event_words(unsigned long long ev, uint32_t iteration, uint32_t channel, uint2 key,
                                            unsigned long long (&k)[D])
{
#pragma unroll
    for (int b = 0; 2 * b < D; ++b) {
        const uint4 c = make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), iteration, (channel << 8) | (uint32_t)b);
        const uint4 o = philox4x32_10(c, key);
        k[2 * b] = ((unsigned long long)(o.x >> 6) << 26) | (unsigned long long)(o.y >> 6);
        if (2 * b + 1 < D) k[2 * b + 1] = ((unsigned long long)(o.z >> 6) << 26) | (unsigned long long)(o.w >> 6);
    }
}

// VEGAS map (Lepage 1978) in double-float.  u nb = (2k + 1) nb 2^-53 is an exact integer
// multiple of 2^-53; rounding it to 53 significant bits, nearest-even, gives fl(u nb), from
// which the bin b = floor(fl(u nb)) (clamped to nb - 1) is exactly the FP64 map's and
// fl(u nb) - b is its fraction.  Then x = e_b + w_b frac and J = prod_d nb w_b with the
// double-float edges gdf [D][nb+1], or where a kernel keeps no such copy (gdf null) with the
// FP64 edges g converted.
template <int D>
__device__ __forceinline__ Df vegas_map_df(const Df* gdf, const double* g, int nb, const unsigned long long (&k)[D],
                                           Df (&x)[D], uint8_t (&bins)[D])
{
    Df jac(1.0f, 0.0f);
    const float nbf = (float)nb;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const unsigned long long N = (2ull * k[d] + 1ull) * (unsigned long long)nb;   // < 2^59
        const int nbits = 64 - __clzll((long long)N);
        const int sh = nbits > 53 ? nbits - 53 : 0;
        unsigned long long q = N >> sh;
        if (sh > 0) {
            const unsigned long long rem = N & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
            q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
        }
        const unsigned long long Y = q << sh;   // fl(u nb) 2^53
        int b = (int)(Y >> 53);
        b = b > nb - 1 ? nb - 1 : b;
        const unsigned long long F = Y - ((unsigned long long)b << 53);   // (fl(u nb) - b) 2^53, at most 2^53
        const Df frac = df_two_sum(__fmul_rn((float)(uint32_t)(F >> 29), 0x1p-24f),
                                   __fmul_rn((float)(uint32_t)(F & 0x1FFFFFFFull), 0x1p-53f));
        const int i0 = d * (nb + 1) + b;
        const Df lo = gdf ? gdf[i0] : Df(g[i0]);
        const Df w = (gdf ? gdf[i0 + 1] : Df(g[i0 + 1])) - lo;
        x[d] = df_add(lo, df_mul(w, frac));
        jac = df_mul(jac, df_mul(w, nbf));
        bins[d] = (uint8_t)b;
    }
    return jac;
}

// RAMBO (Kleiss, Stirling, Ellis, CPC 40 (1986) 359) in double-float, as rambo() of
// mf_device.cuh: particles 0 and 1 of mass mt, the rest massless.  Newton's iteration for the
// massive rescaling stops at |f| < 4e-13 sqrt(shat), the double-float rounding of the energy
// sum being about 1e-14 of it.
template <int N>
__device__ __forceinline__ Df rambo_df(const Df& rs, const Df& mt, const Df* u, Df (&p)[N][4], const Df& vol_massless)
{
    Df q[N][4];
    Df Q0(0.0f, 0.0f), Q1(0.0f, 0.0f), Q2(0.0f, 0.0f), Q3(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const Df c = df_add(df_scale(u[4 * i], 2.0f), -1.0f);
        const Df s = sqrt(df_add(-df_mul(c, c), 1.0f));
        Df sf, cf;
        sincospi(df_scale(u[4 * i + 1], 2.0f), &sf, &cf);
        const Df e = -log(df_mul(u[4 * i + 2], u[4 * i + 3]));
        q[i][0] = e;
        q[i][1] = e * s * cf;
        q[i][2] = e * s * sf;
        q[i][3] = e * c;
        Q0 = Q0 + q[i][0]; Q1 = Q1 + q[i][1]; Q2 = Q2 + q[i][2]; Q3 = Q3 + q[i][3];
    }
    const Df M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
    const Df iM = df_div(Df(1.0f, 0.0f), M);
    const Df b1 = -(Q1 * iM), b2 = -(Q2 * iM), b3 = -(Q3 * iM);
    const Df x = rs * iM;
    const Df g = Q0 * iM, a = df_div(Df(1.0f, 0.0f), df_add(g, 1.0f));
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const Df bq = b1 * q[i][1] + b2 * q[i][2] + b3 * q[i][3];
        const Df q0 = q[i][0];
        p[i][0] = x * (g * q0 + bq);
        p[i][1] = x * (q[i][1] + b1 * q0 + a * bq * b1);
        p[i][2] = x * (q[i][2] + b2 * q0 + a * bq * b2);
        p[i][3] = x * (q[i][3] + b3 * q0 + a * bq * b3);
    }
    if (!(mt.hi > 0.0f)) return vol_massless;
    const Df msum = df_scale(mt, 2.0f);
    if (msum >= rs) return Df(0.0f, 0.0f);
    const Df mr = msum / rs;
    Df xi = sqrt(df_add(-(mr * mr), 1.0f));
    if constexpr (N == 2) {
        // two equal masses: as the FP64 path, the massive pair from the half difference of the
        // massless momenta, rescaled to length xi sqrt(shat)/2 with the first-order correction of
        // its deviation from back to back
        const Df h = df_scale(rs, 0.5f);
        const Df d1 = df_scale(p[0][1] - p[1][1], 0.5f), d2 = df_scale(p[0][2] - p[1][2], 0.5f);
        const Df d3 = df_scale(p[0][3] - p[1][3], 0.5f);
        const Df dd = d1 * d1 + d2 * d2 + d3 * d3;
        const Df c = xi * (1.5 - df_scale(dd / (h * h), 0.5f));
        p[0][0] = h; p[0][1] = c * d1; p[0][2] = c * d2; p[0][3] = c * d3;
        p[1][0] = h; p[1][1] = -(c * d1); p[1][2] = -(c * d2); p[1][3] = -(c * d3);
        return vol_massless * xi;
    } else {
        const Df mt2 = mt * mt;
        Df e2[N];
#pragma unroll
        for (int i = 0; i < N; ++i) e2[i] = p[i][0] * p[i][0];
        const Df tol = df_mul(rs, 4e-13f);
        // f(xi) = sum_i E_i(xi) - sqrt(shat), E_i = sqrt(m_i^2 + xi^2 E0_i^2) (xi E0_i when massless)
        for (int it = 0; it < 40; ++it) {
            Df f = -rs, fp(0.0f, 0.0f);
            const Df xi2 = xi * xi;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (i < 2) {
                    const Df ei = sqrt(xi2 * e2[i] + mt2);
                    f = f + ei;
                    fp = fp + xi * e2[i] / ei;
                } else {
                    f = f + xi * p[i][0];
                    fp = fp + p[i][0];
                }
            }
            xi = xi - f / fp;
            if (fabs(f) < tol) break;
        }
        Df sk(0.0f, 0.0f), sk2e(0.0f, 0.0f), prod(1.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const Df ka = xi * p[i][0];
            const Df e = i < 2 ? sqrt(mt2 + ka * ka) : ka;
            const Df ie = df_div(Df(1.0f, 0.0f), e);
            p[i][1] = p[i][1] * xi; p[i][2] = p[i][2] * xi; p[i][3] = p[i][3] * xi;
            p[i][0] = e;
            sk = sk + ka;
            sk2e = sk2e + ka * ka * ie;
            prod = prod * (ka * ie);
        }
        Df pw(1.0f, 0.0f);
        const Df r = sk / rs;
#pragma unroll
        for (int i = 0; i < 2 * N - 3; ++i) pw = pw * r;
        return vol_massless * pw * prod * rs / sk2e;
    }
}

// ------------------------------------------------------------------ log-bicubic PDF

// cubic Hermite basis at t (the weights of f0, h d0, f1, h d1, as hermite3h)
struct DfHermite { Df h00, h10, h01, h11; };
__device__ __forceinline__ DfHermite df_hermite(const Df& t)
{
    const Df t2 = t * t, t3 = t2 * t;
    DfHermite h;
    h.h00 = df_add(df_add(df_scale(t3, 2.0f), -df_mul(t2, 3.0f)), 1.0f);
    h.h10 = df_add(df_add(t3, -df_scale(t2, 2.0f)), t);
    h.h01 = df_add(-df_scale(t3, 2.0f), df_mul(t2, 3.0f));
    h.h11 = df_add(t3, -t2);
    return h;
}
__device__ __forceinline__ Df df_hermite_sum(const DfHermite& h, const Df& f0, const Df& f1, const Df& hd0, const Df& hd1)
{
    return h.h00 * f0 + h.h10 * hd0 + h.h01 * f1 + h.h11 * hd1;
}
// one grid node: from the double-float copy of the grid where there is one, else converted
__device__ __forceinline__ Df pdf_node(const double* g, const Df* gdf, int idx)
{
    return gdf ? gdf[idx] : Df(g[idx]);
}
// the Hermite interpolation in ln x of row jr over cell i (pdf_row)
__device__ __forceinline__ Df pdf_row_df(const double* g, const Df* gdf, const PdfGeom& G, int i, int jr,
                                         const DfHermite& h)
{
    const int nq = G.nq, nx = G.nx;
    const Df f0 = pdf_node(g, gdf, i * nq + jr), f1 = pdf_node(g, gdf, (i + 1) * nq + jr);
    const Df hd0 = i == 0 ? f1 - f0 : df_scale(f1 - pdf_node(g, gdf, (i - 1) * nq + jr), 0.5f);
    const Df hd1 = (i + 1 == nx - 1) ? f1 - f0 : df_scale(pdf_node(g, gdf, (i + 2) * nq + jr) - f0, 0.5f);
    return df_hermite_sum(h, f0, f1, hd0, hd1);
}
// x f(x, Q^2) from lx = ln x and lq = ln Q^2 (pdf_xf_log in double-float): g the FP64 grid of
// the flavour, gdf its double-float copy (nullable), K the grid geometry in double-float
template <typename KD>
__device__ __forceinline__ Df pdf_xf_df(const double* g, const Df* gdf, const PdfGeom& G, const KD& K, Df lx, Df lq)
{
    if (lq < K.lq0) lq = K.lq0;
    if (lq > K.lq1) lq = K.lq1;
    int i = df_floor((lx - K.lx0) * K.ihx);
    i = i < 0 ? 0 : (i > G.nx - 2 ? G.nx - 2 : i);
    int j = df_floor((lq - K.lq0) * K.ihq);
    j = j < 0 ? 0 : (j > G.nq - 2 ? G.nq - 2 : j);
    const Df t = (lx - df_add(K.lx0, df_mul(K.hx, (float)i))) * K.ihx;
    const Df s = (lq - df_add(K.lq0, df_mul(K.hq, (float)j))) * K.ihq;
    const DfHermite ht = df_hermite(t);
    const Df r1 = pdf_row_df(g, gdf, G, i, j, ht);
    const Df r2 = pdf_row_df(g, gdf, G, i, j + 1, ht);
    const Df r0 = j > 0 ? pdf_row_df(g, gdf, G, i, j - 1, ht) : Df(0.0f, 0.0f);
    const Df r3 = (j + 2 < G.nq) ? pdf_row_df(g, gdf, G, i, j + 2, ht) : Df(0.0f, 0.0f);
    const Df hdj = j == 0 ? r2 - r1 : df_scale(r2 - r0, 0.5f);
    const Df hdj1 = (j + 1 == G.nq - 1) ? r2 - r1 : df_scale(r3 - r1, 0.5f);
    return df_hermite_sum(df_hermite(s), r1, r2, hdj, hdj1);
}

#endif  // __CUDACC__

}  // namespace mf

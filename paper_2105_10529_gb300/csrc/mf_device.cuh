// Device building blocks of the per-event integrand of arXiv:2105.10529
// (Sec. 2.1: random numbers -> phase-space kinematics -> matrix element ->
// histogram accumulation; Sec. 1: VEGAS integrator, PDF interpolation,
// phase-space generator with fiducial cuts).
//
// Bit-exactness contract with the reference implementation: the random
// stream, the VEGAS bin indices and mapped points are integer or correctly
// rounded single operations written with explicit *_rn intrinsics, so no
// contraction or reassociation can change them.
#pragma once
#include <cstdint>
#include "mf_dual.cuh"

namespace mf {

// ------------------------------------------------------------------ a1: Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of the 4x32 Philox S-box,
// key bumped by the golden-ratio Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Two words -> double in (0,1): 52-bit integer from the top 26 bits of each
// word, u = (k + 1/2) 2^-52 (exact).
__device__ __forceinline__ double u01_from(uint32_t a, uint32_t b)
{
    const unsigned long long k = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
    return __dmul_rn(__dadd_rn(__ull2double_rn(k), 0.5), 2.220446049250313080847e-16);
}

// Uniforms of one event: block b of the counter (event lo, event hi,
// iteration, channel<<8 | b) under key (seed lo, seed hi) gives dims 2b, 2b+1.
template <int D>
__device__ __forceinline__ void event_uniforms(unsigned long long ev, uint32_t iteration, uint32_t channel,
                                               uint2 key, double (&u)[D])
{
#pragma unroll
    for (int b = 0; 2 * b < D; ++b) {
        const uint4 c = make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), iteration, (channel << 8) | (uint32_t)b);
        const uint4 o = philox4x32_10(c, key);
        u[2 * b] = u01_from(o.x, o.y);
        if (2 * b + 1 < D) u[2 * b + 1] = u01_from(o.z, o.w);
    }
}

// ------------------------------------------------------------------ a2: VEGAS map
// bin = floor(nb u) (clamped), x = e_b + w (nb u - b), J *= nb w (Lepage 1978).
// grid: [d][nb+1] edges in shared memory.
template <int D>
__device__ __forceinline__ double vegas_map(const double* grid, int nb, const double (&u)[D], double (&x)[D],
                                            uint8_t (&bins)[D])
{
    double jac = 1.0;
    const double nbd = (double)nb;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const double y = __dmul_rn(u[d], nbd);
        int b = __double2int_rz(y);
        b = b > nb - 1 ? nb - 1 : b;
        const double frac = __dsub_rn(y, (double)b);
        const double* e = grid + d * (nb + 1);
        const double lo = e[b], hi = e[b + 1];
        const double width = __dsub_rn(hi, lo);
        x[d] = __fma_rn(width, frac, lo);
        jac = __dmul_rn(jac, __dmul_rn(nbd, width));
        bins[d] = (uint8_t)b;
    }
    return jac;
}

// ------------------------------------------------------------------ a3: parton map
// tau = tau0^x0, x1 = tau^v, x2 = tau^(1-v), J = tau |ln tau| |ln tau0|.
// S: double, or Dual<double> when tau0 carries a derivative.
// Returns tau = x1 x2; lx1, lx2 receive ln x1 = v ln tau and ln x2 = (1 - v) ln tau
// (the PDF lookups and the lab rapidity need only these, not x1 and x2 themselves).
template <typename S>
__device__ __forceinline__ void parton_map(double x0, double v, S ln_tau0, S& tau, S& jac, S& lx1, S& lx2)
{
    const S lt = x0 * ln_tau0;
    lx1 = v * lt;
    lx2 = (1.0 - v) * lt;
    tau = exp(lt);
    jac = tau * (-lt) * (-ln_tau0);
}

// ------------------------------------------------------------------ a4: RAMBO
// Kleiss, Stirling, Ellis, CPC 40 (1986) 359: N isotropic massless momenta
// from 4N uniforms, conformal boost + scale to (sqrt(shat), 0), massive
// rescaling xi by Newton's method (bounded iterations) and the massive
// weight factor.  Returns the phase-space weight; p gets (E,px,py,pz).
template <int N, typename S>
__device__ __forceinline__ S rambo(S rs, const S (&m)[N], const double* u, S (&p)[N][4], S vol_massless)
{
    double q[N][4];
    double Q0 = 0.0, Q1 = 0.0, Q2 = 0.0, Q3 = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double c = 2.0 * u[4 * i] - 1.0;
        const double s = sqrt(1.0 - c * c);
        double sf, cf;
        sincospi(2.0 * u[4 * i + 1], &sf, &cf);
        const double e = -log(u[4 * i + 2] * u[4 * i + 3]);
        q[i][0] = e;
        q[i][1] = e * s * cf;
        q[i][2] = e * s * sf;
        q[i][3] = e * c;
        Q0 += q[i][0]; Q1 += q[i][1]; Q2 += q[i][2]; Q3 += q[i][3];
    }
    const double M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
    const double iM = 1.0 / M;
    const double b1 = -Q1 * iM, b2 = -Q2 * iM, b3 = -Q3 * iM;
    const S x = rs * iM;
    const double g = Q0 * iM, a = 1.0 / (1.0 + g);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double bq = b1 * q[i][1] + b2 * q[i][2] + b3 * q[i][3];
        const double q0 = q[i][0];
        p[i][0] = x * (g * q0 + bq);
        p[i][1] = x * (q[i][1] + b1 * q0 + a * bq * b1);
        p[i][2] = x * (q[i][2] + b2 * q0 + a * bq * b2);
        p[i][3] = x * (q[i][3] + b3 * q0 + a * bq * b3);
    }
    S msum = S(0.0);
    bool massive = false;
#pragma unroll
    for (int i = 0; i < N; ++i) { msum = msum + m[i]; massive |= (val(m[i]) != 0.0); }
    if (!massive) return vol_massless;
    if (msum >= rs) return S(0.0);
    S xi = sqrt(1.0 - (msum / rs) * (msum / rs));
    if constexpr (N == 2 && !is_dual<S>::value) {
        // two equal masses: the massless energies are both sqrt(shat)/2, so this
        // xi solves sum_i E_i(xi) = sqrt(shat) exactly, each massive energy is
        // sqrt(shat)/2 and the weight factor reduces to xi (= beta)
        if (m[0] == m[1]) {
            // The massless momenta leave the conformal map back to back with |k| = sqrt(shat)/2
            // only up to rounding amplified by the map's boost (about gamma^2 eps); the massive
            // pair is built from their half difference d, rescaled to length xi sqrt(shat)/2
            // with a first-order correction of |d| (its deviation is ~1e-10 at most, so the
            // neglected second order is far below rounding): exactly back to back, on its
            // mass shell to rounding
            const S h = 0.5 * rs;
            const S d1 = 0.5 * (p[0][1] - p[1][1]), d2 = 0.5 * (p[0][2] - p[1][2]), d3 = 0.5 * (p[0][3] - p[1][3]);
            const S dd = d1 * d1 + d2 * d2 + d3 * d3;
            const S c = xi * (1.5 - 0.5 * dd / (h * h));
            p[0][0] = h; p[0][1] = c * d1; p[0][2] = c * d2; p[0][3] = c * d3;
            p[1][0] = h; p[1][1] = -(c * d1); p[1][2] = -(c * d2); p[1][3] = -(c * d3);
            return vol_massless * xi;
        }
    }
    S e2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) e2[i] = p[i][0] * p[i][0];
    for (int it = 0; it < 100; ++it) {
        S f = -rs, fp = S(0.0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const S ei = sqrt(m[i] * m[i] + xi * xi * e2[i]);
            f = f + ei;
            fp = fp + xi * e2[i] / ei;
        }
        xi = xi - f / fp;
        if (fabs(val(f)) < 1e-15 * val(rs)) break;
    }
    if constexpr (is_dual<S>::value) {
        // one more Newton step at the converged point carries the derivative
        // of xi through the implicit-function relation sum_i E_i(xi) = rs
        S f = -rs, fp = S(0.0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const S ei = sqrt(m[i] * m[i] + xi * xi * e2[i]);
            f = f + ei;
            fp = fp + xi * e2[i] / ei;
        }
        xi = xi - f / fp;
    }
    S sk = S(0.0), sk2e = S(0.0), prod = S(1.0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const S ka = xi * p[i][0];
        const S e = sqrt(m[i] * m[i] + ka * ka);
        const S ie = 1.0 / e;
        p[i][1] = p[i][1] * xi; p[i][2] = p[i][2] * xi; p[i][3] = p[i][3] * xi;
        p[i][0] = e;
        sk = sk + ka;
        sk2e = sk2e + ka * ka * ie;
        prod = prod * (ka * ie);
    }
    S pw = S(1.0);
    const S r = sk / rs;
#pragma unroll
    for (int i = 0; i < 2 * N - 3; ++i) pw = pw * r;
    return vol_massless * pw * prod * rs / sk2e;
}

// ------------------------------------------------------------------ a7: log-bicubic PDF
// Cubic Hermite in ln x along the Q^2 rows j-1..j+2, then in ln Q^2 over those
// row values; node derivatives are central differences inside, one-sided at
// the ends (LHAPDF6 log-bicubic, EPJC 75 (2015) 132).  g: [ix][iq] x f values.
// ihx = 1 / hx, ihq = 1 / hq
struct PdfGeom { int nx, nq; double lx0, hx, lq0, lq1, hq, ihx, ihq; };

// cubic Hermite on one cell, the end tangents given as their change over the
// cell (h d): central or one-sided differences of the node values need no
// division by the spacing
template <typename A, typename B>
__device__ __forceinline__ B hermite3h(A f0, A f1, A hd0, A hd1, B t)
{
    const B t2 = t * t, t3 = t2 * t;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * f0 + (t3 - 2.0 * t2 + t) * hd0 + (-2.0 * t3 + 3.0 * t2) * f1 +
           (t3 - t2) * hd1;
}

template <typename S>
__device__ __forceinline__ S pdf_row(const double* g, const PdfGeom& G, int i, int jr, S t)
{
    const int nq = G.nq, nx = G.nx;
    const double f0 = g[i * nq + jr], f1 = g[(i + 1) * nq + jr];
    const double hd0 = i == 0 ? f1 - f0 : 0.5 * (f1 - g[(i - 1) * nq + jr]);
    const double hd1 = (i + 1 == nx - 1) ? f1 - f0 : 0.5 * (g[(i + 2) * nq + jr] - f0);
    return hermite3h(f0, f1, hd0, hd1, t);
}

// x f(x, Q^2) from lx = ln x and lq = ln Q^2; S is double or Dual<double>
// (the cells are chosen from the values)
template <typename S>
__device__ __forceinline__ S pdf_xf_log(const double* g, const PdfGeom& G, S lx, S lq)
{
    if (val(lq) < G.lq0) lq = S(G.lq0);
    if (val(lq) > G.lq1) lq = S(G.lq1);
    int i = (int)floor((val(lx) - G.lx0) * G.ihx);
    i = i < 0 ? 0 : (i > G.nx - 2 ? G.nx - 2 : i);
    int j = (int)floor((val(lq) - G.lq0) * G.ihq);
    j = j < 0 ? 0 : (j > G.nq - 2 ? G.nq - 2 : j);
    const S t = (lx - (G.lx0 + i * G.hx)) * G.ihx;
    const S s = (lq - (G.lq0 + j * G.hq)) * G.ihq;
    const S r1 = pdf_row(g, G, i, j, t);
    const S r2 = pdf_row(g, G, i, j + 1, t);
    const S r0 = j > 0 ? pdf_row(g, G, i, j - 1, t) : S(0.0);
    const S r3 = (j + 2 < G.nq) ? pdf_row(g, G, i, j + 2, t) : S(0.0);
    const S hdj = j == 0 ? r2 - r1 : 0.5 * (r2 - r0);
    const S hdj1 = (j + 1 == G.nq - 1) ? r2 - r1 : 0.5 * (r3 - r1);
    return hermite3h(r1, r2, hdj, hdj1, s);
}

}  // namespace mf

// Berends-Giele evaluation of g g -> t tbar + gluons on the GPU (the matrix
// element of Sec. 2.2 of arXiv:2105.10529 for a multi-leg process, Sec. 4).
//
// The straight-line Feynman-diagram code used for up to four gluons grows
// with the diagram count (123 diagrams for four gluons, 1240 for five); here
// one warp evaluates one event with a compact, table-driven recursion
// instead.  For a helicity configuration the warp builds, level by level,
//   * the gluon currents J(s) of every ordered gluon sequence s (one of each
//     pair of reflections: J(reverse s) = (-1)^(|s|+1) J(s)),
//   * the top-line row spinors U(s) after absorbing the ordered gluons s,
//   * the partial amplitude of every colour ordering sigma,
//       A(sigma) = sum_{sigma = (L, R)} U(L) Jslash(R) v(p_tbar),
// with the lanes spread over the currents of a level (every current of a
// level has the same number of splits, so the lanes stay in step), the
// currents in the warp's shared memory, and the index tables of
// generated/bg_*.cuh.  The colour sum sum_{sigma tau} A*_sigma C A_tau takes
// one row of the colour matrix per lane.  Helicity configurations come in
// parity pairs with equal |M|^2; the warp evaluates one of each pair.
//
// Conventions and routines are those of mf_helas.cuh (chiral basis, helicity
// eigenstates); couplings are taken out (|M|^2 carries g_s^(2k)), and the
// factors i common to every term of a partial amplitude are dropped.
// Per-event quantities (subset momenta, inverse propagator denominators,
// polarisation and spinor bases) are formed in FP64 and stored as R.
#pragma once
#include <cstdint>
#include "mf_helas.cuh"

namespace mf {

// one warp's shared-memory state for an event with K gluons (T: the table namespace)
template <typename R, int K, int NJ, int NU, int NPERM>
struct BgWarp {
    W4<R> J[NJ];          // gluon currents (the first K: the polarisations)
    W4<R> U[NU];          // top-line row spinors (U[0]: ubar(p_t))
    W4<R> V;              // v(p_tbar)
    cx<R> A[NPERM];       // partial amplitudes of the helicity being summed
    R P[1 << K][4];       // momentum of every gluon subset (incoming convention)
    R iP2[1 << K];        // 1 / P^2 (subsets of two or more gluons)
    R Q[1 << K][4];       // p_t - P
    R iQ[1 << K];         // 1 / ((p_t - P)^2 - m_t^2)
    R e1[K][3], e2[K][3]; // transverse bases of the gluons (scaled by 1/sqrt 2)
    FermionBasis<R> fb3, fb4;
    R mt;
};

template <typename R> __device__ __forceinline__ W4<R> w4_zero()
{
    W4<R> w;
    for (int m = 0; m < 4; ++m) w.c[m] = mkc(R(0), R(0));
    return w;
}
template <typename R> __device__ __forceinline__ void w4_axpy(W4<R>& y, R a, const W4<R>& x)
{
    for (int m = 0; m < 4; ++m) { y.c[m].r = fma(a, x.c[m].r, y.c[m].r); y.c[m].i = fma(a, x.c[m].i, y.c[m].i); }
}
template <typename R> __device__ __forceinline__ void w4_cxpy(W4<R>& y, cx<R> a, const W4<R>& x)
{
    for (int m = 0; m < 4; ++m) y.c[m] = cfma(a, x.c[m], y.c[m]);
}
template <typename R> __device__ __forceinline__ R ref_sign(uint16_t r) { return (r & 0x8000u) ? R(-1) : R(1); }
__device__ __forceinline__ int ref_id(uint16_t r) { return (int)(r & 0x7FFFu); }

// row spinor times Jslash: (a, b) Jslash = (b Sigmabar(J), a Sigma(J))
template <typename R> __device__ __forceinline__ W4<R> row_jslash(const W4<R>& u, const W4<R>& J)
{
    const M2<R> S = sig(J), Sb = sigbar(J);
    W4<R> o;
    rowm(u.c[2], u.c[3], Sb, o.c[0], o.c[1]);
    rowm(u.c[0], u.c[1], S, o.c[2], o.c[3]);
    return o;
}
// (a', b') (qslash + m) scaled by s: (m a' + b' Sigmabar(q), a' Sigma(q) + m b') s
template <typename R> __device__ __forceinline__ W4<R> row_qprop(const W4<R>& x, const R* q, R m, R s)
{
    cx<R> t0, t1, u0, u1;
    rowq(x.c[2], x.c[3], q, true, t0, t1);
    rowq(x.c[0], x.c[1], q, false, u0, u1);
    W4<R> o;
    o.c[0] = cscale(mkc(fma(m, x.c[0].r, t0.r), fma(m, x.c[0].i, t0.i)), s);
    o.c[1] = cscale(mkc(fma(m, x.c[1].r, t1.r), fma(m, x.c[1].i, t1.i)), s);
    o.c[2] = cscale(mkc(fma(m, x.c[2].r, u0.r), fma(m, x.c[2].i, u0.i)), s);
    o.c[3] = cscale(mkc(fma(m, x.c[3].r, u1.r), fma(m, x.c[3].i, u1.i)), s);
    return o;
}
// the four-gluon term 2 (J1.J3) J2 - (J1.J2) J3 - (J2.J3) J1, scaled by s
template <typename R> __device__ __forceinline__ void v4_add(W4<R>& acc, const W4<R>& J1, const W4<R>& J2,
                                                             const W4<R>& J3, R s)
{
    const cx<R> d13 = cscale(cdot(J1, J3), R(2) * s), d12 = cscale(cdot(J1, J2), -s), d23 = cscale(cdot(J2, J3), -s);
    w4_cxpy(acc, d13, J2);
    w4_cxpy(acc, d12, J3);
    w4_cxpy(acc, d23, J1);
}

template <typename R, typename W>
__device__ __forceinline__ W4<R> ld_w4(const W& w, const W4<R>* base, int id)
{
    return base[id];
}

// gluon current c of level M (sequences of M gluons): V3 splits, V4 splits, propagator
template <typename R, int M, int NV4, class W>
__device__ __forceinline__ void bg_gluon_current(W& w, int c, int joff, const uint8_t* mask, const uint16_t* v3,
                                                 const uint8_t* v3m, const uint16_t* v4)
{
    W4<R> acc = w4_zero<R>();
#pragma unroll
    for (int j = 0; j < M - 1; ++j) {
        const uint16_t ra = __ldg(v3 + (c * (M - 1) + j) * 2), rb = __ldg(v3 + (c * (M - 1) + j) * 2 + 1);
        const int ma = __ldg(v3m + (c * (M - 1) + j) * 2), mb = __ldg(v3m + (c * (M - 1) + j) * 2 + 1);
        const R k1[4] = { w.P[ma][0], w.P[ma][1], w.P[ma][2], w.P[ma][3] };
        const R k2[4] = { w.P[mb][0], w.P[mb][1], w.P[mb][2], w.P[mb][3] };
        // - V3, the reflection signs of both currents folded into the scale
        const W4<R> t = vvv_cur(w.J[ref_id(ra)], w.J[ref_id(rb)], k1, k2, -(ref_sign<R>(ra) * ref_sign<R>(rb)));
        for (int m = 0; m < 4; ++m) { acc.c[m].r += t.c[m].r; acc.c[m].i += t.c[m].i; }
    }
#pragma unroll
    for (int j = 0; j < NV4; ++j) {
        const uint16_t ra = __ldg(v4 + (c * NV4 + j) * 3), rb = __ldg(v4 + (c * NV4 + j) * 3 + 1);
        const uint16_t rc = __ldg(v4 + (c * NV4 + j) * 3 + 2);
        v4_add(acc, w.J[ref_id(ra)], w.J[ref_id(rb)], w.J[ref_id(rc)],
               ref_sign<R>(ra) * ref_sign<R>(rb) * ref_sign<R>(rc));
    }
    const R ip = w.iP2[__ldg(mask + c)];
    W4<R> o;
    for (int m = 0; m < 4; ++m) o.c[m] = cscale(acc.c[m], ip);
    w.J[joff + c] = o;
}

// top-line current c of level M: sum over the split points, then the propagator
template <typename R, int M, class W>
__device__ __forceinline__ void bg_top_current(W& w, int c, int uoff, const uint8_t* mask, const uint16_t* terms)
{
    W4<R> acc = w4_zero<R>();
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int ui = __ldg(terms + (c * M + j) * 2);
        const uint16_t r = __ldg(terms + (c * M + j) * 2 + 1);
        w4_axpy(acc, ref_sign<R>(r), row_jslash(w.U[ui], w.J[ref_id(r)]));
    }
    const int msk = __ldg(mask + c);
    const R q[4] = { w.Q[msk][0], w.Q[msk][1], w.Q[msk][2], w.Q[msk][3] };
    w.U[uoff + c] = row_qprop(acc, q, w.mt, -w.iQ[msk]);
}

}  // namespace mf

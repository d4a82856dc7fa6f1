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

// An array of N four-component wavefunctions in shared memory, each split into 16-byte
// chunks kept in NCH separate arrays: lanes reading different entries then fall into
// different 16-byte bank groups eight entries apart (with whole 32- or 64-byte entries, two
// or four apart), which removes most bank conflicts of the lanes' scattered reads.  Entries
// are read by value (a[i]) and written with set().
template <typename R, int N> struct W4Arr {
    static constexpr int NCH = (int)(sizeof(W4<R>) / 16);
    static_assert(NCH * 16 == (int)sizeof(W4<R>), "16-byte chunks");
    float4 ch[NCH][N];
    __device__ __forceinline__ W4<R> operator[](int i) const
    {
        W4<R> o;
        float* f = reinterpret_cast<float*>(&o);
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const float4 v = ch[k][i];
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
        return o;
    }
    __device__ __forceinline__ void set(int i, const W4<R>& v)
    {
        const float* f = reinterpret_cast<const float*>(&v);
#pragma unroll
        for (int k = 0; k < NCH; ++k) ch[k][i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    }
};

// one warp's shared-memory state for an event with K gluons (T: the table namespace)
template <typename R, int K, int NJ, int NU, int NPERM>
struct BgWarp {
    W4Arr<R, NJ> J;       // gluon currents (the first K: the polarisations)
    W4Arr<R, NU> U;       // top-line row spinors (U[0]: ubar(p_t))
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
// butterfly step of a warp sum, for plain and dual numbers
template <typename T> __device__ __forceinline__ T shfl_xor_r(T v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
template <typename T> __device__ __forceinline__ Dual<T> shfl_xor_r(const Dual<T>& v, int off)
{
    return Dual<T>(__shfl_xor_sync(0xffffffffu, v.v, off), __shfl_xor_sync(0xffffffffu, v.d, off));
}
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
    w.J.set(joff + c, o);
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
    w.U.set(uoff + c, row_qprop(acc, q, w.mt, -w.iQ[msk]));
}


// ------------------------------------------------------------------ adjoints (reverse sweep)
//
// For a complex intermediate z the adjoint is zb = dL/dRe z + i dL/dIm z, L the real
// colour- and helicity-summed |M|^2.  A holomorphic multilinear map w(x, y, ..)
// passes xb += conj(dw/dx) wb; a real parameter s of w = s z gets
// sb += Re(wb conj(z)).  Adjoints that several lanes add to (the currents of lower
// levels) are accumulated with shared-memory atomics; those of the per-event invariants
// in each lane's registers (BgInvAcc).

template <typename R, int K, int NJ, int NU>
struct BgAdj {
    W4<R> Jb[NJ];                      // adjoints of the gluon currents (helicity being summed)
    W4<R> Ub[NU];                      // adjoints of the top-line currents
    // adjoints of the polarisation and spinor pieces, summed over helicities (one lane each)
    R e1b[K][3], e2b[K][3];
    cx<R> chi3b[2][2], chi4b[2][2];
    R om3b[2], om4b[2];
};

// The adjoints of the subset invariants (P_S, 1/P_S^2, Q_S = p_t - P_S, 1/(Q_S^2 - m_t^2) and
// the propagators' m_t) pushed on at once to the external momenta and m_t, in the lane's
// registers: gp[e][c] = dL/dp_e^c and gmt = dL/dm_t through the invariants, summed over
// the lane's terms and helicities (the warp adds its lanes up once per event).  This keeps
// the many currents that share a subset from updating one shared word.
//
// The same registers hold the lane's part of the adjoints of the warp's most shared
// currents, the K external gluons (hJ) and ubar(p_t) (hU0): nearly every current and
// ordering reaches them, so they are added up over the warp once per helicity instead.
template <typename R, int K>
struct BgInvAcc {
    R gp[K + 2][4];
    R gmt;
    W4<R> hJ[K];
    W4<R> hU0;
};
template <typename R, int K> __device__ __forceinline__ void inv_acc_zero(BgInvAcc<R, K>& g)
{
#pragma unroll
    for (int e = 0; e < K + 2; ++e)
#pragma unroll
        for (int c = 0; c < 4; ++c) g.gp[e][c] = R(0);
    g.gmt = R(0);
}
template <typename R, int K> __device__ __forceinline__ void hub_zero(BgInvAcc<R, K>& g)
{
#pragma unroll
    for (int i = 0; i < K; ++i) g.hJ[i] = w4_zero<R>();
    g.hU0 = w4_zero<R>();
}
// b: the adjoint of P_S (S = msk; gluon i enters P_S with + if incoming, i < 2, else -)
template <typename R, int K> __device__ __forceinline__ void inv_acc_P(BgInvAcc<R, K>& g, int msk, const R* b)
{
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const R s = (msk >> i & 1) ? (i < 2 ? R(1) : R(-1)) : R(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) g.gp[i < 2 ? i : i + 2][c] = fma(s, b[c], g.gp[i < 2 ? i : i + 2][c]);
    }
}
// b: the adjoint of Q_S = p_t - P_S
template <typename R, int K> __device__ __forceinline__ void inv_acc_Q(BgInvAcc<R, K>& g, int msk, const R* b)
{
    R nb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { g.gp[2][c] += b[c]; nb[c] = -b[c]; }
    inv_acc_P(g, msk, nb);
}

template <typename R> __device__ __forceinline__ void atomic_add_cx(cx<R>* d, cx<R> v)
{
    atomicAdd(&d->r, v.r);
    atomicAdd(&d->i, v.i);
}
template <typename R> __device__ __forceinline__ void atomic_add_w4(W4<R>& d, const W4<R>& v)
{
    for (int m = 0; m < 4; ++m) atomic_add_cx(&d.c[m], v.c[m]);
}
template <typename R> __device__ __forceinline__ void w4_add(W4<R>& d, const W4<R>& v)
{
    for (int m = 0; m < 4; ++m) { d.c[m].r += v.c[m].r; d.c[m].i += v.c[m].i; }
}
// v summed over the warp (every lane gets the sum)
template <typename R> __device__ __forceinline__ void w4_warp_sum(W4<R>& v)
{
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v.c[m].r += __shfl_xor_sync(0xffffffffu, v.c[m].r, off);
            v.c[m].i += __shfl_xor_sync(0xffffffffu, v.c[m].i, off);
        }
}
// add v to the adjoint of gluon current id / top-line current ui: the lane's registers for
// the external gluons and ubar, a shared-memory atomic for the others
template <typename R, int K, class A>
__device__ __forceinline__ void adj_add_J(A& a, BgInvAcc<R, K>& g, int id, const W4<R>& v)
{
    if (id < K) {
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (i == id) w4_add(g.hJ[i], v);
    } else {
        atomic_add_w4(a.Jb[id], v);
    }
}
template <typename R, int K, class A>
__device__ __forceinline__ void adj_add_U(A& a, BgInvAcc<R, K>& g, int ui, const W4<R>& v)
{
    if (ui == 0) w4_add(g.hU0, v);
    else atomic_add_w4(a.Ub[ui], v);
}
template <typename R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b)   // a conj(b)
{
    return mkc(a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i);
}
template <typename R> __device__ __forceinline__ R re_mulc(cx<R> a, cx<R> b)      // Re(a conj(b))
{
    return a.r * b.r + a.i * b.i;
}
__device__ __forceinline__ float metric(int mu) { return mu == 0 ? 1.0f : -1.0f; }

// adjoint of vvv_cur(J1, J2, k1, k2, s) given ob: J1b, J2b (accumulated, per call), k1b, k2b
template <typename R>
__device__ __forceinline__ void vvv_cur_adj(const W4<R>& J1, const W4<R>& J2, const R* k1, const R* k2, R s,
                                            const W4<R>& ob, W4<R>& J1b, W4<R>& J2b, R* k1b, R* k2b)
{
    R a[4], b[4], c[4];
    for (int m = 0; m < 4; ++m) {
        a[m] = k1[m] - k2[m];
        b[m] = k1[m] + R(2) * k2[m];
        c[m] = -(R(2) * k1[m] + k2[m]);
    }
    const cx<R> j12 = cdot(J1, J2), bj1 = rdot(b, J1), cj2 = rdot(c, J2);
    cx<R> j12b = mkc(R(0), R(0)), bj1b = mkc(R(0), R(0)), cj2b = mkc(R(0), R(0));
    for (int m = 0; m < 4; ++m) {
        const cx<R> o = cscale(ob.c[m], s);
        j12b = mkc(j12b.r + o.r * a[m], j12b.i + o.i * a[m]);
        bj1b = cadd(bj1b, cmulc(o, J2.c[m]));
        cj2b = cadd(cj2b, cmulc(o, J1.c[m]));
        J2b.c[m] = cadd(J2b.c[m], cmulc(o, bj1));
        J1b.c[m] = cadd(J1b.c[m], cmulc(o, cj2));
        const R ab = re_mulc(o, j12);
        k1b[m] += ab;
        k2b[m] -= ab;
    }
    for (int m = 0; m < 4; ++m) {
        const R eta = R(metric(m));
        J1b.c[m] = cadd(J1b.c[m], cscale(cmulc(j12b, J2.c[m]), eta));
        J2b.c[m] = cadd(J2b.c[m], cscale(cmulc(j12b, J1.c[m]), eta));
        J1b.c[m] = cadd(J1b.c[m], cscale(bj1b, eta * b[m]));
        J2b.c[m] = cadd(J2b.c[m], cscale(cj2b, eta * c[m]));
        const R bb = eta * re_mulc(bj1b, J1.c[m]), cb = eta * re_mulc(cj2b, J2.c[m]);
        k1b[m] += bb - R(2) * cb;
        k2b[m] += R(2) * bb - cb;
    }
}

// adjoint of v4_add(acc, J1, J2, J3, s) given ab (the adjoint of acc)
template <typename R>
__device__ __forceinline__ void v4_adj(const W4<R>& J1, const W4<R>& J2, const W4<R>& J3, R s, const W4<R>& ab,
                                       W4<R>& J1b, W4<R>& J2b, W4<R>& J3b)
{
    const cx<R> d13 = cdot(J1, J3), d12 = cdot(J1, J2), d23 = cdot(J2, J3);
    cx<R> d13b = mkc(R(0), R(0)), d12b = mkc(R(0), R(0)), d23b = mkc(R(0), R(0));
    for (int m = 0; m < 4; ++m) {
        d13b = cadd(d13b, cscale(cmulc(ab.c[m], J2.c[m]), R(2) * s));
        d12b = cadd(d12b, cscale(cmulc(ab.c[m], J3.c[m]), -s));
        d23b = cadd(d23b, cscale(cmulc(ab.c[m], J1.c[m]), -s));
        J2b.c[m] = cadd(J2b.c[m], cscale(cmulc(ab.c[m], d13), R(2) * s));
        J3b.c[m] = cadd(J3b.c[m], cscale(cmulc(ab.c[m], d12), -s));
        J1b.c[m] = cadd(J1b.c[m], cscale(cmulc(ab.c[m], d23), -s));
    }
    for (int m = 0; m < 4; ++m) {
        const R eta = R(metric(m));
        J1b.c[m] = cadd(J1b.c[m], cscale(cadd(cmulc(d13b, J3.c[m]), cmulc(d12b, J2.c[m])), eta));
        J3b.c[m] = cadd(J3b.c[m], cscale(cadd(cmulc(d13b, J1.c[m]), cmulc(d23b, J2.c[m])), eta));
        J2b.c[m] = cadd(J2b.c[m], cscale(cadd(cmulc(d12b, J1.c[m]), cmulc(d23b, J3.c[m])), eta));
    }
}

// adjoint of o = row_jslash(u, J) given ob: ub and Jb accumulated
template <typename R>
__device__ __forceinline__ void row_jslash_adj(const W4<R>& u, const W4<R>& J, const W4<R>& ob, W4<R>& ub, W4<R>& Jb)
{
    const M2<R> S = sig(J), Sb = sigbar(J);
    // o_left = u_right Sigmabar, o_right = u_left Sigma (row times matrix, o_c = sum_r u_r M_rc)
    ub.c[2] = cadd(ub.c[2], cadd(cmulc(ob.c[0], Sb.m00), cmulc(ob.c[1], Sb.m01)));
    ub.c[3] = cadd(ub.c[3], cadd(cmulc(ob.c[0], Sb.m10), cmulc(ob.c[1], Sb.m11)));
    ub.c[0] = cadd(ub.c[0], cadd(cmulc(ob.c[2], S.m00), cmulc(ob.c[3], S.m01)));
    ub.c[1] = cadd(ub.c[1], cadd(cmulc(ob.c[2], S.m10), cmulc(ob.c[3], S.m11)));
    // adjoints of the matrix entries
    const cx<R> bb00 = cmulc(ob.c[0], u.c[2]), bb01 = cmulc(ob.c[1], u.c[2]);
    const cx<R> bb10 = cmulc(ob.c[0], u.c[3]), bb11 = cmulc(ob.c[1], u.c[3]);
    const cx<R> ss00 = cmulc(ob.c[2], u.c[0]), ss01 = cmulc(ob.c[3], u.c[0]);
    const cx<R> ss10 = cmulc(ob.c[2], u.c[1]), ss11 = cmulc(ob.c[3], u.c[1]);
    // Sigma: m00 = J0 - J3, m11 = J0 + J3, m01 = -J1 + i J2, m10 = -J1 - i J2;
    // Sigmabar: m00 = J0 + J3, m11 = J0 - J3, m01 = J1 - i J2, m10 = J1 + i J2
    Jb.c[0] = cadd(Jb.c[0], cadd(cadd(ss00, ss11), cadd(bb00, bb11)));
    Jb.c[3] = cadd(Jb.c[3], cadd(csub(ss11, ss00), csub(bb00, bb11)));
    Jb.c[1] = cadd(Jb.c[1], csub(cadd(bb01, bb10), cadd(ss01, ss10)));
    // J2: conj(i) ss01 + conj(-i) ss10 + conj(-i) bb01 + conj(i) bb10 = -i (ss01 - ss10 - bb01 + bb10)
    const cx<R> t = cadd(csub(ss01, ss10), csub(bb10, bb01));
    Jb.c[2] = cadd(Jb.c[2], mkc(t.i, -t.r));
}

// adjoint of o = row_qprop(x, q, m, s) given ob: xb (accumulated), qb, mb, sb
template <typename R>
__device__ __forceinline__ void row_qprop_adj(const W4<R>& x, const R* q, R m, R s, const W4<R>& ob, W4<R>& xb,
                                              R* qb, R& mb, R& sb)
{
    // inner = o / s: (m x_left + x_right Sb_q, x_left S_q + m x_right); Sb_q = q0 + q.sigma, S_q = q0 - q.sigma
    const W4<R> inner = row_qprop(x, q, m, R(1));
    for (int c = 0; c < 4; ++c) sb += re_mulc(ob.c[c], inner.c[c]);
    W4<R> o;
    for (int c = 0; c < 4; ++c) o.c[c] = cscale(ob.c[c], s);
    // matrices as [[M00, M01], [M10, M11]] with row-vector products y_c = sum_r x_r M_rc
    const cx<R> Sb00 = mkc(q[0] + q[3], R(0)), Sb11 = mkc(q[0] - q[3], R(0));
    const cx<R> Sb01 = mkc(q[1], -q[2]), Sb10 = mkc(q[1], q[2]);
    const cx<R> S00 = mkc(q[0] - q[3], R(0)), S11 = mkc(q[0] + q[3], R(0));
    const cx<R> S01 = mkc(-q[1], q[2]), S10 = mkc(-q[1], -q[2]);
    // x_left: m o_left + o_right S_q^dagger rows; x_right: o_left Sb_q^dagger rows + m o_right
    xb.c[0] = cadd(xb.c[0], cadd(cscale(o.c[0], m), cadd(cmulc(o.c[2], S00), cmulc(o.c[3], S01))));
    xb.c[1] = cadd(xb.c[1], cadd(cscale(o.c[1], m), cadd(cmulc(o.c[2], S10), cmulc(o.c[3], S11))));
    xb.c[2] = cadd(xb.c[2], cadd(cadd(cmulc(o.c[0], Sb00), cmulc(o.c[1], Sb01)), cscale(o.c[2], m)));
    xb.c[3] = cadd(xb.c[3], cadd(cadd(cmulc(o.c[0], Sb10), cmulc(o.c[1], Sb11)), cscale(o.c[3], m)));
    for (int c = 0; c < 4; ++c) mb += re_mulc(o.c[c], x.c[c]);
    // entry adjoints: Sb_rc from o_left_c and x_right_r, S_rc from o_right_c and x_left_r
    const cx<R> b00 = cmulc(o.c[0], x.c[2]), b01 = cmulc(o.c[1], x.c[2]), b10 = cmulc(o.c[0], x.c[3]), b11 = cmulc(o.c[1], x.c[3]);
    const cx<R> a00 = cmulc(o.c[2], x.c[0]), a01 = cmulc(o.c[3], x.c[0]), a10 = cmulc(o.c[2], x.c[1]), a11 = cmulc(o.c[3], x.c[1]);
    // dq for a real q: Re(entry adjoint * conj(d entry / dq))
    qb[0] += b00.r + b11.r + a00.r + a11.r;
    qb[3] += b00.r - b11.r - a00.r + a11.r;
    qb[1] += b01.r + b10.r - a01.r - a10.r;
    qb[2] += -b01.i + b10.i + a01.i - a10.i;
}

// reverse of gluon current c of level M (its adjoint a.Jb[joff + c] complete)
template <typename R, int M, int NV4, class W, class A, class I>
__device__ __forceinline__ void bg_gluon_current_adj(const W& w, A& a, I& gi, int c, int joff, const uint8_t* mask,
                                                     const uint16_t* v3, const uint8_t* v3m, const uint16_t* v4)
{
    const int msk = __ldg(mask + c);
    const W4<R> Jo = w.J[joff + c], Jb = a.Jb[joff + c];
    const R ip = w.iP2[msk];
    // J = ip acc: accb = ip Jb; ipb = Re sum Jb conj(acc) = Re sum Jb conj(J) / ip
    W4<R> accb;
    R ipb = R(0);
    for (int m = 0; m < 4; ++m) { accb.c[m] = cscale(Jb.c[m], ip); ipb += re_mulc(Jb.c[m], Jo.c[m]); }
    {
        // d(1/P^2) = -2 (P.dP) / P^4: the adjoint of P from that of 1/P^2 (ipb / ip)
        const R f = R(-2) * (ipb / ip) * ip * ip;
        R pb[4];
        for (int m = 0; m < 4; ++m) pb[m] = f * R(metric(m)) * w.P[msk][m];
        inv_acc_P(gi, msk, pb);
    }
#pragma unroll
    for (int j = 0; j < M - 1; ++j) {
        const uint16_t ra = __ldg(v3 + (c * (M - 1) + j) * 2), rb = __ldg(v3 + (c * (M - 1) + j) * 2 + 1);
        const int ma = __ldg(v3m + (c * (M - 1) + j) * 2), mb = __ldg(v3m + (c * (M - 1) + j) * 2 + 1);
        const R k1[4] = { w.P[ma][0], w.P[ma][1], w.P[ma][2], w.P[ma][3] };
        const R k2[4] = { w.P[mb][0], w.P[mb][1], w.P[mb][2], w.P[mb][3] };
        W4<R> J1b = w4_zero<R>(), J2b = w4_zero<R>();
        R k1b[4] = { R(0), R(0), R(0), R(0) }, k2b[4] = { R(0), R(0), R(0), R(0) };
        vvv_cur_adj(w.J[ref_id(ra)], w.J[ref_id(rb)], k1, k2, -(ref_sign<R>(ra) * ref_sign<R>(rb)), accb, J1b, J2b,
                    k1b, k2b);
        adj_add_J(a, gi, ref_id(ra), J1b);
        adj_add_J(a, gi, ref_id(rb), J2b);
        inv_acc_P(gi, ma, k1b);
        inv_acc_P(gi, mb, k2b);
    }
#pragma unroll
    for (int j = 0; j < NV4; ++j) {
        const uint16_t ra = __ldg(v4 + (c * NV4 + j) * 3), rb = __ldg(v4 + (c * NV4 + j) * 3 + 1);
        const uint16_t rc = __ldg(v4 + (c * NV4 + j) * 3 + 2);
        W4<R> J1b = w4_zero<R>(), J2b = w4_zero<R>(), J3b = w4_zero<R>();
        v4_adj(w.J[ref_id(ra)], w.J[ref_id(rb)], w.J[ref_id(rc)], ref_sign<R>(ra) * ref_sign<R>(rb) * ref_sign<R>(rc),
               accb, J1b, J2b, J3b);
        adj_add_J(a, gi, ref_id(ra), J1b);
        adj_add_J(a, gi, ref_id(rb), J2b);
        adj_add_J(a, gi, ref_id(rc), J3b);
    }
}

// reverse of top-line current c of level M (its adjoint a.Ub[uoff + c] complete); the
// sum before the propagator is recomputed from the stored currents
template <typename R, int M, class W, class A, class I>
__device__ __forceinline__ void bg_top_current_adj(const W& w, A& a, I& gi, int c, int uoff, const uint8_t* mask,
                                                   const uint16_t* terms)
{
    W4<R> x = w4_zero<R>();
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int ui = __ldg(terms + (c * M + j) * 2);
        const uint16_t r = __ldg(terms + (c * M + j) * 2 + 1);
        w4_axpy(x, ref_sign<R>(r), row_jslash(w.U[ui], w.J[ref_id(r)]));
    }
    const int msk = __ldg(mask + c);
    const R q[4] = { w.Q[msk][0], w.Q[msk][1], w.Q[msk][2], w.Q[msk][3] };
    const R s = -w.iQ[msk];
    W4<R> xb = w4_zero<R>();
    R qb[4] = { R(0), R(0), R(0), R(0) }, mb = R(0), sb = R(0);
    row_qprop_adj(x, q, w.mt, s, a.Ub[uoff + c], xb, qb, mb, sb);
    {
        // s = -1/(Q^2 - m^2): d(1/(Q^2 - m^2)) = -2 (Q.dQ - m dm) / (Q^2 - m^2)^2
        const R iq = w.iQ[msk], f = R(-2) * (-sb) * iq * iq;
        for (int m = 0; m < 4; ++m) qb[m] += f * R(metric(m)) * q[m];
        inv_acc_Q(gi, msk, qb);
        gi.gmt += mb - f * w.mt;
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int ui = __ldg(terms + (c * M + j) * 2);
        const uint16_t r = __ldg(terms + (c * M + j) * 2 + 1);
        W4<R> ob;
        const R sg = ref_sign<R>(r);
        for (int m = 0; m < 4; ++m) ob.c[m] = cscale(xb.c[m], sg);
        W4<R> ub = w4_zero<R>(), Jb = w4_zero<R>();
        row_jslash_adj(w.U[ui], w.J[ref_id(r)], ob, ub, Jb);
        adj_add_U(a, gi, ui, ub);
        adj_add_J(a, gi, ref_id(r), Jb);
    }
}


// ------------------------------------------------------------------ one event, one warp

// The per-event invariants (FP64 arithmetic, stored as R) of the K gluons (incoming
// convention: gluons 0 and 1 incoming, the rest outgoing with minus their momenta), the
// top and the antitop: subset momenta and inverse denominators, one subset per lane,
// polarisation and spinor bases.  Particle order of p: g, g, t, tbar, g, ...
//
// S: the momenta's scalar, double, or Dual<double> for a forward-mode derivative (the
// invariants of R = Dual<float> or Dual<double> then carry their tangents).
template <int K, typename R, class W, typename S>
__device__ __forceinline__ void bg_event_invariants(W& w, const S (&p)[K + 2][4], S mt, int lane)
{
    const int msk = lane;
    if (msk >= 1 && msk < (1 << K)) {
        S P[4] = { S(0.0), S(0.0), S(0.0), S(0.0) };
        for (int i = 0; i < K; ++i)
            if (msk >> i & 1) {
                const int e = i < 2 ? i : i + 2;
                const double sg = i < 2 ? 1.0 : -1.0;
                for (int c = 0; c < 4; ++c) P[c] += sg * p[e][c];
            }
        S q[4];
        for (int c = 0; c < 4; ++c) { w.P[msk][c] = R(P[c]); q[c] = p[2][c] - P[c]; w.Q[msk][c] = R(q[c]); }
        w.iP2[msk] = __popc(msk) >= 2 ? R(1.0 / mdot(P, P)) : R(0);
        // every gluon absorbed leaves q = -p_tbar, on its mass shell: no propagator there
        w.iQ[msk] = msk != (1 << K) - 1 ? R(1.0 / (mdot(q, q) - mt * mt)) : R(0);
    }
    if (lane < K) {
        S a[3], b[3];
        gluon_basis(p[lane < 2 ? lane : lane + 2], a, b);
        for (int j = 0; j < 3; ++j) { w.e1[lane][j] = R(a[j]); w.e2[lane][j] = R(b[j]); }
    }
    if (lane == K) w.fb3 = fermion_basis<R>(p[2], mt);
    if (lane == K + 1) w.fb4 = fermion_basis<R>(p[3], mt);
    if (lane == K + 2) w.mt = R(mt);
}

// external states of helicity configuration ih (bit i: helicity of external particle i)
template <int K, typename R, class W>
__device__ __forceinline__ void bg_external_states(W& w, int ih, int lane)
{
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
    if (lane < K) w.J.set(lane, ext_gluon(w.e1[lane], w.e2[lane], HEL(lane < 2 ? lane : lane + 2), lane >= 2));
    else if (lane == K) w.U.set(0, ext_ubar(w.fb3, HEL(2)));
    else if (lane == K + 1) w.V = ext_v(w.fb4, HEL(3));
#undef HEL
}

// partial amplitudes: the top line closed on v(p_tbar), lanes over the orderings
template <class G, typename R, class W>
__device__ __forceinline__ void bg_closures(W& w, int lane)
{
    const uint16_t* cl = G::closure();
    for (int s = lane; s < G::NPERM; s += 32) {
        cx<R> a = mkc(R(0), R(0));
#pragma unroll
        for (int j = 0; j < G::K; ++j) {
            const int ui = __ldg(cl + (s * G::K + j) * 2);
            const uint16_t r = __ldg(cl + (s * G::K + j) * 2 + 1);
            const cx<R> t = ffv_amp(w.U[ui], w.V, w.J[ref_id(r)]);
            const R sg = ref_sign<R>(r);
            a.r = fma(sg, t.r, a.r);
            a.i = fma(sg, t.i, a.i);
        }
        w.A[s] = a;
    }
}

// the colour sum of the helicity: every lane's rows sigma = lane, lane + 32, ... of
// sum_tau C A_tau (C scaled to integers, rows CROW floats apart in shared memory); with
// yout the rows' complex sums are kept (the adjoint of the partial amplitudes is 2 y).
// Returns the warp's sum (all lanes).
template <class G, typename R, class W>
__device__ __forceinline__ R bg_colour_sum(W& w, const float* cs, int crow, int lane, cx<R>* yout)
{
    R part = R(0);
    for (int s = lane; s < G::NPERM; s += 32) {
        const float* row = cs + s * crow;
        R yr = R(0), yi = R(0);
#pragma unroll 8
        for (int t = 0; t < G::NPERM; ++t) {
            const R c = R(row[t]);
            yr = fma(c, w.A[t].r, yr);
            yi = fma(c, w.A[t].i, yi);
        }
        part = fma(w.A[s].r, yr, fma(w.A[s].i, yi, part));
        if (yout) yout[s] = mkc(yr, yi);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += shfl_xor_r(part, off);
    return part;
}

// The same colour sum from the upper triangle of the symmetric C:
//   sum_{s t} A*_s C_st A_t = sum_s Re A*_s (C_ss A_s + 2 sum_{t > s} C_st A_t),
// half the multiply-adds.  The rows are paired as (s, N - 1 - s), so every lane walks N - 1
// entries of the triangle in one loop (the two rows one after the other).
template <class G, typename R, class W>
__device__ __forceinline__ R bg_colour_sum_sym(W& w, const float* cs, int crow, int lane)
{
    constexpr int N = G::NPERM, NPAIR = (N + 1) / 2;
    R part = R(0);
    // Re A*_s (C_ss A_s + 2 y) for row s with its upper-triangle sum y
    auto row_term = [&](int sr, R yr, R yi) {
        const R d = R(cs[sr * crow + sr]);
        part = fma(w.A[sr].r, fma(d, w.A[sr].r, R(2) * yr), fma(w.A[sr].i, fma(d, w.A[sr].i, R(2) * yi), part));
    };
    for (int pr = lane; pr < NPAIR; pr += 32) {
        const int s1 = pr, s2 = N - 1 - pr;
        const int n1 = N - 1 - s1;                       // entries right of the diagonal in row s1
        const int len = s2 > s1 ? N - 1 : n1;            // both rows, or the middle row of an odd N
        R yr = R(0), yi = R(0);
        int srow = s1, t = s1 + 1;
        for (int k = 0; k < len; ++k) {
            if (k == n1) {                               // row s1 done: its term, then row s2
                row_term(srow, yr, yi);
                yr = R(0); yi = R(0);
                srow = s2; t = s2 + 1;
            }
            const R c = R(cs[srow * crow + t]);
            yr = fma(c, w.A[t].r, yr);
            yi = fma(c, w.A[t].i, yi);
            ++t;
        }
        row_term(srow, yr, yi);
        if (s2 > s1 && srow == s1) row_term(s2, R(0), R(0));   // row N - 1: the diagonal alone
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += shfl_xor_r(part, off);
    return part;
}

// Sum over helicities of sum_{sigma tau} A*_sigma C_{sigma tau} A_tau / COLOUR_DEN for one
// event, by the whole warp (couplings and averages not applied).  pev: the event's FP64
// momenta, component 4 i + c of particle i at pev[(4 i + c) stride].  all_hel: every
// configuration (else one of each parity pair, doubled); hel_out (nullable, all_hel):
// each configuration's value times hel_scale, written by lane 0.
//
// Helicity sampling (nsamp > 0, a power of two dividing NHEL / 2): instead of every
// configuration of the parity-halved sum, the warp evaluates nsamp of them, one drawn
// uniformly from each of nsamp strata of NHEL / (2 nsamp) consecutive configurations with the
// bits of rnd (four random words of the event), each weighted by the stratum size: an
// unbiased estimate of the helicity sum (nsamp = NHEL / 2 is the full sum itself).
template <class G, typename R, class W>
__device__ double bg_warp_me2(W& w, const float* cs, int crow, const double* pev, int stride, double mt, bool all_hel,
                              double* hel_out, double hel_scale, int nsamp = 0, uint4 rnd = uint4{ 0u, 0u, 0u, 0u })
{
    constexpr int K = G::K, NEXT = K + 2, NHEL = 1 << NEXT, HALF = NHEL / 2;
    const int lane = threadIdx.x & 31;
    double p[NEXT][4];
    for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = pev[(size_t)f * stride];
    bg_event_invariants<K, R>(w, p, mt, lane);
    __syncwarp();
    R total = R(0);
    const bool sample = nsamp > 0 && !all_hel;
    const int h0 = all_hel ? 0 : 1, hstep = all_hel ? 1 : 2;
    const int nloop = sample ? nsamp : (all_hel ? NHEL : HALF);
    const int ssize = sample ? HALF / nsamp : 1;          // configurations per stratum
    const int sbits = sample ? __ffs(ssize) - 1 : 0;      // random bits per draw
#pragma unroll 1
    for (int it = 0; it < nloop; ++it) {
        int ih;
        if (sample) {
            // draw it: bits [it sbits, (it + 1) sbits) of the 128 random bits
            const int b0 = it * sbits;
            const uint32_t wd = b0 < 32 ? rnd.x : (b0 < 64 ? rnd.y : (b0 < 96 ? rnd.z : rnd.w));
            const int r = sbits ? (int)((wd >> (b0 & 31)) & ((1u << sbits) - 1u)) : 0;
            ih = 1 + 2 * (it * ssize + r);
        } else {
            ih = h0 + hstep * it;
        }
        bg_external_states<K, R>(w, ih, lane);
        __syncwarp();
        G::template forward<R>(w, lane);
        bg_closures<G, R>(w, lane);
        __syncwarp();
        const R part = bg_colour_sum_sym<G, R>(w, cs, crow, lane);
        if (hel_out && lane == 0) hel_out[ih] = double(part) * hel_scale;
        total += part;
        __syncwarp();
    }
    return double(total) * (all_hel ? 1.0 : 2.0) * double(ssize) / G::COLOUR_DEN;
}

// One directional derivative of bg_warp_me2's parity-halved sum by forward mode: the whole
// recursion in dual numbers D = Dual<R> (value and tangent of every current, closure and
// colour sum), the FP64 momenta pev seeded with the tangents dev (same layout) and m_t with
// dmt.  One pass per helicity, nothing stored, no reverse sweep: the cheap way to a single
// direction (the m_t derivative of a pass); the full gradient takes bg_warp_grad.  w: the
// warp's state in dual numbers.  Returns the value (as bg_warp_me2) and writes the
// derivative to *dout (every lane).
template <class G, typename R, class W>
__device__ double bg_warp_me2_dir(W& w, const float* cs, int crow, const double* pev, const double* dev, int stride,
                                  double mt, double dmt, double* dout)
{
    constexpr int K = G::K, NEXT = K + 2, NHEL = 1 << NEXT;
    using D = Dual<R>;
    using S = Dual<double>;
    const int lane = threadIdx.x & 31;
    S p[NEXT][4];
    for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = S(pev[(size_t)f * stride], dev[(size_t)f * stride]);
    bg_event_invariants<K, D>(w, p, S(mt, dmt), lane);
    __syncwarp();
    D total = D(0);
#pragma unroll 1
    for (int ih = 1; ih < NHEL; ih += 2) {
        bg_external_states<K, D>(w, ih, lane);
        __syncwarp();
        G::template forward<D>(w, lane);
        bg_closures<G, D>(w, lane);
        __syncwarp();
        total += bg_colour_sum_sym<G, D>(w, cs, crow, lane);
        __syncwarp();
    }
    *dout = double(total.d) * 2.0 / G::COLOUR_DEN;
    return double(total.v) * 2.0 / G::COLOUR_DEN;
}


// The value of bg_warp_me2 (parity-halved helicity sum, doubled) and its derivatives by a
// reverse sweep.  For every helicity the warp recomputes the currents forward (nothing is
// kept from one helicity to the next), seeds the adjoints of the partial amplitudes with
// the colour sum (dL/dA*_sigma = 2 sum_tau C A_tau, doubled for the parity mirror), and
// runs the closures, the recursion levels and the external states backwards, summing the
// adjoints of the per-event invariants over helicities.  Then lane j < 4 (K + 2) carries
// the tangent of momentum component j (and, with dir, lane 4 (K + 2) the tangent along
// dir[0 .. 4 (K + 2) - 1] for the momenta and dir[4 (K + 2)] for m_t) through the
// invariants' FP64 arithmetic and contracts it with their adjoints: dout[j] (lane j) is
// the derivative of the returned value along that direction, the momentum components
// taken as independent variables of this formula.  a: the warp's adjoint state.
template <class G, typename R, class W, class A>
__device__ double bg_warp_grad(W& w, A& a, const float* cs, int crow, const double* pev, int stride, double mt,
                               double* dout, const double* dir, bool only_dir = false)
{
    constexpr int K = G::K, NEXT = K + 2, NHEL = 1 << NEXT, NM = 1 << K;
    constexpr int ROWS = (G::NPERM + 31) / 32;
    using D = Dual<double>;
    const int lane = threadIdx.x & 31;
    double p[NEXT][4];
    for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = pev[(size_t)f * stride];
    bg_event_invariants<K, R>(w, p, mt, lane);
    // the invariants' adjoints start at zero (registers), and those of the bases (shared)
    BgInvAcc<R, K> gi;
    inv_acc_zero(gi);
    if (lane < K)
        for (int j = 0; j < 3; ++j) { a.e1b[lane][j] = R(0); a.e2b[lane][j] = R(0); }
    if (lane == K) {
        for (int x = 0; x < 4; ++x) { a.chi3b[x >> 1][x & 1] = mkc(R(0), R(0)); a.chi4b[x >> 1][x & 1] = mkc(R(0), R(0)); }
        a.om3b[0] = a.om3b[1] = a.om4b[0] = a.om4b[1] = R(0);
    }
    __syncwarp();
    R total = R(0);
#pragma unroll 1
    for (int ih = 1; ih < NHEL; ih += 2) {
        bg_external_states<K, R>(w, ih, lane);
        for (int i = lane; i < G::NJ; i += 32) a.Jb[i] = w4_zero<R>();
        for (int i = lane; i < G::NU; i += 32) a.Ub[i] = w4_zero<R>();
        hub_zero(gi);
        __syncwarp();
        G::template forward<R>(w, lane);
        bg_closures<G, R>(w, lane);
        __syncwarp();
        cx<R> y[ROWS];
        R part = R(0);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int sg = lane + 32 * r;
            if (sg < G::NPERM) {
                const float* row = cs + sg * crow;
                R yr = R(0), yi = R(0);
                for (int t = 0; t < G::NPERM; ++t) {
                    const R c = R(row[t]);
                    yr = fma(c, w.A[t].r, yr);
                    yi = fma(c, w.A[t].i, yi);
                }
                part = fma(w.A[sg].r, yr, fma(w.A[sg].i, yi, part));
                y[r] = mkc(yr, yi);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        total += part;
        __syncwarp();
        // the partial amplitudes' adjoints replace them: 2 (C A)_sigma, times 2 for the parity mirror
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int sg = lane + 32 * r;
            if (sg < G::NPERM) w.A[sg] = cscale(y[r], R(4));
        }
        __syncwarp();
        // closures backwards: A_sigma = sum_j sg_j (U_j Jslash_j) . v
        W4<R> vb = w4_zero<R>();      // the lane's part of v's adjoint
        {
            const uint16_t* cl = G::closure();
            for (int sgm = lane; sgm < G::NPERM; sgm += 32) {
                const cx<R> ab = w.A[sgm];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int ui = __ldg(cl + (sgm * K + j) * 2);
                    const uint16_t r = __ldg(cl + (sgm * K + j) * 2 + 1);
                    const R sgn = ref_sign<R>(r);
                    const W4<R> t = row_jslash(w.U[ui], w.J[ref_id(r)]);
                    W4<R> tb;
                    for (int c = 0; c < 4; ++c) {
                        vb.c[c] = cadd(vb.c[c], cscale(cmulc(ab, t.c[c]), sgn));
                        tb.c[c] = cscale(cmulc(ab, w.V.c[c]), sgn);
                    }
                    W4<R> ub = w4_zero<R>(), jb = w4_zero<R>();
                    row_jslash_adj(w.U[ui], w.J[ref_id(r)], tb, ub, jb);
                    adj_add_U(a, gi, ui, ub);
                    adj_add_J(a, gi, ref_id(r), jb);
                }
            }
        }
        __syncwarp();
        G::template reverse<R>(w, a, gi, lane);
        // the register-held adjoints of v, ubar and the external gluons summed over the warp
        w4_warp_sum(vb);
        w4_warp_sum(gi.hU0);
#pragma unroll
        for (int i = 0; i < K; ++i) w4_warp_sum(gi.hJ[i]);
        W4<R> jb_ext = gi.hJ[0];
#pragma unroll
        for (int i = 1; i < K; ++i)
            if (i == lane) jb_ext = gi.hJ[i];
        // external states backwards into the polarisation and spinor pieces (one lane each)
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
        if (lane < K) {
            const R l = HEL(lane < 2 ? lane : lane + 2) > 0 ? R(1) : R(-1), so = lane >= 2 ? R(1) : R(-1);
            for (int j = 0; j < 3; ++j) {
                a.e1b[lane][j] += -l * jb_ext.c[j + 1].r;
                a.e2b[lane][j] += so * jb_ext.c[j + 1].i;
            }
        } else if (lane == K) {
            // ubar = (conj(chi_l) om_l, conj(chi_l) om_-l)
            const int l = HEL(2) > 0 ? 0 : 1;
            const W4<R>& ub = gi.hU0;
            const R wl = w.fb3.om[l], wml = w.fb3.om[1 - l];
            for (int b = 0; b < 2; ++b) {
                a.chi3b[l][b] = cadd(a.chi3b[l][b], cadd(cscale(conjc(ub.c[b]), wl), cscale(conjc(ub.c[2 + b]), wml)));
                a.om3b[l] += ub.c[b].r * w.fb3.chi[l][b].r - ub.c[b].i * w.fb3.chi[l][b].i;
                a.om3b[1 - l] += ub.c[2 + b].r * w.fb3.chi[l][b].r - ub.c[2 + b].i * w.fb3.chi[l][b].i;
            }
        } else if (lane == K + 1) {
            // v = (chi_-l (-s om_l), chi_-l (s om_-l))
            const int l = HEL(3) > 0 ? 0 : 1;
            const R sl = HEL(3) > 0 ? R(1) : R(-1);
            const R wl = w.fb4.om[l], wml = w.fb4.om[1 - l];
            for (int b = 0; b < 2; ++b) {
                a.chi4b[1 - l][b] = cadd(a.chi4b[1 - l][b], cadd(cscale(vb.c[b], -sl * wl), cscale(vb.c[2 + b], sl * wml)));
                a.om4b[l] += -sl * re_mulc(vb.c[b], w.fb4.chi[1 - l][b]);
                a.om4b[1 - l] += sl * re_mulc(vb.c[2 + b], w.fb4.chi[1 - l][b]);
            }
        }
#undef HEL
        __syncwarp();
    }
    // the lanes' invariant adjoints added up (every lane gets the sums)
#pragma unroll
    for (int f = 0; f < NEXT * 4; ++f)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) gi.gp[f >> 2][f & 3] += __shfl_xor_sync(0xffffffffu, gi.gp[f >> 2][f & 3], off);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gi.gmt += __shfl_xor_sync(0xffffffffu, gi.gmt, off);
    // tangents through the invariants (only_dir: lane 0 carries dir alone)
    const int nd = only_dir ? 1 : NEXT * 4 + (dir ? 1 : 0);
    if (lane < nd && dout) {
        const int td = only_dir ? NEXT * 4 : lane;   // the direction this lane carries
        D pd[NEXT][4];
        D mtd(mt, 0.0);
        for (int i = 0; i < NEXT; ++i)
            for (int c = 0; c < 4; ++c)
                pd[i][c] = D(p[i][c], td < NEXT * 4 ? ((4 * i + c) == td ? 1.0 : 0.0) : dir[4 * i + c]);
        if (td == NEXT * 4) mtd = D(mt, dir[NEXT * 4]);
        double g = 0.0;
        {
            // through the subset invariants and the propagators' mass: the adjoints gp, gmt
            // (working precision R) contracted with the direction
            R gr = R(0);
#pragma unroll
            for (int f = 0; f < NEXT * 4; ++f) gr = fma(gi.gp[f >> 2][f & 3], R(pd[f >> 2][f & 3].d), gr);
            gr = fma(gi.gmt, R(mtd.d), gr);
            g = double(gr);
        }
        for (int gl = 0; gl < K; ++gl) {
            // parallel-transported basis tangent: de = -(e . dn) n (see gluon_basis)
            const D* q = pd[gl < 2 ? gl : gl + 2];
            const double pa = sqrt(q[1].v * q[1].v + q[2].v * q[2].v + q[3].v * q[3].v);
            const double n[3] = { q[1].v / pa, q[2].v / pa, q[3].v / pa };
            const double ndp = n[0] * q[1].d + n[1] * q[2].d + n[2] * q[3].d;
            const double dn[3] = { (q[1].d - n[0] * ndp) / pa, (q[2].d - n[1] * ndp) / pa, (q[3].d - n[2] * ndp) / pa };
            double c1 = 0.0, c2 = 0.0, b1 = 0.0, b2 = 0.0;
            for (int j = 0; j < 3; ++j) {
                c1 += double(w.e1[gl][j]) * dn[j];
                c2 += double(w.e2[gl][j]) * dn[j];
                b1 += n[j] * double(a.e1b[gl][j]);
                b2 += n[j] * double(a.e2b[gl][j]);
            }
            g -= c1 * b1 + c2 * b2;
        }
        {
            const FermionBasis<D> f3 = fermion_basis<D>(pd[2], mtd), f4 = fermion_basis<D>(pd[3], mtd);
            for (int x = 0; x < 2; ++x)
                for (int b = 0; b < 2; ++b) {
                    g += f3.chi[x][b].r.d * double(a.chi3b[x][b].r) + f3.chi[x][b].i.d * double(a.chi3b[x][b].i);
                    g += f4.chi[x][b].r.d * double(a.chi4b[x][b].r) + f4.chi[x][b].i.d * double(a.chi4b[x][b].i);
                }
            for (int x = 0; x < 2; ++x) g += f3.om[x].d * double(a.om3b[x]) + f4.om[x].d * double(a.om4b[x]);
        }
        dout[lane] = g / G::COLOUR_DEN;
    }
    return double(total) * 2.0 / G::COLOUR_DEN;
}

// state of a warp for one forward-mode direction (bg_warp_me2_dir)
template <class G, typename R>
using BgDirWarp = BgWarp<Dual<R>, G::K, G::NJ, G::NU, G::NPERM>;

// state of a warp for the derivative: forward currents and their adjoints
template <class G, typename R>
struct BgGradWarp {
    BgWarp<R, G::K, G::NJ, G::NU, G::NPERM> w;
    BgAdj<R, G::K, G::NJ, G::NU> a;
};

// mf_evaluate with derivatives for a gluon process of the recursion: one warp per point,
// WARPS warps per CTA; the colour matrix and the warps' states in dynamic shared memory.
// me2 [n] and dme2 [n][K + 2][4]: averaged |M|^2 (norm: couplings, averages, symmetry)
// and its derivatives with respect to every momentum component
template <class G, typename R>
__global__ void __launch_bounds__(128) bg_evaluate_grad_kernel(const double* __restrict__ mom, long long n,
                                                               double* __restrict__ me2, double* __restrict__ dme2,
                                                               double mt, double norm)
{
    constexpr int NEXT = G::K + 2, CROW = G::NPERM + 1;
    extern __shared__ __align__(128) unsigned char mf_bgg_smem[];
    float* cs = reinterpret_cast<float*>(mf_bgg_smem);
    for (int i = threadIdx.x; i < G::NPERM * G::NPERM; i += blockDim.x)
        cs[(i / G::NPERM) * CROW + i % G::NPERM] = __ldg(G::colour() + i);
    __syncthreads();
    const size_t cbytes = ((sizeof(float) * G::NPERM * CROW) + 127) & ~(size_t)127;
    const size_t wbytes = (sizeof(BgGradWarp<G, R>) + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    auto& st = *reinterpret_cast<BgGradWarp<G, R>*>(mf_bgg_smem + cbytes + warp * wbytes);
    for (long long e = (long long)blockIdx.x * nw + warp; e < n; e += (long long)gridDim.x * nw) {
        double dbuf[32];   // lane j keeps the derivative along component j
        const double v = bg_warp_grad<G, R>(st.w, st.a, cs, CROW, mom + e * NEXT * 4, 1, mt, dbuf, nullptr);
        if (lane < NEXT * 4 && dme2) dme2[e * NEXT * 4 + lane] = dbuf[lane] * norm;
        if (lane == 0 && me2) me2[e] = v * norm;
    }
}

template <class G, typename R>
constexpr size_t bg_grad_smem_bytes(int warps)
{
    return (((sizeof(float) * G::NPERM * (G::NPERM + 1)) + 127) & ~(size_t)127) +
           (size_t)warps * ((sizeof(BgGradWarp<G, R>) + 15) & ~(size_t)15);
}
template <class G, typename R>
inline size_t bg_grad_smem(int warps) { return bg_grad_smem_bytes<G, R>(warps); }


// host launcher of bg_evaluate_grad_kernel for a gluon process with tables G and
// symmetry factor 1/SYM_DEN: |M|^2 averaged over the initial spins and colours (1/256)
// largest number of warps (1 .. 4) whose states and the colour matrix fit 227 KB of shared memory
template <class G, typename R>
constexpr int bg_grad_warps()
{
    constexpr size_t cap = 227 * 1024;
    int w = 4;
    while (w > 1 && bg_grad_smem_bytes<G, R>(w) > cap) --w;
    return w;
}

template <class G, int SYM_DEN>
struct BgEvalGrad {
    template <typename R>
    static cudaError_t run(const double* mom, long long n, double* me2, double* dme2, double mt, double norm,
                           cudaStream_t s)
    {
        constexpr int W = bg_grad_warps<G, R>();
        const size_t sm = bg_grad_smem<G, R>(W);
        static bool attr = false;   // per precision
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute((const void*)bg_evaluate_grad_kernel<G, R>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const long long want = (n + W - 1) / W;
        const int nblk = (int)(want < 8192 ? want : 8192);
        bg_evaluate_grad_kernel<G, R><<<nblk, 32 * W, sm, s>>>(mom, n, me2, dme2, mt, norm);
        return cudaGetLastError();
    }
    static cudaError_t launch(int prec, const double* mom, long long n, double* me2, double* dme2, double mt, double gs,
                              int, cudaStream_t s)
    {
        double norm = 1.0 / (256.0 * SYM_DEN);
        for (int i = 0; i < G::K; ++i) norm *= gs * gs;
        return prec ? run<float>(mom, n, me2, dme2, mt, norm, s) : run<double>(mom, n, me2, dme2, mt, norm, s);
    }
};

}  // namespace mf

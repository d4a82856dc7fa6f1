// d|M|^2/dp of g g -> t tbar g g by a reverse sweep of the helicity-recycled recursion
// (mf_rc.cuh), one warp per point, mixed precision: the derivative of the matrix element of
// Sec. 2.2 with respect to every momentum component (the momenta as independent variables).
//
// Forward: the record (double-float arithmetic), the recycled currents and each lane's 24 partial
// amplitudes, as the value kernel.  Backward, with a second store of the same layout for the
// adjoints (zb = dL/dRe z + i dL/dIm z of L, the helicity-summed colour sum):
//  * the colour sum: Abar = 2 (C A), doubled for the parity mirrors;
//  * the contractions X . Y of every ordering: Xbar += s g conj(Y) Abar, Ybar likewise.  The
//    lanes whose helicity bits agree on an operand's mask share its slot: their contributions are
//    summed by a butterfly over the other bits and one lane adds the sum to the slot;
//  * the tasks stage by stage backwards, each lane its task: the adjoints of the operands added
//    to their slots with shared-memory atomics (tasks of one step may share an operand), those of
//    the per-event invariants pushed onto the external momenta and m_t in the lane's registers,
//    those of the polarisation and spinor bases into the warp's shared arrays;
//  * then lane j carries the tangent of momentum component j through the invariants' FP64
//    arithmetic and contracts it with their adjoints (as the reverse sweep of mf_bg.cuh).
#pragma once
#include "mf_rc.cuh"

namespace mf {

// ---------------------------------------------------------------- adjoints of the column routines

// adjoint of o = col_jslash(J, f) = (Sigma(J) (f2, f3) ; Sigmabar(J) (f0, f1)) given ob: Jb, fb accumulated
template <typename R>
__device__ __forceinline__ void col_jslash_adj(const W4<R>& J, const W4<R>& f, const W4<R>& ob, W4<R>& Jb, W4<R>& fb)
{
    const M2<R> S = sig(J), Sb = sigbar(J);
    // column products y_c = sum_r M_cr x_r: x_r gets sum_c yb_c conj(M_cr)
    fb.c[2] = cadd(fb.c[2], cadd(cmulc(ob.c[0], S.m00), cmulc(ob.c[1], S.m10)));
    fb.c[3] = cadd(fb.c[3], cadd(cmulc(ob.c[0], S.m01), cmulc(ob.c[1], S.m11)));
    fb.c[0] = cadd(fb.c[0], cadd(cmulc(ob.c[2], Sb.m00), cmulc(ob.c[3], Sb.m10)));
    fb.c[1] = cadd(fb.c[1], cadd(cmulc(ob.c[2], Sb.m01), cmulc(ob.c[3], Sb.m11)));
    // entry adjoints M_cr: yb_c conj(x_r)
    const cx<R> ss00 = cmulc(ob.c[0], f.c[2]), ss01 = cmulc(ob.c[0], f.c[3]);
    const cx<R> ss10 = cmulc(ob.c[1], f.c[2]), ss11 = cmulc(ob.c[1], f.c[3]);
    const cx<R> bb00 = cmulc(ob.c[2], f.c[0]), bb01 = cmulc(ob.c[2], f.c[1]);
    const cx<R> bb10 = cmulc(ob.c[3], f.c[0]), bb11 = cmulc(ob.c[3], f.c[1]);
    // the entries' dependence on J as in row_jslash_adj
    Jb.c[0] = cadd(Jb.c[0], cadd(cadd(ss00, ss11), cadd(bb00, bb11)));
    Jb.c[3] = cadd(Jb.c[3], cadd(csub(ss11, ss00), csub(bb00, bb11)));
    Jb.c[1] = cadd(Jb.c[1], csub(cadd(bb01, bb10), cadd(ss01, ss10)));
    const cx<R> t = cadd(csub(ss01, ss10), csub(bb10, bb01));
    Jb.c[2] = cadd(Jb.c[2], mkc(t.i, -t.r));
}

// adjoint of o = s (qslash + m) x on a column spinor (the propagator part of ffv_col) given ob:
// xb accumulated, qb, mb, sb
template <typename R>
__device__ __forceinline__ void col_qprop_adj(const W4<R>& x, const R* q, R m, R s, const W4<R>& ob, W4<R>& xb,
                                              R* qb, R& mb, R& sb)
{
    cx<R> t0, t1, u0, u1;
    qcol(q, false, x.c[2], x.c[3], t0, t1);
    qcol(q, true, x.c[0], x.c[1], u0, u1);
    W4<R> inner;
    inner.c[0] = mkc(fma(m, x.c[0].r, t0.r), fma(m, x.c[0].i, t0.i));
    inner.c[1] = mkc(fma(m, x.c[1].r, t1.r), fma(m, x.c[1].i, t1.i));
    inner.c[2] = mkc(fma(m, x.c[2].r, u0.r), fma(m, x.c[2].i, u0.i));
    inner.c[3] = mkc(fma(m, x.c[3].r, u1.r), fma(m, x.c[3].i, u1.i));
    for (int c = 0; c < 4; ++c) sb += re_mulc(ob.c[c], inner.c[c]);
    W4<R> o;
    for (int c = 0; c < 4; ++c) o.c[c] = cscale(ob.c[c], s);
    // S_q = [[q0 - q3, -q1 + i q2], [-q1 - i q2, q0 + q3]] acts on (x2, x3) into (o0, o1);
    // Sb_q = [[q0 + q3, q1 - i q2], [q1 + i q2, q0 - q3]] on (x0, x1) into (o2, o3)
    const cx<R> S00 = mkc(q[0] - q[3], R(0)), S11 = mkc(q[0] + q[3], R(0));
    const cx<R> S01 = mkc(-q[1], q[2]), S10 = mkc(-q[1], -q[2]);
    const cx<R> Sb00 = mkc(q[0] + q[3], R(0)), Sb11 = mkc(q[0] - q[3], R(0));
    const cx<R> Sb01 = mkc(q[1], -q[2]), Sb10 = mkc(q[1], q[2]);
    xb.c[0] = cadd(xb.c[0], cadd(cscale(o.c[0], m), cadd(cmulc(o.c[2], Sb00), cmulc(o.c[3], Sb10))));
    xb.c[1] = cadd(xb.c[1], cadd(cscale(o.c[1], m), cadd(cmulc(o.c[2], Sb01), cmulc(o.c[3], Sb11))));
    xb.c[2] = cadd(xb.c[2], cadd(cscale(o.c[2], m), cadd(cmulc(o.c[0], S00), cmulc(o.c[1], S10))));
    xb.c[3] = cadd(xb.c[3], cadd(cscale(o.c[3], m), cadd(cmulc(o.c[0], S01), cmulc(o.c[1], S11))));
    for (int c = 0; c < 4; ++c) mb += re_mulc(o.c[c], x.c[c]);
    const cx<R> a00 = cmulc(o.c[0], x.c[2]), a01 = cmulc(o.c[0], x.c[3]), a10 = cmulc(o.c[1], x.c[2]), a11 = cmulc(o.c[1], x.c[3]);
    const cx<R> b00 = cmulc(o.c[2], x.c[0]), b01 = cmulc(o.c[2], x.c[1]), b10 = cmulc(o.c[3], x.c[0]), b11 = cmulc(o.c[3], x.c[1]);
    qb[0] += a00.r + a11.r + b00.r + b11.r;
    qb[3] += -a00.r + a11.r + b00.r - b11.r;
    qb[1] += -a01.r - a10.r + b01.r + b10.r;
    qb[2] += a01.i - a10.i - b01.i + b10.i;
}

// adjoint of X = ffv_cur(fb, f, 1) = fb gamma^mu f given Xb: fbb (the row's) and fcb accumulated
template <typename R>
__device__ __forceinline__ void ffv_cur_adj(const W4<R>& fbr, const W4<R>& f, const W4<R>& Xb, W4<R>& fbb, W4<R>& fcb)
{
    const cx<R> a0 = fbr.c[0], a1 = fbr.c[1], b0 = fbr.c[2], b1 = fbr.c[3];
    const cx<R> c0 = f.c[0], c1 = f.c[1], d0 = f.c[2], d1 = f.c[3];
    // X0 = ad00 + ad11 + bc00 + bc11, X1 = ad01 + ad10 - bc01 - bc10,
    // X2 = i (ad10 - ad01 - bc10 + bc01), X3 = ad00 - ad11 - bc00 + bc11
    const cx<R> iX2 = mkc(-Xb.c[2].i, Xb.c[2].r);     // i Xb2
    const cx<R> ad00 = cadd(Xb.c[0], Xb.c[3]), ad11 = csub(Xb.c[0], Xb.c[3]);
    const cx<R> ad01 = cadd(Xb.c[1], iX2), ad10 = csub(Xb.c[1], iX2);
    const cx<R> bc00 = csub(Xb.c[0], Xb.c[3]), bc11 = cadd(Xb.c[0], Xb.c[3]);
    const cx<R> bc01 = csub(mkc(-Xb.c[1].r, -Xb.c[1].i), iX2), bc10 = cadd(mkc(-Xb.c[1].r, -Xb.c[1].i), iX2);
    fbb.c[0] = cadd(fbb.c[0], cadd(cmulc(ad00, d0), cmulc(ad01, d1)));
    fbb.c[1] = cadd(fbb.c[1], cadd(cmulc(ad10, d0), cmulc(ad11, d1)));
    fbb.c[2] = cadd(fbb.c[2], cadd(cmulc(bc00, c0), cmulc(bc01, c1)));
    fbb.c[3] = cadd(fbb.c[3], cadd(cmulc(bc10, c0), cmulc(bc11, c1)));
    fcb.c[0] = cadd(fcb.c[0], cadd(cmulc(bc00, b0), cmulc(bc10, b1)));
    fcb.c[1] = cadd(fcb.c[1], cadd(cmulc(bc01, b0), cmulc(bc11, b1)));
    fcb.c[2] = cadd(fcb.c[2], cadd(cmulc(ad00, a0), cmulc(ad10, a1)));
    fcb.c[3] = cadd(fcb.c[3], cadd(cmulc(ad01, a0), cmulc(ad11, a1)));
}

// ---------------------------------------------------------------- the adjoint store

// the adjoints of the store's slots: the layout of RcWarpT<float>::W
struct RcAdj {
    float4 W[2][rcT::NSLOT];
    float e1b[4][3], e2b[4][3];          // the gluons' transverse bases
    cx<float> chi3b[2][2], chi4b[2][2];  // the spinor pieces of t and tbar
    float om3b[2], om4b[2];
};

__device__ __forceinline__ W4<float> rcb_ld(const RcAdj& a, int i)
{
    const float4 x = a.W[0][i], y = a.W[1][i];
    W4<float> o;
    o.c[0] = mkc(x.x, x.y); o.c[1] = mkc(x.z, x.w); o.c[2] = mkc(y.x, y.y); o.c[3] = mkc(y.z, y.w);
    return o;
}
// add v to slot i (one writer per slot and instruction)
__device__ __forceinline__ void rcb_add(RcAdj& a, int i, const W4<float>& v)
{
    float4 x = a.W[0][i], y = a.W[1][i];
    x.x += v.c[0].r; x.y += v.c[0].i; x.z += v.c[1].r; x.w += v.c[1].i;
    y.x += v.c[2].r; y.y += v.c[2].i; y.z += v.c[3].r; y.w += v.c[3].i;
    a.W[0][i] = x;
    a.W[1][i] = y;
}
// add v to slot i with shared-memory atomics (several lanes of a step may share the slot)
__device__ __forceinline__ void rcb_atomic(RcAdj& a, int i, const W4<float>& v)
{
    float* x = &a.W[0][i].x;
    float* y = &a.W[1][i].x;
    atomicAdd(x, v.c[0].r); atomicAdd(x + 1, v.c[0].i); atomicAdd(x + 2, v.c[1].r); atomicAdd(x + 3, v.c[1].i);
    atomicAdd(y, v.c[2].r); atomicAdd(y + 1, v.c[2].i); atomicAdd(y + 2, v.c[3].r); atomicAdd(y + 3, v.c[3].i);
}
// v summed over the lanes that agree with this lane on the bits of mask (a butterfly over the
// other lane bits; mask uniform over the warp), every lane of a group left with the group's sum
__device__ __forceinline__ void rc_group_sum(W4<float>& v, unsigned mask)
{
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        if ((mask >> b) & 1u) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            v.c[m].r += __shfl_xor_sync(0xffffffffu, v.c[m].r, 1 << b);
            v.c[m].i += __shfl_xor_sync(0xffffffffu, v.c[m].i, 1 << b);
        }
    }
}

// ---------------------------------------------------------------- the tasks backwards

using RcInv = BgInvAcc<float, 4>;

// the adjoint of a current J = ip acc (ip = 1/P^2 of subset m): accb = ip Jb, and the adjoint
// of P_m from that of ip (d(1/P^2) = -2 P.dP / P^4) pushed onto the external momenta
__device__ __forceinline__ W4<float> rc_scale_adj(const RcWarp& w, RcInv& gi, int out, const W4<float>& Jb, int m)
{
    const W4<float> Jo = rc_ld(w, out);
    const float ip = w.r.iP2[m];
    W4<float> accb;
    float ipb = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) { accb.c[c] = cscale(Jb.c[c], ip); ipb += re_mulc(Jb.c[c], Jo.c[c]); }
    const float f = -2.0f * (ipb / ip) * ip * ip;
    float P[4], pb[4];
    rc_mom(w, m, P);
#pragma unroll
    for (int c = 0; c < 4; ++c) pb[c] = f * metric(c) * P[c];
    inv_acc_P(gi, m, pb);
    return accb;
}
// the adjoint of a propagator scale s = -1/(Q^2 - m^2), Q = p_t - P_qm, and of q and m_t
__device__ __forceinline__ void rc_prop_adj(const RcWarp& w, RcInv& gi, int qm, const float* q, float* qb, float mb,
                                            float sb)
{
    const float iq = w.r.iQ[qm], f = -2.0f * (-sb) * iq * iq;
#pragma unroll
    for (int c = 0; c < 4; ++c) qb[c] += f * metric(c) * q[c];
    inv_acc_Q(gi, qm, qb);
    gi.gmt += mb - f * w.r.mt;
}
__device__ __forceinline__ void rc_vvv_adj(const RcWarp& w, RcInv& gi, int sa, int sb_, int ma, int mb, float s,
                                           const W4<float>& accb, W4<float>& Jab, W4<float>& Jbb)
{
    float k1[4], k2[4], k1b[4] = { 0.f, 0.f, 0.f, 0.f }, k2b[4] = { 0.f, 0.f, 0.f, 0.f };
    rc_mom(w, ma, k1);
    rc_mom(w, mb, k2);
    vvv_cur_adj(rc_ld(w, sa), rc_ld(w, sb_), k1, k2, s, accb, Jab, Jbb, k1b, k2b);
    inv_acc_P(gi, ma, k1b);
    inv_acc_P(gi, mb, k2b);
}

template <class T> __device__ __forceinline__ void rc_adj_j2(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const W4<float> accb = rc_scale_adj(w, gi, t.f(0), rcb_ld(a, t.f(0)), t.f(6));
    W4<float> ab = w4_zero<float>(), bb = w4_zero<float>();
    rc_vvv_adj(w, gi, t.f(1), t.f(2), t.f(4), t.f(5), -1.0f, accb, ab, bb);
    rcb_atomic(a, t.f(1), ab);
    rcb_atomic(a, t.f(2), bb);
}

template <class T> __device__ __forceinline__ void rc_adj_j3(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const unsigned sg = t.f(6);
    const W4<float> accb = rc_scale_adj(w, gi, t.f(0), rcb_ld(a, t.f(0)), t.f(11));
    W4<float> xb = w4_zero<float>(), yb = w4_zero<float>(), zb = w4_zero<float>();
    W4<float> xyb = w4_zero<float>(), yzb = w4_zero<float>();
    rc_vvv_adj(w, gi, t.f(1), t.f(5), t.f(7), t.f(8), -rc_sign<float>(sg, 0), accb, xb, yzb);
    rc_vvv_adj(w, gi, t.f(4), t.f(3), t.f(9), t.f(10), -rc_sign<float>(sg, 1), accb, xyb, zb);
    v4_adj(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), rc_ld(w, t.f(3)), 1.0f, accb, xb, yb, zb);
    rcb_atomic(a, t.f(1), xb);
    rcb_atomic(a, t.f(2), yb);
    rcb_atomic(a, t.f(3), zb);
    rcb_atomic(a, t.f(4), xyb);
    rcb_atomic(a, t.f(5), yzb);
}

template <class T> __device__ __forceinline__ void rc_adj_j4(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const unsigned sg = t.f(10);
    const W4<float> accb = rc_scale_adj(w, gi, t.f(0), rcb_ld(a, t.f(0)), t.f(17));
    // operand adjoints in the order of the fields: w, x, y, z, wx, xy, yz, wxy, xyz
    W4<float> ob[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) ob[i] = w4_zero<float>();
    rc_vvv_adj(w, gi, t.f(1), t.f(9), t.f(11), t.f(12), -rc_sign<float>(sg, 0), accb, ob[0], ob[8]);
    rc_vvv_adj(w, gi, t.f(5), t.f(7), t.f(13), t.f(14), -rc_sign<float>(sg, 1), accb, ob[4], ob[6]);
    rc_vvv_adj(w, gi, t.f(8), t.f(4), t.f(15), t.f(16), -rc_sign<float>(sg, 2), accb, ob[7], ob[3]);
    v4_adj(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), rc_ld(w, t.f(7)), rc_sign<float>(sg, 3), accb, ob[0], ob[1], ob[6]);
    v4_adj(rc_ld(w, t.f(1)), rc_ld(w, t.f(6)), rc_ld(w, t.f(4)), rc_sign<float>(sg, 4), accb, ob[0], ob[5], ob[3]);
    v4_adj(rc_ld(w, t.f(5)), rc_ld(w, t.f(3)), rc_ld(w, t.f(4)), rc_sign<float>(sg, 5), accb, ob[4], ob[2], ob[3]);
#pragma unroll
    for (int i = 0; i < 9; ++i) rcb_atomic(a, t.f(1 + i), ob[i]);
}

template <class T> __device__ __forceinline__ void rc_adj_u1(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const int qm = t.f(3);
    float q[4], qb[4] = { 0.f, 0.f, 0.f, 0.f }, mb = 0.f, sb = 0.f;
    rc_qmom(w, qm, q);
    const W4<float> ub = rc_ld(w, t.f(1)), g = rc_ld(w, t.f(2));
    W4<float> xb = w4_zero<float>();
    row_qprop_adj(row_jslash(ub, g), q, w.r.mt, -w.r.iQ[qm], rcb_ld(a, t.f(0)), xb, qb, mb, sb);
    rc_prop_adj(w, gi, qm, q, qb, mb, sb);
    W4<float> ubb = w4_zero<float>(), gb = w4_zero<float>();
    row_jslash_adj(ub, g, xb, ubb, gb);
    rcb_atomic(a, t.f(1), ubb);
    rcb_atomic(a, t.f(2), gb);
}

template <class T> __device__ __forceinline__ void rc_adj_vr1(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const int qm = t.f(3);
    float q[4], qb[4] = { 0.f, 0.f, 0.f, 0.f }, mb = 0.f, sb = 0.f;
    rc_qmom(w, qm, q);
    const W4<float> g = rc_ld(w, t.f(1)), v = rc_ld(w, t.f(2));
    W4<float> xb = w4_zero<float>();
    col_qprop_adj(col_jslash(g, v), q, w.r.mt, -w.r.iQ[qm], rcb_ld(a, t.f(0)), xb, qb, mb, sb);
    rc_prop_adj(w, gi, qm, q, qb, mb, sb);
    W4<float> gb = w4_zero<float>(), vb = w4_zero<float>();
    col_jslash_adj(g, v, xb, gb, vb);
    rcb_atomic(a, t.f(1), gb);
    rcb_atomic(a, t.f(2), vb);
}

template <class T> __device__ __forceinline__ void rc_adj_u2(const RcWarp& w, RcAdj& a, RcInv& gi, const T& t)
{
    const int qm = t.f(6);
    const float s = rc_sign<float>(t.f(3), 0);
    const W4<float> ub = rc_ld(w, t.f(1)), jab = rc_ld(w, t.f(2)), u1a = rc_ld(w, t.f(4)), gb_ = rc_ld(w, t.f(5));
    W4<float> x = row_jslash(u1a, gb_);
    w4_fma(x, s, row_jslash(ub, jab));
    float q[4], qb[4] = { 0.f, 0.f, 0.f, 0.f }, mb = 0.f, sb = 0.f;
    rc_qmom(w, qm, q);
    W4<float> xb = w4_zero<float>();
    row_qprop_adj(x, q, w.r.mt, -w.r.iQ[qm], rcb_ld(a, t.f(0)), xb, qb, mb, sb);
    rc_prop_adj(w, gi, qm, q, qb, mb, sb);
    W4<float> u1ab = w4_zero<float>(), gbb = w4_zero<float>(), ubb = w4_zero<float>(), jabb = w4_zero<float>();
    row_jslash_adj(u1a, gb_, xb, u1ab, gbb);
    W4<float> xs;
#pragma unroll
    for (int c = 0; c < 4; ++c) xs.c[c] = cscale(xb.c[c], s);
    row_jslash_adj(ub, jab, xs, ubb, jabb);
    rcb_atomic(a, t.f(1), ubb);
    rcb_atomic(a, t.f(2), jabb);
    rcb_atomic(a, t.f(4), u1ab);
    rcb_atomic(a, t.f(5), gbb);
}

template <class T> __device__ __forceinline__ void rc_adj_w2(const RcWarp& w, RcAdj& a, RcInv&, const T& t)
{
    const float s = rc_sign<float>(t.f(2), 0);
    const W4<float> ob = rcb_ld(a, t.f(0));
    W4<float> jcdb = w4_zero<float>(), vb = w4_zero<float>(), gcb = w4_zero<float>(), vrb = w4_zero<float>();
    col_jslash_adj(rc_ld(w, t.f(4)), rc_ld(w, t.f(5)), ob, gcb, vrb);
    W4<float> os;
#pragma unroll
    for (int c = 0; c < 4; ++c) os.c[c] = cscale(ob.c[c], s);
    col_jslash_adj(rc_ld(w, t.f(1)), rc_ld(w, t.f(3)), os, jcdb, vb);
    rcb_atomic(a, t.f(1), jcdb);
    rcb_atomic(a, t.f(3), vb);
    rcb_atomic(a, t.f(4), gcb);
    rcb_atomic(a, t.f(5), vrb);
}

template <class T> __device__ __forceinline__ void rc_adj_x(const RcWarp& w, RcAdj& a, RcInv&, const T& t)
{
    W4<float> rb = w4_zero<float>(), cb = w4_zero<float>();
    ffv_cur_adj(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), rcb_ld(a, t.f(0)), rb, cb);
    rcb_atomic(a, t.f(1), rb);
    rcb_atomic(a, t.f(2), cb);
}

// the external states backwards into the bases' adjoints (shared, atomics: the two
// helicities of a particle are two lanes)
template <class T> __device__ __forceinline__ void rc_adj_ext(const RcWarp& w, RcAdj& a, RcInv&, const T& t)
{
    const int code = t.f(1), hel = t.f(2) ? 1 : -1;
    const W4<float> ob = rcb_ld(a, t.f(0));
    if (code < 4) {
        const float l = hel > 0 ? 1.0f : -1.0f, so = code >= 2 ? 1.0f : -1.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            atomicAdd(&a.e1b[code][j], -l * ob.c[j + 1].r);
            atomicAdd(&a.e2b[code][j], so * ob.c[j + 1].i);
        }
    } else if (code == 4) {
        // ubar = (conj(chi_l) om_l, conj(chi_l) om_-l)
        const int l = hel > 0 ? 0 : 1;
        const float wl = w.r.fb3.om[l], wml = w.r.fb3.om[1 - l];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const cx<float> d = cadd(cscale(conjc(ob.c[b]), wl), cscale(conjc(ob.c[2 + b]), wml));
            atomic_add_cx(&a.chi3b[l][b], d);
            const cx<float> ch = w.r.fb3.chi[l][b];
            atomicAdd(&a.om3b[l], ob.c[b].r * ch.r - ob.c[b].i * ch.i);
            atomicAdd(&a.om3b[1 - l], ob.c[2 + b].r * ch.r - ob.c[2 + b].i * ch.i);
        }
    } else {
        // v = (chi_-l (-s om_l), chi_-l (s om_-l))
        const int l = hel > 0 ? 0 : 1;
        const float sl = hel > 0 ? 1.0f : -1.0f;
        const float wl = w.r.fb4.om[l], wml = w.r.fb4.om[1 - l];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const cx<float> d = cadd(cscale(ob.c[b], -sl * wl), cscale(ob.c[2 + b], sl * wml));
            atomic_add_cx(&a.chi4b[1 - l][b], d);
            const cx<float> ch = w.r.fb4.chi[1 - l][b];
            atomicAdd(&a.om4b[l], -sl * re_mulc(ob.c[b], ch));
            atomicAdd(&a.om4b[1 - l], sl * re_mulc(ob.c[2 + b], ch));
        }
    }
}

#define MF_RC_ADJ_STEPS(TYPE, FN)                                                                          \
    for (int s_ = rcT::STEPS_##TYPE - 1; s_ >= 0; --s_) {                                                 \
        const auto t_ = rc_task<rcT::NQ_##TYPE>(&rcT::task_##TYPE[0][0][0][0], s_, lane);                  \
        if (t_.f(0) != 0xFFFF) FN(w, a, gi, t_);                                                           \
    }

// every task backwards, stage by stage (the stages of rc_currents in reverse order)
__device__ __forceinline__ void rc_currents_adj(const RcWarp& w, RcAdj& a, RcInv& gi, int lane)
{
    MF_RC_ADJ_STEPS(X, rc_adj_x)
    MF_RC_ADJ_STEPS(W2, rc_adj_w2)
    MF_RC_ADJ_STEPS(U2, rc_adj_u2)
    MF_RC_ADJ_STEPS(J4, rc_adj_j4)
    __syncwarp();
    MF_RC_ADJ_STEPS(VR1, rc_adj_vr1)
    MF_RC_ADJ_STEPS(U1, rc_adj_u1)
    MF_RC_ADJ_STEPS(J3, rc_adj_j3)
    __syncwarp();
    MF_RC_ADJ_STEPS(J2, rc_adj_j2)
    __syncwarp();
    MF_RC_ADJ_STEPS(EXT, rc_adj_ext)
    __syncwarp();
}
#undef MF_RC_ADJ_STEPS

// ---------------------------------------------------------------- one point, one warp

constexpr int RCE_WARPS = 4, RCE_ROW = 2 * rcT::NPERM + 1;
struct RcEvalWarp {
    RcWarp w;
    RcAdj a;
    float rows[32][RCE_ROW];   // each lane's partial amplitudes, then their adjoints
};
__host__ __device__ constexpr size_t rce_warp_bytes() { return (sizeof(RcEvalWarp) + 15) & ~(size_t)15; }

// me2 [n] and dme2 [n][6][4]: |M|^2 and its derivatives with respect to every momentum component
// (norm: couplings, averages and the identical-gluon factor)
__global__ void __launch_bounds__(32 * RCE_WARPS, 1) rc_evaluate_grad_kernel(const double* __restrict__ mom, long long n,
                                                                             double* __restrict__ me2,
                                                                             double* __restrict__ dme2, double mt,
                                                                             double norm)
{
    constexpr int N = rcT::NPERM, NEXT = 6;
    using D = Dual<double>;
    extern __shared__ __align__(128) unsigned char mf_rce_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RcEvalWarp& st = *reinterpret_cast<RcEvalWarp*>(mf_rce_smem + (size_t)warp * rce_warp_bytes());
    const uint32_t* lt = &rcT::lane_terms[0][0][0] + lane;
    float* row = st.rows[lane];
    const Df mt_df(mt);
    for (long long e = (long long)blockIdx.x * RCE_WARPS + warp; e < n; e += (long long)gridDim.x * RCE_WARPS) {
        double p[NEXT][4];
#pragma unroll
        for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = mom[e * NEXT * 4 + f];
        {
            // every lane forms the record (in double-float arithmetic, as the integrand's), each
            // stores its share of the words
            Df pdf[NEXT][4];
#pragma unroll
            for (int f = 0; f < NEXT * 4; ++f) pdf[f >> 2][f & 3] = Df(p[f >> 2][f & 3]);
            RcRec rec;
            rc_record<float>(pdf, mt_df, rec);
            const float* ws = reinterpret_cast<const float*>(&rec);
            float* wd = reinterpret_cast<float*>(&st.w.r);
            for (int f = lane; f < RC_REC_WORDS; f += 32) wd[f] = ws[f];
        }
        __syncwarp();
        rc_currents<float, false>(st.w, lane);
        const W4<float> jq = rc_jq(st.w, lt, true);
#pragma unroll 1
        for (int pc = 0; pc < N / 2; ++pc) {
            cx<float> a[2];
            rc_amp_pair<float, true>(st.w, lt, pc, jq, a);
            row[4 * pc] = a[0].r; row[4 * pc + 1] = a[0].i; row[4 * pc + 2] = a[1].r; row[4 * pc + 3] = a[1].i;
        }
        // colour sum of the lane's configuration, and the amplitudes' adjoints 2 (54 C A) doubled
        // for the parity mirror
        float v = 0.0f;
        {
            float ar[N], ai[N], yr[N], yi[N];
#pragma unroll
            for (int s_ = 0; s_ < N; ++s_) { ar[s_] = row[2 * s_]; ai[s_] = row[2 * s_ + 1]; }
#pragma unroll
            for (int t = 0; t < N; ++t) {
                float r = 0.0f, i = 0.0f;
#pragma unroll
                for (int s_ = 0; s_ < N; ++s_) {
                    r = fmaf(rcT::colour[t * N + s_], ar[s_], r);
                    i = fmaf(rcT::colour[t * N + s_], ai[s_], i);
                }
                yr[t] = r;
                yi[t] = i;
                v = fmaf(ar[t], r, fmaf(ai[t], i, v));
            }
#pragma unroll
            for (int t = 0; t < N; ++t) { row[2 * t] = 4.0f * yr[t]; row[2 * t + 1] = 4.0f * yi[t]; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0 && me2) me2[e] = (double)v * 2.0 / rcT::COLOUR_DEN * norm;
        // the adjoint store and the bases' adjoints start at zero
        for (int i = lane; i < rcT::NSLOT; i += 32) {
            st.a.W[0][i] = make_float4(0.f, 0.f, 0.f, 0.f);
            st.a.W[1][i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (lane < 12) { st.a.e1b[lane / 3][lane % 3] = 0.0f; st.a.e2b[lane / 3][lane % 3] = 0.0f; }
        if (lane < 8) {
            cx<float>* c3 = &st.a.chi3b[0][0];
            cx<float>* c4 = &st.a.chi4b[0][0];
            if (lane < 4) c3[lane] = mkc(0.0f, 0.0f); else c4[lane - 4] = mkc(0.0f, 0.0f);
        }
        if (lane < 2) { st.a.om3b[lane] = 0.0f; st.a.om4b[lane] = 0.0f; }
        __syncwarp();
        RcInv gi;
        inv_acc_zero(gi);
        // the contractions backwards: Xbar += s g conj(Y) Abar, Ybar += s g conj(X) Abar, summed
        // over the lanes that share a slot
#pragma unroll 1
        for (int sg = 0; sg < N; ++sg) {
            const cx<float> ab = mkc(row[2 * sg], row[2 * sg + 1]);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const uint32_t word = __ldg(lt + (sg * 5 + k) * 32);
                const unsigned masks = rcT::term_masks[sg][k];
                const int sa = (int)(word & 0xFFFu), sb = (int)((word >> 12) & 0xFFFu);
                const float sgn = ((word >> 24) & 1u) ? -1.0f : 1.0f;
                const W4<float> x = rc_ld(st.w, sa), y = rc_ld(st.w, sb);
                W4<float> xb, yb;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float g = sgn * (k == 0 ? 1.0f : metric(m));
                    xb.c[m] = cscale(cmulc(ab, y.c[m]), g);
                    yb.c[m] = cscale(cmulc(ab, x.c[m]), g);
                }
                const unsigned ma = masks & 31u, mb = (masks >> 5) & 31u;
                rc_group_sum(xb, ma);
                if ((lane & ~ma & 31) == 0) rcb_add(st.a, sa, xb);
                __syncwarp();
                rc_group_sum(yb, mb);
                if ((lane & ~mb & 31) == 0) rcb_add(st.a, sb, yb);
                __syncwarp();
            }
        }
        rc_currents_adj(st.w, st.a, gi, lane);
        // the lanes' invariant adjoints added up (every lane gets the sums)
#pragma unroll
        for (int f = 0; f < NEXT * 4; ++f)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) gi.gp[f >> 2][f & 3] += __shfl_xor_sync(0xffffffffu, gi.gp[f >> 2][f & 3], off);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) gi.gmt += __shfl_xor_sync(0xffffffffu, gi.gmt, off);
        // lane j < 24: the tangent of momentum component j through the invariants' FP64
        // arithmetic, contracted with their adjoints
        if (lane < NEXT * 4) {
            D pd[NEXT][4];
            for (int i = 0; i < NEXT; ++i)
                for (int c = 0; c < 4; ++c) pd[i][c] = D(p[i][c], (4 * i + c) == lane ? 1.0 : 0.0);
            const D mtd(mt, 0.0);
            double g = double(gi.gp[lane >> 2][lane & 3]);
            for (int gl = 0; gl < 4; ++gl) {
                // parallel-transported basis tangent: de = -(e . dn) n (see gluon_basis)
                const D* q = pd[gl < 2 ? gl : gl + 2];
                const double pa = sqrt(q[1].v * q[1].v + q[2].v * q[2].v + q[3].v * q[3].v);
                const double nn[3] = { q[1].v / pa, q[2].v / pa, q[3].v / pa };
                const double ndp = nn[0] * q[1].d + nn[1] * q[2].d + nn[2] * q[3].d;
                const double dn[3] = { (q[1].d - nn[0] * ndp) / pa, (q[2].d - nn[1] * ndp) / pa,
                                       (q[3].d - nn[2] * ndp) / pa };
                double c1 = 0.0, c2 = 0.0, b1 = 0.0, b2 = 0.0;
                for (int j = 0; j < 3; ++j) {
                    c1 += double(st.w.r.e1[gl][j]) * dn[j];
                    c2 += double(st.w.r.e2[gl][j]) * dn[j];
                    b1 += nn[j] * double(st.a.e1b[gl][j]);
                    b2 += nn[j] * double(st.a.e2b[gl][j]);
                }
                g -= c1 * b1 + c2 * b2;
            }
            {
                const FermionBasis<D> f3 = fermion_basis<D>(pd[2], mtd), f4 = fermion_basis<D>(pd[3], mtd);
                for (int x = 0; x < 2; ++x)
                    for (int b = 0; b < 2; ++b) {
                        g += f3.chi[x][b].r.d * double(st.a.chi3b[x][b].r) + f3.chi[x][b].i.d * double(st.a.chi3b[x][b].i);
                        g += f4.chi[x][b].r.d * double(st.a.chi4b[x][b].r) + f4.chi[x][b].i.d * double(st.a.chi4b[x][b].i);
                    }
                for (int x = 0; x < 2; ++x) g += f3.om[x].d * double(st.a.om3b[x]) + f4.om[x].d * double(st.a.om4b[x]);
            }
            if (dme2) dme2[e * NEXT * 4 + lane] = g / rcT::COLOUR_DEN * norm;
        }
        __syncwarp();
    }
}

}  // namespace mf


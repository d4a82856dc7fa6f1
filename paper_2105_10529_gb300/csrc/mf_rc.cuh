// g g -> t tbar g g by the helicity-recycled Berends-Giele recursion, one warp per
// event (the matrix element of Sec. 2.2 of arXiv:2105.10529, re-associated).
//
// The paper's generated code evaluates every Feynman diagram once per helicity
// configuration.  Here the colour-ordered partial amplitudes of the 32 configurations of
// the parity-halved sum are built together, from the tables of generated/rc_gg_ttgg.cuh:
//
//  * an off-shell current depends only on the helicities of the particles it contains,
//    so each of its distinct values ("helicity combination") is computed once and kept
//    in a slot of the warp's store in shared memory.  A task is one (current,
//    combination) pair; a step runs 32 tasks of one routine, one per lane, and the steps
//    of a stage only read slots of earlier stages;
//  * the partial amplitude of an ordering (a b c d) is closed in the middle:
//        A = U2(a b) W2(c d) + X(ubar, Vr1(d)) . J(a b c) + X(ubar, v) . J(a b c d)
//          + X(U1(a), Vr1(d)) . J(b c) + X(U1(a), v) . J(b c d),
//    with U1, U2 the top line after one or two gluons (propagator included), Vr1, W2
//    the line from v(p_tbar) after one or two gluons, and X(row, col) the bilinear
//    row gamma^mu col (a current like the others).  Lane l then forms the 24 amplitudes
//    of configuration ih = 1 + 2 l from five complex contractions each, reading every
//    operand from the slot of its own combination.
//
// The amplitudes go straight into tensor memory for the colour sum (mf_tc.cuh,
// tc_rc_put_pair and tc_rc_colour_sum).  Conventions and routines are those of
// mf_helas.cuh and mf_bg.cuh.  The per-event invariants (subset momenta and inverse
// propagator denominators formed in FP64, stored as FP32) are computed one event per
// thread, like the records of the diagram schedule, and each warp copies its event's.
#pragma once
#include <cstdint>
#include "mf_bg.cuh"
#include "mf_integrand.cuh"
#include "mf_tc.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/rc_gg_ttgg.cuh"

namespace mf {

namespace rcT = rc_gg_ttgg;

// The per-event invariants of one event: the incoming-convention momentum of every
// non-empty gluon subset m (gluons 0, 1 incoming, the rest outgoing with minus their
// momenta) at P[m - 1], p_t, 1 / P^2 of the subsets of two or more gluons, 1 / ((p_t - P)^2
// - m_t^2) of the subsets short of all four, the gluons' transverse bases, the spinor
// pieces of t and tbar and m_t.  R: float (the value kernels) or Dual<float> (the m_t
// derivative pass: every word with its tangent).
template <typename R> struct RcRecT {
    R P[15][4];
    R pt[4];
    R iP2[16];
    R iQ[16];
    R e1[4][3], e2[4][3];
    FermionBasis<R> fb3, fb4;
    R mt;
    R pad[3];
};
using RcRec = RcRecT<float>;
template <typename R> constexpr int rc_rec_words() { return (int)(sizeof(RcRecT<R>) / sizeof(float)); }
constexpr int RC_REC_WORDS = rc_rec_words<float>();
static_assert(RC_REC_WORDS * sizeof(float) == sizeof(RcRec) && RC_REC_WORDS <= LH_INV_WORDS_MAX, "record words");

// one warp's shared-memory state: the store, each slot's components split into 16-byte
// chunks in NCH arrays (so that eight lanes reading eight consecutive slots touch 128
// consecutive bytes, free of bank conflicts), then its event's record
template <typename R> struct RcWarpT {
    static constexpr int NCH = (int)(sizeof(W4<R>) / 16);
    float4 W[NCH][rcT::NSLOT];
    RcRecT<R> r;
};
using RcWarp = RcWarpT<float>;

// the record of one event (one thread; S = Df, double-float for the value path, or double
// or Dual<double> with the m_t tangent for the FP64 and derivative paths); p: g g t tbar g g
template <typename R, typename S>
__device__ __forceinline__ void rc_record(const S (&p)[6][4], S mt, RcRecT<R>& r)
{
    S K[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) K[i][c] = i < 2 ? p[i][c] : -p[i + 2][c];
    S P[16][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) P[0][c] = S(0.0);
#pragma unroll
    for (int m = 1; m < 16; ++m) {
        const int low = __ffs(m) - 1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            P[m][c] = P[m & (m - 1)][c] + K[low][c];
            r.P[m - 1][c] = R(P[m][c]);
        }
        r.iP2[m] = __popc(m) >= 2 ? R(1.0 / mdot(P[m], P[m])) : R(0.0f);
        S q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = p[2][c] - P[m][c];
        r.iQ[m] = m != 15 ? R(1.0 / (mdot(q, q) - mt * mt)) : R(0.0f);
    }
    r.iP2[0] = R(0.0f);
    r.iQ[0] = R(0.0f);
#pragma unroll
    for (int c = 0; c < 4; ++c) r.pt[c] = R(p[2][c]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        S a[3], b[3];
        gluon_basis(p[i < 2 ? i : i + 2], a, b);
#pragma unroll
        for (int j = 0; j < 3; ++j) { r.e1[i][j] = R(a[j]); r.e2[i][j] = R(b[j]); }
    }
    r.fb3 = fermion_basis<R>(p[2], mt);
    r.fb4 = fermion_basis<R>(p[3], mt);
    r.mt = R(mt);
    r.pad[0] = r.pad[1] = r.pad[2] = R(0.0f);
}

// the per-lane words of the five contractions of every ordering (rc_gg_ttgg::lane_terms),
// copied into shared memory once per CTA by the value kernel
constexpr int RC_TERM_BYTES = rcT::TERM_WORDS * (int)sizeof(uint32_t);

template <typename R> __device__ __forceinline__ W4<R> rc_ld(const RcWarpT<R>& w, int i)
{
    W4<R> o;
    float* f = reinterpret_cast<float*>(&o);
#pragma unroll
    for (int k = 0; k < RcWarpT<R>::NCH; ++k) {
        const float4 v = w.W[k][i];
        f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
    return o;
}
template <typename R> __device__ __forceinline__ void rc_st(RcWarpT<R>& w, int i, const W4<R>& v)
{
    const float* f = reinterpret_cast<const float*>(&v);
#pragma unroll
    for (int k = 0; k < RcWarpT<R>::NCH; ++k) w.W[k][i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// one lane's task of a step: NQ 16-byte words of 16-bit fields (low half first)
template <int NQ> struct RcTask {
    uint32_t q[4 * NQ];
    __device__ __forceinline__ int f(int i) const { return (int)((q[i >> 1] >> (16 * (i & 1))) & 0xFFFFu); }
};
template <int NQ> __device__ __forceinline__ RcTask<NQ> rc_task(const uint32_t* tab, int step, int lane)
{
    RcTask<NQ> t;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(tab) + ((size_t)step * NQ + q) * 32 + lane);
        t.q[4 * q] = v.x; t.q[4 * q + 1] = v.y; t.q[4 * q + 2] = v.z; t.q[4 * q + 3] = v.w;
    }
    return t;
}
// a 4-vector of the record (its words read 16 bytes at a time)
template <typename R> __device__ __forceinline__ void rc_vec(const R* src, R (&k)[4])
{
    static_assert(sizeof(R) * 4 % 16 == 0, "16-byte chunks");
    float* f = reinterpret_cast<float*>(&k[0]);
#pragma unroll
    for (int c = 0; c < (int)(sizeof(R) * 4 / 16); ++c) {
        const float4 v = reinterpret_cast<const float4*>(src)[c];
        f[4 * c] = v.x; f[4 * c + 1] = v.y; f[4 * c + 2] = v.z; f[4 * c + 3] = v.w;
    }
}
template <typename R> __device__ __forceinline__ void rc_mom(const RcWarpT<R>& w, int m, R (&k)[4])
{
    rc_vec(&w.r.P[m - 1][0], k);
}
// p_t - P of subset m (the momentum of the top line after absorbing it), in working precision
template <typename R> __device__ __forceinline__ void rc_qmom(const RcWarpT<R>& w, int m, R (&q)[4])
{
    R v[4], t[4];
    rc_vec(&w.r.P[m - 1][0], v);
    rc_vec(&w.r.pt[0], t);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = t[c] - v[c];
}
template <typename R> __device__ __forceinline__ R rc_sign(unsigned bits, int b) { return R((bits >> b) & 1u ? -1.0f : 1.0f); }

// Jslash times a column spinor: (Sigma(J) d ; Sigmabar(J) c) for the column (c ; d)
template <typename R> __device__ __forceinline__ W4<R> col_jslash(const W4<R>& J, const W4<R>& f)
{
    const M2<R> S = sig(J), Sb = sigbar(J);
    W4<R> o;
    mcol(S, f.c[2], f.c[3], o.c[0], o.c[1]);
    mcol(Sb, f.c[0], f.c[1], o.c[2], o.c[3]);
    return o;
}
template <typename R> __device__ __forceinline__ void w4_fma(W4<R>& acc, R s, const W4<R>& x)
{
#pragma unroll
    for (int m = 0; m < 4; ++m) { acc.c[m].r = fma(s, x.c[m].r, acc.c[m].r); acc.c[m].i = fma(s, x.c[m].i, acc.c[m].i); }
}
template <typename R> __device__ __forceinline__ void w4_acc(W4<R>& acc, const W4<R>& x)
{
#pragma unroll
    for (int m = 0; m < 4; ++m) { acc.c[m].r = acc.c[m].r + x.c[m].r; acc.c[m].i = acc.c[m].i + x.c[m].i; }
}

// ---------------------------------------------------------------- the routines of phase 1
// t: this lane's task, the fields of rc_tables.TASK_FIELDS (slot indices of the store)

template <typename R, class T> __device__ __forceinline__ void rc_task_ext(RcWarpT<R>& w, const T& t)
{
    const int code = t.f(1), hel = t.f(2) ? 1 : -1;
    W4<R> o;
    if (code < 4) o = ext_gluon(w.r.e1[code], w.r.e2[code], hel, code >= 2);
    else if (code == 4) o = ext_ubar(w.r.fb3, hel);
    else o = ext_v(w.r.fb4, hel);
    rc_st(w, t.f(0), o);
}

template <typename R, class T> __device__ __forceinline__ void rc_task_j2(RcWarpT<R>& w, const T& t)
{
    R ka[4], kb[4];
    rc_mom(w, t.f(4), ka);
    rc_mom(w, t.f(5), kb);
    const W4<R> o = vvv_cur(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), ka, kb, -w.r.iP2[t.f(6)]);
    rc_st(w, t.f(0), o);
}

// J(x y z) = [ - V3(J(x), J(y z)) - V3(J(x y), J(z)) + V4(J(x), J(y), J(z)) ] / P^2
template <typename R, class T> __device__ __forceinline__ void rc_task_j3(RcWarpT<R>& w, const T& t)
{
    const unsigned sg = t.f(6);
    const W4<R> x = rc_ld(w, t.f(1)), y = rc_ld(w, t.f(2)), z = rc_ld(w, t.f(3));
    R k1[4], k2[4];
    rc_mom(w, t.f(7), k1);
    rc_mom(w, t.f(8), k2);
    W4<R> acc = vvv_cur(x, rc_ld(w, t.f(5)), k1, k2, -rc_sign<R>(sg, 0));
    rc_mom(w, t.f(9), k1);
    rc_mom(w, t.f(10), k2);
    w4_acc(acc, vvv_cur(rc_ld(w, t.f(4)), z, k1, k2, -rc_sign<R>(sg, 1)));
    v4_add(acc, x, y, z, R(1.0f));
    const R ip = w.r.iP2[t.f(11)];
    W4<R> o;
#pragma unroll
    for (int m = 0; m < 4; ++m) o.c[m] = cscale(acc.c[m], ip);
    rc_st(w, t.f(0), o);
}

// J(w x y z): three V3 splits (w | x y z), (w x | y z), (w x y | z) and three V4 splits
// (w, x, y z), (w, x y, z), (w x, y, z)
template <typename R, class T> __device__ __forceinline__ void rc_task_j4(RcWarpT<R>& w, const T& t)
{
    const unsigned sg = t.f(10);
    R k1[4], k2[4];
    W4<R> acc;
    {
        rc_mom(w, t.f(11), k1);
        rc_mom(w, t.f(12), k2);
        acc = vvv_cur(rc_ld(w, t.f(1)), rc_ld(w, t.f(9)), k1, k2, -rc_sign<R>(sg, 0));
    }
    {
        rc_mom(w, t.f(13), k1);
        rc_mom(w, t.f(14), k2);
        w4_acc(acc, vvv_cur(rc_ld(w, t.f(5)), rc_ld(w, t.f(7)), k1, k2, -rc_sign<R>(sg, 1)));
    }
    {
        rc_mom(w, t.f(15), k1);
        rc_mom(w, t.f(16), k2);
        w4_acc(acc, vvv_cur(rc_ld(w, t.f(8)), rc_ld(w, t.f(4)), k1, k2, -rc_sign<R>(sg, 2)));
    }
    v4_add(acc, rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), rc_ld(w, t.f(7)), rc_sign<R>(sg, 3));
    v4_add(acc, rc_ld(w, t.f(1)), rc_ld(w, t.f(6)), rc_ld(w, t.f(4)), rc_sign<R>(sg, 4));
    v4_add(acc, rc_ld(w, t.f(5)), rc_ld(w, t.f(3)), rc_ld(w, t.f(4)), rc_sign<R>(sg, 5));
    const R ip = w.r.iP2[t.f(17)];
    W4<R> o;
#pragma unroll
    for (int m = 0; m < 4; ++m) o.c[m] = cscale(acc.c[m], ip);
    rc_st(w, t.f(0), o);
}

// U1(a) = - ubar Jslash(a) (qslash + m) / (q^2 - m^2), q = p_t - K_a
template <typename R, class T> __device__ __forceinline__ void rc_task_u1(RcWarpT<R>& w, const T& t)
{
    const int qm = t.f(3);
    R q[4];
    rc_qmom(w, qm, q);
    rc_st(w, t.f(0), ffv_row(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), q, w.r.mt, -w.r.iQ[qm]));
}

// Vr1(d) = - (qslash + m) Jslash(d) v / (q^2 - m^2), q = p_t - (every gluon but d)
template <typename R, class T> __device__ __forceinline__ void rc_task_vr1(RcWarpT<R>& w, const T& t)
{
    const int qm = t.f(3);
    R q[4];
    rc_qmom(w, qm, q);
    rc_st(w, t.f(0), ffv_col(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), q, w.r.mt, -w.r.iQ[qm]));
}

// U2(a b) = - [ ubar Jslash(J(a b)) + U1(a) Jslash(b) ] (qslash + m) / (q^2 - m^2)
template <typename R, class T> __device__ __forceinline__ void rc_task_u2(RcWarpT<R>& w, const T& t)
{
    W4<R> acc = row_jslash(rc_ld(w, t.f(4)), rc_ld(w, t.f(5)));
    w4_fma(acc, rc_sign<R>(t.f(3), 0), row_jslash(rc_ld(w, t.f(1)), rc_ld(w, t.f(2))));
    const int qm = t.f(6);
    R q[4];
    rc_qmom(w, qm, q);
    rc_st(w, t.f(0), row_qprop(acc, q, w.r.mt, -w.r.iQ[qm]));
}

// W2(c d) = Jslash(J(c d)) v + Jslash(c) Vr1(d)   (no propagator at its left end)
template <typename R, class T> __device__ __forceinline__ void rc_task_w2(RcWarpT<R>& w, const T& t)
{
    W4<R> acc = col_jslash(rc_ld(w, t.f(4)), rc_ld(w, t.f(5)));
    w4_fma(acc, rc_sign<R>(t.f(2), 0), col_jslash(rc_ld(w, t.f(1)), rc_ld(w, t.f(3))));
    rc_st(w, t.f(0), acc);
}

// X = row gamma^mu col
template <typename R, class T> __device__ __forceinline__ void rc_task_x(RcWarpT<R>& w, const T& t)
{
    rc_st(w, t.f(0), ffv_cur(rc_ld(w, t.f(1)), rc_ld(w, t.f(2)), R(1.0f)));
}

// the steps of one routine: lane takes task [step][lane] (field 0 = 0xFFFF: none)
#define MF_RC_STEPS(TYPE, FN)                                                                              \
    for (int s_ = 0; s_ < rcT::STEPS_##TYPE; ++s_) {                                                      \
        const auto t_ = rc_task<rcT::NQ_##TYPE>(&rcT::task_##TYPE[0][0][0][0], s_, lane);                  \
        if (t_.f(0) != 0xFFFF) FN<R>(w, t_);                                                               \
    }

// Phase 1: every current of the event's store, stage by stage (a __syncwarp between
// stages: a stage reads only the slots of earlier ones).  CTA_SYNC: every warp of the CTA
// calls together, and a CTA barrier between the stages keeps the warps on the same code.
template <typename R, bool CTA_SYNC>
__device__ __forceinline__ void rc_currents(RcWarpT<R>& w, int lane)
{
    MF_RC_STEPS(EXT, rc_task_ext)
    __syncwarp();
    MF_RC_STEPS(J2, rc_task_j2)
    if (CTA_SYNC) __syncthreads(); else __syncwarp();
    MF_RC_STEPS(J3, rc_task_j3)
    MF_RC_STEPS(U1, rc_task_u1)
    MF_RC_STEPS(VR1, rc_task_vr1)
    if (CTA_SYNC) __syncthreads(); else __syncwarp();
    MF_RC_STEPS(J4, rc_task_j4)
    if (CTA_SYNC) __syncthreads();
    MF_RC_STEPS(U2, rc_task_u2)
    MF_RC_STEPS(W2, rc_task_w2)
    MF_RC_STEPS(X, rc_task_x)
    if (CTA_SYNC) __syncthreads(); else __syncwarp();
}
#undef MF_RC_STEPS

// row spinor times column spinor
template <typename R> __device__ __forceinline__ cx<R> rc_rowcol(const W4<R>& a, const W4<R>& b)
{
    cx<R> s = cmul(a.c[0], b.c[0]);
    s = cfma(a.c[1], b.c[1], s);
    s = cfma(a.c[2], b.c[2], s);
    return cfma(a.c[3], b.c[3], s);
}

// Phase 2: the partial amplitudes of orderings 2 pc and 2 pc + 1 (an ordering and its
// reverse) for lane l's configuration ih = 1 + 2 l, five contractions each.  lt: the per-lane
// words (rc_gg_ttgg::lane_terms) at this lane, in shared memory (GLOBAL false) or the
// generated table itself (read through the L1 cache).  The third term of every ordering is
// X(ubar, v) . J(sigma), X(ubar, v) the lane's jq (loaded once per event), and the pair's two
// third terms contract the same slots (the generator checks it): computed once.
template <typename R> __device__ __forceinline__ W4<R> rc_jq(const RcWarpT<R>& w, const uint32_t* lt, bool global)
{
    const uint32_t word = global ? __ldg(lt + 2 * 32) : lt[2 * 32];
    return rc_ld(w, (int)(word & 0xFFFu));
}
template <typename R, bool GLOBAL>
__device__ __forceinline__ void rc_amp_pair(const RcWarpT<R>& w, const uint32_t* lt, int pc, const W4<R>& jq,
                                            cx<R> (&a)[2])
{
    cx<R> v3 = mkc(R(0.0f), R(0.0f));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        cx<R> acc = mkc(R(0.0f), R(0.0f));
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const uint32_t word = GLOBAL ? __ldg(lt + ((2 * pc + h) * 5 + k) * 32) : lt[((2 * pc + h) * 5 + k) * 32];
            cx<R> v;
            if (k == 2) {
                if (h == 0) v3 = cdot(jq, rc_ld(w, (int)((word >> 12) & 0xFFFu)));
                v = v3;
            } else {
                const W4<R> x = rc_ld(w, (int)(word & 0xFFFu)), y = rc_ld(w, (int)((word >> 12) & 0xFFFu));
                v = k == 0 ? rc_rowcol(x, y) : cdot(x, y);
            }
            const R sg = R(((word >> 24) & 1u) ? -1.0f : 1.0f);
            acc.r = fma(sg, v.r, acc.r);
            acc.i = fma(sg, v.i, acc.i);
        }
        a[h] = acc;
    }
}

// Lane l's 24 partial amplitudes of configuration ih = 1 + 2 l, two at a time into its TMEM
// lane (bf16 pieces of the A operand and the FP32 u of the colour sum); lane_base: tc_rc_lane.
template <bool GLOBAL>
__device__ __forceinline__ void rc_amplitudes(const RcWarp& w, const uint32_t* terms, int lane, uint32_t lane_base)
{
    const uint32_t* lt = terms + lane;
    const W4<float> jq = rc_jq(w, lt, GLOBAL);
#pragma unroll 1
    for (int pc = 0; pc < rcT::NPERM / 2; ++pc) {
        cx<float> a[2];
        rc_amp_pair<float, GLOBAL>(w, lt, pc, jq, a);
        tc_rc_put_pair(lane_base, pc, a[0].r, a[0].i, a[1].r, a[1].i);
    }
}

// ---------------------------------------------------------------- the integrand's schedule 4

template <> struct RcTraits<Me_gg_ttgg> {
    // the colour matrix times 54 in the recursion's flow order (orderings paired with their reverses)
    __device__ static const short* colour54() { return rcT::colour54; }
    static constexpr size_t warp_bytes() { return sizeof(RcWarp); }
    // CTAs of 256 threads keep the contraction words in shared memory; CTAs of 128 threads
    // (two per SM) read them through the L1 cache and leave the room to the second CTA
    static constexpr size_t extra_bytes(int tpb) { return tpb == 256 ? RC_TERM_BYTES : 0; }
};
template <> struct HasRc<Me_gg_ttgg> : std::true_type {};

// after tc_setup (every thread of the CTA calls): the zero padding of the A operand and
// the per-lane contraction words in shared memory
template <class P, int TPB>
__device__ void rc_cta_setup(unsigned char* smem_raw, TcCta* tc)
{
    using L = SmemLayout<P, float, TPB, 2>;
    static_assert(L::LH_EXTRA_OFF % 16 == 0, "aligned table");
    tc_rc_zero_pad<P::Me::NCOL>(tc);
    if constexpr (RcTraits<typename P::Me>::extra_bytes(TPB) > 0) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(smem_raw + L::LH_EXTRA_OFF);
        for (int i = threadIdx.x; i < rcT::TERM_WORDS; i += TPB) dst[i] = __ldg(&rcT::lane_terms[0][0][0] + i);
    }
    __syncthreads();
}

// |M|^2 of a batch of queued events (every thread of the CTA calls; as lh_batch_me2): the
// events' records, formed from their double-float momenta, go to this CTA's region of
// kp.inv_rec, then warp w evaluates events
// w, w + WARPS, ... (a warp without an event in a round repeats entry 0 and discards it,
// so that every warp takes part in the CTA barriers of each round): the invariants one
// subset per lane, the recycled currents, each lane's amplitudes into its TMEM lane, the
// colour sum of all 256 rows on the tensor cores, and the event's sum over its lanes by a
// fixed shuffle tree.  Returns this thread's event's |M|^2 (meaningful where mine).
template <class P, int TPB>
__device__ double rc_batch_me2(const KParams& kp, unsigned char* smem_raw, TcCta* tc, double* sme, int take, bool mine,
                               const Df (&pm)[P::NEXT][4])
{
    using ME = typename P::Me;
    using L = SmemLayout<P, float, TPB, 2>;
    constexpr int WARPS = TPB / 32, NEXT = P::NEXT;
    static_assert(NEXT == 6 && ME::NCOL == rcT::NPERM && (TPB == 128 || TPB == 256),
                  "g g -> t tbar g g, one TMEM lane per thread");
    constexpr bool GLOBAL_TERMS = RcTraits<ME>::extra_bytes(TPB) == 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // this CTA's records, field-major: word f of entry j at grec[f TPB + j]
    float* grec = kp.inv_rec + (size_t)blockIdx.x * LH_INV_WORDS_MAX * TPB;
    if (mine) {
        RcRec rec;
        rc_record(pm, kp.kd.mt, rec);
        const float* wsrc = reinterpret_cast<const float*>(&rec);
#pragma unroll
        for (int f = 0; f < RC_REC_WORDS; ++f) grec[(size_t)f * TPB + tid] = wsrc[f];
    }
    __syncthreads();
    RcWarp& w = *reinterpret_cast<RcWarp*>(smem_raw + L::LH_REC_OFF + (size_t)warp * L::LH_REC_STRIDE);
    const uint32_t* terms = GLOBAL_TERMS ? &rcT::lane_terms[0][0][0]
                                         : reinterpret_cast<const uint32_t*>(smem_raw + L::LH_EXTRA_OFF);
    const uint32_t lb = tc_rc_lane(tc);
    const int nsub = (take + WARPS - 1) / WARPS;
    for (int sub = 0; sub < nsub; ++sub) {
        const int j = sub * WARPS + warp;
        const int jj = j < take ? j : 0;
        float* wwords = reinterpret_cast<float*>(&w.r);
        for (int f = lane; f < RC_REC_WORDS; f += 32) wwords[f] = grec[(size_t)f * TPB + jj];
        __syncwarp();
        rc_currents<float, true>(w, lane);
        rc_amplitudes<GLOBAL_TERMS>(w, terms, lane, lb);
        float mh = tc_rc_colour_sum<ME::NCOL>(tc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mh += __shfl_xor_sync(0xffffffffu, mh, off);
        if (lane == 0 && j < take) sme[j] = (double)mh;
        __syncwarp();
    }
    __syncthreads();
    const float acc = 2.0f * (float)sme[tid < take ? tid : 0];
    double gk = 1.0;
    for (int i = 0; i < ME::NGLUON; ++i) gk = gk * (kp.gs * kp.gs);
    __syncthreads();   // sme is reused by the caller
    return (double)acc / ME::COLOUR_DEN * gk * ME::AVG * ME::SYM;
}

// ---------------------------------------------------------------- the m_t derivative pass

// Per-lane colour sum of one configuration and its derivative: with y = 54 C A (the value
// parts of the amplitudes), |M_h|^2 54 = Re(A^+ y) and d|M_h|^2 54 = 2 Re(dA^+ y) (C real and
// symmetric).  row: the lane's 24 amplitudes as (Re A, Re dA, Im A, Im dA), 4 floats each.
__device__ __forceinline__ void rc_colour_dual(const float* row, float& me, float& dme)
{
    constexpr int N = rcT::NPERM;
    float ar[N], ai[N];
#pragma unroll
    for (int s = 0; s < N; ++s) { ar[s] = row[4 * s]; ai[s] = row[4 * s + 2]; }
    float v = 0.0f, d = 0.0f;
#pragma unroll
    for (int t = 0; t < N; ++t) {
        float yr = 0.0f, yi = 0.0f;
#pragma unroll
        for (int s = 0; s < N; ++s) {
            yr = fmaf(rcT::colour[t * N + s], ar[s], yr);
            yi = fmaf(rcT::colour[t * N + s], ai[s], yi);
        }
        v = fmaf(ar[t], yr, fmaf(ai[t], yi, v));
        d = fmaf(row[4 * t + 1], yr, fmaf(row[4 * t + 3], yi, d));
    }
    me = v;
    dme = 2.0f * d;
}

// shared memory of the derivative pass: RC_GRAD_WARPS warp states, the lanes' amplitude rows,
// the VEGAS grid, per-event results and reductions
constexpr int RC_GRAD_TPB = 128, RC_GRAD_WARPS = RC_GRAD_TPB / 32, RC_GRAD_ROW = 4 * rcT::NPERM + 1;
__host__ __device__ constexpr size_t rc_grad_warp_bytes() { return (sizeof(RcWarpT<Dual<float>>) + 15) & ~(size_t)15; }
__host__ __device__ constexpr size_t rc_grad_rows_off() { return RC_GRAD_WARPS * rc_grad_warp_bytes(); }
__host__ __device__ constexpr size_t rc_grad_grid_off()
{
    return (rc_grad_rows_off() + sizeof(float) * RC_GRAD_TPB * RC_GRAD_ROW + 15) & ~(size_t)15;
}
template <int D> __host__ __device__ constexpr size_t rc_grad_smem(int nb)
{
    return rc_grad_grid_off() + sizeof(double) * (D * (nb + 1) + 2 * RC_GRAD_TPB + 4 * RC_GRAD_WARPS) +
           sizeof(int) * RC_GRAD_TPB;
}

// The m_t derivative pass of g g -> t tbar g g by the helicity-recycled recursion in forward
// mode: each thread carries one event's kinematics with the m_t tangent (Dual<double>: the
// parton map, RAMBO's mass rescaling, the scale and the PDFs) and, if it passes, forms its
// record with tangents (Dual<float> words) into this CTA's region of kp.inv_rec; then warp w
// evaluates the round's passing events w, w + 4, ...: the recycled currents and the 24
// partial amplitudes of each lane's configuration in dual numbers, the colour sum per lane,
// and the event's |M|^2 and derivative along (dp/dm_t, dm_t = 1) summed over its lanes.  Per
// CTA the same four sums as grad_kernel: sum w/N, sum dw/N, sum (dw/N)^2, k sum w/(N alpha_s).
// Every CTA needs a whole record region: CTAs beyond kp.inv_ctas write zero sums and the
// others share the events among themselves.
template <class P, int SYM_DEN>
__global__ void __launch_bounds__(RC_GRAD_TPB, 1) rc_grad_kernel(KParams kp, double* partials, int k_as, double alpha_s)
{
    using S = Dual<double>;
    using R = Dual<float>;
    constexpr int D = P::D, NEXT = P::NEXT, TPB = RC_GRAD_TPB, WARPS = RC_GRAD_WARPS, NW = rc_rec_words<R>();
    static_assert(NEXT == 6 && NW * TPB <= LH_INV_WORDS_MAX * LH_TPB, "a record region holds the CTA's dual records");
    extern __shared__ __align__(128) unsigned char mf_rcg_smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwork = (int)gridDim.x < kp.inv_ctas ? (int)gridDim.x : kp.inv_ctas;
    if (kp.inv_rec == nullptr || nwork < 1 || (int)blockIdx.x >= nwork) {
        if (tid == 0 && kp.dev_err && (kp.inv_rec == nullptr || nwork < 1)) atomicExch(kp.dev_err, 1u);
        if (tid < 4) partials[(size_t)blockIdx.x * 4 + tid] = 0.0;
        return;
    }
    auto& w = *reinterpret_cast<RcWarpT<R>*>(mf_rcg_smem + (size_t)warp * rc_grad_warp_bytes());
    float* rows = reinterpret_cast<float*>(mf_rcg_smem + rc_grad_rows_off());
    double* sgrid = reinterpret_cast<double*>(mf_rcg_smem + rc_grad_grid_off());
    double* sres = sgrid + D * (kp.nb + 1);            // [TPB][2]: |M|^2 and its derivative
    double* sred = sres + 2 * TPB;                      // [WARPS][4]
    int* smask = reinterpret_cast<int*>(sred + 4 * WARPS);
    float* grec = kp.inv_rec + (size_t)blockIdx.x * LH_INV_WORDS_MAX * LH_TPB;   // [NW][TPB]
    for (int i = tid; i < D * (kp.nb + 1); i += TPB) sgrid[i] = kp.grid[i];
    __syncthreads();
    double norm = 2.0 / (rcT::COLOUR_DEN * 256.0 * SYM_DEN);   // parity mirrors, colour, averages
    for (int i = 0; i < 4; ++i) norm *= kp.gs * kp.gs;
    double acc[4] = { 0.0, 0.0, 0.0, 0.0 };
    const long long n = kp.n_events;
    const S mt(kp.mt, 1.0);
    const uint32_t* lt = &rcT::lane_terms[0][0][0] + lane;
    float* row = rows + (size_t)tid * RC_GRAD_ROW;
    for (long long base = (long long)blockIdx.x * TPB; base < n; base += (long long)nwork * TPB) {
        const long long e = base + tid;
        int pass = 0;
        S pref = S(0.0);
        if (e < n) {
            EventOut<D> o;
            S pm[NEXT][4];
            kinematics_tops_t<P, S>(kp, sgrid, kp.pdf, (unsigned long long)(kp.ev_offset + e), mt, o, pm, pref);
            pass = o.mask;
            if (pass) {
                RcRecT<R> rec;
                rc_record<R>(pm, mt, rec);
                const float* wsrc = reinterpret_cast<const float*>(&rec);
#pragma unroll 8
                for (int f = 0; f < NW; ++f) grec[(size_t)f * TPB + tid] = wsrc[f];
            }
        }
        smask[tid] = pass;
        __syncthreads();
        for (int j = warp; j < TPB; j += WARPS) {
            if (!smask[j]) continue;                    // the same j for the whole warp
            float* wwords = reinterpret_cast<float*>(&w.r);
            for (int f = lane; f < NW; f += 32) wwords[f] = grec[(size_t)f * TPB + j];
            __syncwarp();
            rc_currents<R, false>(w, lane);
            const W4<R> jq = rc_jq(w, lt, true);
#pragma unroll 1
            for (int pc = 0; pc < rcT::NPERM / 2; ++pc) {
                cx<R> a[2];
                rc_amp_pair<R, true>(w, lt, pc, jq, a);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float* q = row + 4 * (2 * pc + h);
                    q[0] = a[h].r.v; q[1] = a[h].r.d; q[2] = a[h].i.v; q[3] = a[h].i.d;
                }
            }
            float me, dme;
            rc_colour_dual(row, me, dme);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                me += __shfl_xor_sync(0xffffffffu, me, off);
                dme += __shfl_xor_sync(0xffffffffu, dme, off);
            }
            if (lane == 0) { sres[2 * j] = (double)me * norm; sres[2 * j + 1] = (double)dme * norm; }
            __syncwarp();
        }
        __syncthreads();
        if (pass) {
            const double me = sres[2 * tid], dme = sres[2 * tid + 1];
            const double wv = pref.v * me, dw = pref.d * me + pref.v * dme;
            if (isfinite(wv) && isfinite(dw)) {
                const double wn = wv * kp.inv_n, dn = dw * kp.inv_n;
                acc[0] += wn;
                acc[1] += dn;
                acc[2] += dn * dn;
                acc[3] += k_as * wn / alpha_s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sred[4 * warp + k] = v;
    }
    __syncthreads();
    if (tid < 4) {
        double v = 0.0;
        for (int k = 0; k < WARPS; ++k) v += sred[4 * k + tid];
        partials[(size_t)blockIdx.x * 4 + tid] = v;
    }
}

}  // namespace mf


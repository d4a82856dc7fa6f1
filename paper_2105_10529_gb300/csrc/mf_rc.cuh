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
// mf_helas.cuh and mf_bg.cuh; the invariants (subset momenta and inverse propagator
// denominators in FP64, stored as FP32) are those of bg_event_invariants.
#pragma once
#include <cstdint>
#include "mf_bg.cuh"
#include "mf_integrand.cuh"
#include "mf_tc.cuh"
#include "generated/me_gg_ttgg.cuh"
#include "generated/rc_gg_ttgg.cuh"

namespace mf {

namespace rcT = rc_gg_ttgg;

// one warp's shared-memory state: the store first (16-byte aligned slots), then the
// per-event invariants in the field names of bg_event_invariants
struct RcWarp {
    W4<float> W[rcT::NSLOT];
    float P[16][4];
    float iP2[16];
    float Q[16][4];
    float iQ[16];
    float e1[4][3], e2[4][3];
    FermionBasis<float> fb3, fb4;
    float mt;
};

// the combination offset of lane l for a lane-bit mask m: the bits of l selected by m,
// packed (a table of 32 x 32 bytes in shared memory, filled once per CTA)
constexpr int RC_OFFTAB_BYTES = 32 * 32;
__device__ __forceinline__ void rc_fill_offtab(uint8_t* tab)
{
    for (int i = threadIdx.x; i < RC_OFFTAB_BYTES; i += blockDim.x) {
        const int m = i >> 5, l = i & 31;
        int r = 0, j = 0;
        for (int b = 0; b < 5; ++b)
            if ((m >> b) & 1) r |= ((l >> b) & 1) << j++;
        tab[i] = (uint8_t)r;
    }
}

__device__ __forceinline__ W4<float> rc_ld(const W4<float>* p)
{
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    W4<float> w;
    w.c[0] = mkc(a.x, a.y); w.c[1] = mkc(a.z, a.w); w.c[2] = mkc(b.x, b.y); w.c[3] = mkc(b.z, b.w);
    return w;
}
__device__ __forceinline__ void rc_st(W4<float>* p, const W4<float>& w)
{
    reinterpret_cast<float4*>(p)[0] = make_float4(w.c[0].r, w.c[0].i, w.c[1].r, w.c[1].i);
    reinterpret_cast<float4*>(p)[1] = make_float4(w.c[2].r, w.c[2].i, w.c[3].r, w.c[3].i);
}
__device__ __forceinline__ void rc_mom(const RcWarp& w, int m, float (&k)[4])
{
    const float4 v = *reinterpret_cast<const float4*>(&w.P[m][0]);
    k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
}
__device__ __forceinline__ void rc_qmom(const RcWarp& w, int m, float (&q)[4])
{
    const float4 v = *reinterpret_cast<const float4*>(&w.Q[m][0]);
    q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
}
__device__ __forceinline__ float rc_sign(unsigned bits, int b) { return (bits >> b) & 1u ? -1.0f : 1.0f; }

// Jslash times a column spinor: (Sigma(J) d ; Sigmabar(J) c) for the column (c ; d)
__device__ __forceinline__ W4<float> col_jslash(const W4<float>& J, const W4<float>& f)
{
    const M2<float> S = sig(J), Sb = sigbar(J);
    W4<float> o;
    mcol(S, f.c[2], f.c[3], o.c[0], o.c[1]);
    mcol(Sb, f.c[0], f.c[1], o.c[2], o.c[3]);
    return o;
}
__device__ __forceinline__ void w4_fma(W4<float>& acc, float s, const W4<float>& x)
{
#pragma unroll
    for (int m = 0; m < 4; ++m) { acc.c[m].r = fmaf(s, x.c[m].r, acc.c[m].r); acc.c[m].i = fmaf(s, x.c[m].i, acc.c[m].i); }
}
__device__ __forceinline__ void w4_acc(W4<float>& acc, const W4<float>& x)
{
#pragma unroll
    for (int m = 0; m < 4; ++m) { acc.c[m].r += x.c[m].r; acc.c[m].i += x.c[m].i; }
}

// ---------------------------------------------------------------- the routines of phase 1
// t: this lane's task, the fields of rc_tables.TASK_FIELDS (slot indices into w.W)

__device__ __forceinline__ void rc_task_ext(RcWarp& w, const uint16_t* t)
{
    const int code = __ldg(t + 1), hel = __ldg(t + 2) ? 1 : -1;
    W4<float> o;
    if (code < 4) o = ext_gluon(w.e1[code], w.e2[code], hel, code >= 2);
    else if (code == 4) o = ext_ubar(w.fb3, hel);
    else o = ext_v(w.fb4, hel);
    rc_st(&w.W[__ldg(t)], o);
}

__device__ __forceinline__ void rc_task_j2(RcWarp& w, const uint16_t* t)
{
    float ka[4], kb[4];
    rc_mom(w, __ldg(t + 4), ka);
    rc_mom(w, __ldg(t + 5), kb);
    const W4<float> o = vvv_cur(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)]), ka, kb, -w.iP2[__ldg(t + 6)]);
    rc_st(&w.W[__ldg(t)], o);
}

// J(x y z) = [ - V3(J(x), J(y z)) - V3(J(x y), J(z)) + V4(J(x), J(y), J(z)) ] / P^2
__device__ __forceinline__ void rc_task_j3(RcWarp& w, const uint16_t* t)
{
    const unsigned sg = __ldg(t + 6);
    const W4<float> x = rc_ld(&w.W[__ldg(t + 1)]), y = rc_ld(&w.W[__ldg(t + 2)]), z = rc_ld(&w.W[__ldg(t + 3)]);
    float k1[4], k2[4];
    rc_mom(w, __ldg(t + 7), k1);
    rc_mom(w, __ldg(t + 8), k2);
    W4<float> acc = vvv_cur(x, rc_ld(&w.W[__ldg(t + 5)]), k1, k2, -rc_sign(sg, 0));
    rc_mom(w, __ldg(t + 9), k1);
    rc_mom(w, __ldg(t + 10), k2);
    w4_acc(acc, vvv_cur(rc_ld(&w.W[__ldg(t + 4)]), z, k1, k2, -rc_sign(sg, 1)));
    v4_add(acc, x, y, z, 1.0f);
    const float ip = w.iP2[__ldg(t + 11)];
    W4<float> o;
#pragma unroll
    for (int m = 0; m < 4; ++m) o.c[m] = cscale(acc.c[m], ip);
    rc_st(&w.W[__ldg(t)], o);
}

// J(w x y z): three V3 splits (w | x y z), (w x | y z), (w x y | z) and three V4 splits
// (w, x, y z), (w, x y, z), (w x, y, z)
__device__ __forceinline__ void rc_task_j4(RcWarp& w, const uint16_t* t)
{
    const unsigned sg = __ldg(t + 10);
    float k1[4], k2[4];
    W4<float> acc;
    {
        rc_mom(w, __ldg(t + 11), k1);
        rc_mom(w, __ldg(t + 12), k2);
        acc = vvv_cur(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 9)]), k1, k2, -rc_sign(sg, 0));
    }
    {
        rc_mom(w, __ldg(t + 13), k1);
        rc_mom(w, __ldg(t + 14), k2);
        w4_acc(acc, vvv_cur(rc_ld(&w.W[__ldg(t + 5)]), rc_ld(&w.W[__ldg(t + 7)]), k1, k2, -rc_sign(sg, 1)));
    }
    {
        rc_mom(w, __ldg(t + 15), k1);
        rc_mom(w, __ldg(t + 16), k2);
        w4_acc(acc, vvv_cur(rc_ld(&w.W[__ldg(t + 8)]), rc_ld(&w.W[__ldg(t + 4)]), k1, k2, -rc_sign(sg, 2)));
    }
    v4_add(acc, rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)]), rc_ld(&w.W[__ldg(t + 7)]), rc_sign(sg, 3));
    v4_add(acc, rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 6)]), rc_ld(&w.W[__ldg(t + 4)]), rc_sign(sg, 4));
    v4_add(acc, rc_ld(&w.W[__ldg(t + 5)]), rc_ld(&w.W[__ldg(t + 3)]), rc_ld(&w.W[__ldg(t + 4)]), rc_sign(sg, 5));
    const float ip = w.iP2[__ldg(t + 17)];
    W4<float> o;
#pragma unroll
    for (int m = 0; m < 4; ++m) o.c[m] = cscale(acc.c[m], ip);
    rc_st(&w.W[__ldg(t)], o);
}

// U1(a) = - ubar Jslash(a) (qslash + m) / (q^2 - m^2), q = p_t - K_a
__device__ __forceinline__ void rc_task_u1(RcWarp& w, const uint16_t* t)
{
    const int qm = __ldg(t + 3);
    float q[4];
    rc_qmom(w, qm, q);
    rc_st(&w.W[__ldg(t)], ffv_row(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)]), q, w.mt, -w.iQ[qm]));
}

// Vr1(d) = - (qslash + m) Jslash(d) v / (q^2 - m^2), q = p_t - (every gluon but d)
__device__ __forceinline__ void rc_task_vr1(RcWarp& w, const uint16_t* t)
{
    const int qm = __ldg(t + 3);
    float q[4];
    rc_qmom(w, qm, q);
    rc_st(&w.W[__ldg(t)], ffv_col(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)]), q, w.mt, -w.iQ[qm]));
}

// U2(a b) = - [ ubar Jslash(J(a b)) + U1(a) Jslash(b) ] (qslash + m) / (q^2 - m^2)
__device__ __forceinline__ void rc_task_u2(RcWarp& w, const uint16_t* t)
{
    W4<float> acc = row_jslash(rc_ld(&w.W[__ldg(t + 4)]), rc_ld(&w.W[__ldg(t + 5)]));
    w4_fma(acc, rc_sign(__ldg(t + 3), 0), row_jslash(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)])));
    const int qm = __ldg(t + 6);
    float q[4];
    rc_qmom(w, qm, q);
    rc_st(&w.W[__ldg(t)], row_qprop(acc, q, w.mt, -w.iQ[qm]));
}

// W2(c d) = Jslash(J(c d)) v + Jslash(c) Vr1(d)   (no propagator at its left end)
__device__ __forceinline__ void rc_task_w2(RcWarp& w, const uint16_t* t)
{
    W4<float> acc = col_jslash(rc_ld(&w.W[__ldg(t + 4)]), rc_ld(&w.W[__ldg(t + 5)]));
    w4_fma(acc, rc_sign(__ldg(t + 2), 0), col_jslash(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 3)])));
    rc_st(&w.W[__ldg(t)], acc);
}

// X = row gamma^mu col
__device__ __forceinline__ void rc_task_x(RcWarp& w, const uint16_t* t)
{
    rc_st(&w.W[__ldg(t)], ffv_cur(rc_ld(&w.W[__ldg(t + 1)]), rc_ld(&w.W[__ldg(t + 2)]), 1.0f));
}

// the steps of one routine: lane takes task [step][lane] (out = 0xFFFF: none)
#define MF_RC_STEPS(TYPE, FN)                                                            \
    for (int s_ = 0; s_ < rcT::STEPS_##TYPE; ++s_) {                                    \
        const uint16_t* t_ = &rcT::task_##TYPE[s_][lane][0];                            \
        if (__ldg(t_) != 0xFFFFu) FN(w, t_);                                            \
    }

// Phase 1: every current of the event's store, stage by stage (a __syncwarp between
// stages: a stage reads only the slots of earlier ones).  CTA_SYNC: every warp of the CTA
// calls together, and a CTA barrier between the stages keeps the warps on the same code.
template <bool CTA_SYNC>
__device__ __forceinline__ void rc_currents(RcWarp& w, int lane)
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
__device__ __forceinline__ cx<float> rc_rowcol(const W4<float>& a, const W4<float>& b)
{
    cx<float> s = cmul(a.c[0], b.c[0]);
    s = cfma(a.c[1], b.c[1], s);
    s = cfma(a.c[2], b.c[2], s);
    return cfma(a.c[3], b.c[3], s);
}

// Phase 2: lane l's 24 partial amplitudes of configuration ih = 1 + 2 l, two orderings
// at a time into its TMEM lane (bf16 pieces of the A operand and the FP32 u of the
// colour sum).  offtab: rc_fill_offtab's table; lane_base: tc_rc_lane.
__device__ __forceinline__ void rc_amplitudes(const RcWarp& w, const uint8_t* offtab, int lane, uint32_t lane_base)
{
#pragma unroll 1
    for (int pc = 0; pc < rcT::NPERM / 2; ++pc) {
        float re[2], im[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint16_t* tr = &rcT::terms[2 * pc + h][0][0];
            cx<float> acc = mkc(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int sa = tr[6 * k + 1] + offtab[tr[6 * k + 2] * 32 + lane];
                const int sb = tr[6 * k + 3] + offtab[tr[6 * k + 4] * 32 + lane];
                const W4<float> x = rc_ld(&w.W[sa]), y = rc_ld(&w.W[sb]);
                const cx<float> v = k == 0 ? rc_rowcol(x, y) : cdot(x, y);
                const float s = tr[6 * k + 5] ? -1.0f : 1.0f;
                acc.r = fmaf(s, v.r, acc.r);
                acc.i = fmaf(s, v.i, acc.i);
            }
            re[h] = acc.r;
            im[h] = acc.i;
        }
        tc_rc_put_pair(lane_base, pc, re[0], im[0], re[1], im[1]);
    }
}

// ---------------------------------------------------------------- the integrand's schedule 4

template <> struct RcTraits<Me_gg_ttgg> {
    static constexpr size_t warp_bytes() { return sizeof(RcWarp); }
    static constexpr size_t extra_bytes() { return RC_OFFTAB_BYTES; }
};
template <> struct HasRc<Me_gg_ttgg> : std::true_type {};

// after tc_setup (every thread of the CTA calls): the zero padding of the A operand and
// the combination-offset table
template <class P, int TPB>
__device__ void rc_cta_setup(unsigned char* smem_raw, TcCta* tc)
{
    using L = SmemLayout<P, float, TPB, 2>;
    tc_rc_zero_pad<P::Me::NCOL>(tc);
    rc_fill_offtab(smem_raw + L::LH_EXTRA_OFF);
    __syncthreads();
}

// |M|^2 of a batch of queued events (every thread of the CTA calls; as lh_batch_me2): the
// events' FP64 momenta go to this CTA's region of kp.inv_rec, then warp w evaluates events
// w, w + WARPS, ... (a warp without an event in a round repeats entry 0 and discards it,
// so that every warp takes part in the CTA barriers of each round): the invariants one
// subset per lane, the recycled currents, each lane's amplitudes into its TMEM lane, the
// colour sum of all 256 rows on the tensor cores, and the event's sum over its lanes by a
// fixed shuffle tree.  Returns this thread's event's |M|^2 (meaningful where mine).
template <class P, int TPB>
__device__ double rc_batch_me2(const KParams& kp, unsigned char* smem_raw, TcCta* tc, double* sme, int take, bool mine,
                               const double (&pm)[P::NEXT][4])
{
    using ME = typename P::Me;
    using L = SmemLayout<P, float, TPB, 2>;
    constexpr int WARPS = TPB / 32, NEXT = P::NEXT;
    static_assert(NEXT == 6 && ME::NCOL == rcT::NPERM && TPB == LH_TPB, "g g -> t tbar g g, one TMEM lane per thread");
    static_assert(NEXT * 4 * TPB <= LH_INV_WORDS_MAX * LH_TPB / 2, "momenta fit the CTA's record region");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* grec = reinterpret_cast<double*>(kp.inv_rec + (size_t)blockIdx.x * LH_INV_WORDS_MAX * LH_TPB);
    if (mine) {
#pragma unroll
        for (int f = 0; f < NEXT * 4; ++f) grec[(size_t)f * TPB + tid] = pm[f >> 2][f & 3];
    }
    __syncthreads();
    RcWarp& w = *reinterpret_cast<RcWarp*>(smem_raw + L::LH_REC_OFF + (size_t)warp * L::LH_REC_STRIDE);
    const uint8_t* offtab = smem_raw + L::LH_EXTRA_OFF;
    const uint32_t lb = tc_rc_lane(tc);
    const int nsub = (take + WARPS - 1) / WARPS;
    for (int sub = 0; sub < nsub; ++sub) {
        const int j = sub * WARPS + warp;
        const int jj = j < take ? j : 0;
        double p[NEXT][4];
#pragma unroll
        for (int f = 0; f < NEXT * 4; ++f) p[f >> 2][f & 3] = grec[(size_t)f * TPB + jj];
        bg_event_invariants<4, float>(w, p, kp.mt, lane);
        __syncwarp();
        rc_currents<true>(w, lane);
        rc_amplitudes(w, offtab, lane, lb);
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

}  // namespace mf


// Generated by paper_2105_10529_gb300/gen/qcd_diagrams.py -- do not edit.
// gg_ttg: 16 Feynman diagrams (18 amplitudes with the four-gluon
// colour structures counted apart), 6 colour flows, 32 helicities.
// Wavefunction/vertex calls per helicity: {'vvv': 3, 'vvvv': 0, 'ffv_row': 3, 'ffv_col': 3, 'ffv_amp': 12, 'vvv_amp': 3, 'vvvv_amp': 1, 'ffv_cur': 1}
#pragma once
#include "mf_helas.cuh"
#include "mf_tc.cuh"
namespace mf {
struct Me_gg_ttg {
  static constexpr int NEXT = 5;
  static constexpr int NCOL = 6;
  static constexpr int NHEL = 32;
  static constexpr int NGLUON = 3;
  static constexpr int NDIAG = 16;
  static constexpr double COLOUR_DEN = 9.0;
  static constexpr double AVG = 1.0 / 256.0;
  static constexpr double SYM = 1.0;
  // colour sum on the tensor cores available (a dense 24 x 24 contraction)
  static constexpr bool TC_COLOUR = false;
  // helicity-independent per-event pieces
  // per-thread slot: internal momenta, FP64-computed inverse denominators,
  // polarisation bases and spinor pieces of the event (kept in shared memory)
  template <typename R> struct Inv {
    R K[7][4]; R p3[4]; R iG[4]; R iQ[6];
    R e1[3][3]; R e2[3][3]; FermionBasis<R> fb3, fb4; R mt;
    cx<R> jamp[6];   // colour-flow amplitudes of the helicity being summed
    float pad[2];
  };
  // averaged |M|^2 (spin/colour average and identical-particle factor included);
  // p: momenta (E,px,py,pz) incoming first: g, g, t, tbar, g...
  // slot: this thread's Inv<R> in shared memory, or null for a private local copy
  // SYNC: a CTA barrier after every helicity (every thread of the CTA must call)
  // R: float or double (or Dual of them for derivatives); the momenta, masses and
  // the result use the scalar S of the momenta: the matching FP64 scalar Widen<R>::type,
  // or Df (double-float) where the mixed-precision kinematics hand theirs on
  // TC: colour sum on the tensor cores (float, SYNC, CTAs of 128 or 256 threads; cta: the CTA's TcCta)
  // hpart, hparts: helicity split, this call sums every hparts-th evaluated helicity
  // from the hpart-th on (the caller adds the hparts partial sums)
  template <typename R, bool SYNC = false, bool TC = false, typename S = typename Widen<R>::type>
  __device__ static S me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt, typename NoDeduce<S>::type gs,
                         void* slot, void* cta = nullptr, int hpart = 0, int hparts = 1);
  template <typename R> static constexpr size_t slot_bytes() { return sizeof(Inv<R>); }
  // per-helicity averaged |M_h|^2 of all NHEL configurations into out[NHEL] (diagnostic)
  template <typename R>
  __device__ static void hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,
                                     typename Widen<R>::type gs, double* out);
};

// one helicity configuration: amplitudes, colour flows and (CSUM) the colour sum;
// out of line so that its register allocation sees only one helicity
template <typename R, bool CSUM = true>
__device__ __noinline__ R hel_gg_ttg(const Me_gg_ttg::Inv<R>& v, int ih)
{
    constexpr int NCOL = Me_gg_ttg::NCOL;
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
    // colour-flow amplitudes accumulate in the slot (shared memory), not in registers
    volatile cx<R>* jamp = reinterpret_cast<volatile cx<R>*>(const_cast<cx<R>*>(v.jamp));
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) { vset(jamp[c].r, R(0)); vset(jamp[c].i, R(0)); }
    W4<R> g0; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[0][j]); b[j] = ldv(v.e2[0][j]); }
      g0 = ext_gluon(a, b, HEL(0), false); }
    W4<R> g1; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[1][j]); b[j] = ldv(v.e2[1][j]); }
      g1 = ext_gluon(a, b, HEL(1), false); }
    W4<R> g2; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[2][j]); b[j] = ldv(v.e2[2][j]); }
      g2 = ext_gluon(a, b, HEL(4), true); }
    const W4<R> ub3 = ext_ubar(load_basis(v.fb3), HEL(2));
    const W4<R> v4 = ext_v(load_basis(v.fb4), HEL(3));
    const R k1_1[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k2_2[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w3 = vvv_cur(g0, g1, k1_1, k2_2, ldv(v.iG[0]));
    const R k1_4[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k4_5[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w6 = vvv_cur(g0, g2, k1_4, k4_5, ldv(v.iG[1]));
    const R k2_7[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k4_8[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w9 = vvv_cur(g1, g2, k2_7, k4_8, ldv(v.iG[2]));
    const R q1_10[4] = {ldv(v.p3[0]) - ldv(v.K[0][0]), ldv(v.p3[1]) - ldv(v.K[0][1]), ldv(v.p3[2]) - ldv(v.K[0][2]), ldv(v.p3[3]) - ldv(v.K[0][3])};
    const W4<R> w11 = ffv_row(ub3, g0, q1_10, ldv(v.mt), ldv(v.iQ[0]));
    const R q3_13[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w12 = ffv_col(g2, v4, q3_13, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a1 = ffv_amp(w11, w12, g1);
    jadd_pi(jamp[0], a1);
    const R q5_15[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w14 = ffv_col(g1, v4, q5_15, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a2 = ffv_amp(w11, w14, g2);
    jadd_pi(jamp[1], a2);
    const cx<R> a3 = ffv_amp(w11, v4, w9);
    jadd_pi(jamp[0], a3);
    jadd_mi(jamp[1], a3);
    const R q2_16[4] = {ldv(v.p3[0]) - ldv(v.K[1][0]), ldv(v.p3[1]) - ldv(v.K[1][1]), ldv(v.p3[2]) - ldv(v.K[1][2]), ldv(v.p3[3]) - ldv(v.K[1][3])};
    const W4<R> w17 = ffv_row(ub3, g1, q2_16, ldv(v.mt), ldv(v.iQ[1]));
    const cx<R> a4 = ffv_amp(w17, w12, g0);
    jadd_pi(jamp[2], a4);
    const R q6_19[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w18 = ffv_col(g0, v4, q6_19, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a5 = ffv_amp(w17, w18, g2);
    jadd_pi(jamp[3], a5);
    const cx<R> a6 = ffv_amp(w17, v4, w6);
    jadd_pi(jamp[2], a6);
    jadd_mi(jamp[3], a6);
    const R q4_20[4] = {ldv(v.p3[0]) - ldv(v.K[3][0]), ldv(v.p3[1]) - ldv(v.K[3][1]), ldv(v.p3[2]) - ldv(v.K[3][2]), ldv(v.p3[3]) - ldv(v.K[3][3])};
    const W4<R> w21 = ffv_row(ub3, g2, q4_20, ldv(v.mt), ldv(v.iQ[3]));
    const cx<R> a7 = ffv_amp(w21, w14, g0);
    jadd_pi(jamp[4], a7);
    const cx<R> a8 = ffv_amp(w21, w18, g1);
    jadd_pi(jamp[5], a8);
    const cx<R> a9 = ffv_amp(w21, v4, w3);
    jadd_pi(jamp[4], a9);
    jadd_mi(jamp[5], a9);
    const cx<R> a10 = ffv_amp(ub3, w12, w3);
    jadd_pi(jamp[0], a10);
    jadd_mi(jamp[2], a10);
    const cx<R> a11 = ffv_amp(ub3, w14, w6);
    jadd_pi(jamp[1], a11);
    jadd_mi(jamp[4], a11);
    const cx<R> a12 = ffv_amp(ub3, w18, w9);
    jadd_pi(jamp[3], a12);
    jadd_mi(jamp[5], a12);
    const W4<R> jq = ffv_cur(ub3, v4, ldv(v.iG[3]));
    const R k1_22[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k6_23[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const R k7_24[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R nkk7_24[4] = {-k7_24[0], -k7_24[1], -k7_24[2], -k7_24[3]};
    const cx<R> a13 = vvv_amp(g0, w9, jq, k1_22, k6_23, nkk7_24);
    jadd_pi(jamp[0], a13);
    jadd_mi(jamp[1], a13);
    jadd_mi(jamp[3], a13);
    jadd_pi(jamp[5], a13);
    const R k3_25[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k4_26[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k7_27[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R nkk7_27[4] = {-k7_27[0], -k7_27[1], -k7_27[2], -k7_27[3]};
    const cx<R> a14 = vvv_amp(w3, g2, jq, k3_25, k4_26, nkk7_27);
    jadd_pi(jamp[0], a14);
    jadd_mi(jamp[2], a14);
    jadd_mi(jamp[4], a14);
    jadd_pi(jamp[5], a14);
    const R k5_28[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k2_29[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k7_30[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R nkk7_30[4] = {-k7_30[0], -k7_30[1], -k7_30[2], -k7_30[3]};
    const cx<R> a15 = vvv_amp(w6, g1, jq, k5_28, k2_29, nkk7_30);
    jadd_pi(jamp[1], a15);
    jadd_mi(jamp[2], a15);
    jadd_pi(jamp[3], a15);
    jadd_mi(jamp[4], a15);
    cx<R> a16, a17, a18;
    vvvv_amp(g0, g1, g2, jq, a16, a17, a18);
    jadd_pi(jamp[0], a16);
    jadd_mi(jamp[2], a16);
    jadd_mi(jamp[4], a16);
    jadd_pi(jamp[5], a16);
    jadd_pi(jamp[1], a17);
    jadd_mi(jamp[2], a17);
    jadd_pi(jamp[3], a17);
    jadd_mi(jamp[4], a17);
    jadd_mi(jamp[0], a18);
    jadd_pi(jamp[1], a18);
    jadd_pi(jamp[3], a18);
    jadd_mi(jamp[5], a18);
    if constexpr (!CSUM) return R(0);   // the caller sums the colour flows left in the slot
    cx<R> J[NCOL];
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) J[c] = mkc(vget(jamp[c].r), vget(jamp[c].i));
    R me = R(0);
    { const R zr = R(64.0) * J[0].r + R(-16.0) * J[1].r + R(-16.0) * J[2].r + R(2.0) * J[3].r + R(2.0) * J[4].r + R(20.0) * J[5].r; const R zi = R(64.0) * J[0].i + R(-16.0) * J[1].i + R(-16.0) * J[2].i + R(2.0) * J[3].i + R(2.0) * J[4].i + R(20.0) * J[5].i;
      me = fma(J[0].r, zr, fma(J[0].i, zi, me)); }
    { const R zr = R(64.0) * J[1].r + R(2.0) * J[2].r + R(20.0) * J[3].r + R(-16.0) * J[4].r + R(2.0) * J[5].r; const R zi = R(64.0) * J[1].i + R(2.0) * J[2].i + R(20.0) * J[3].i + R(-16.0) * J[4].i + R(2.0) * J[5].i;
      me = fma(J[1].r, zr, fma(J[1].i, zi, me)); }
    { const R zr = R(64.0) * J[2].r + R(-16.0) * J[3].r + R(20.0) * J[4].r + R(2.0) * J[5].r; const R zi = R(64.0) * J[2].i + R(-16.0) * J[3].i + R(20.0) * J[4].i + R(2.0) * J[5].i;
      me = fma(J[2].r, zr, fma(J[2].i, zi, me)); }
    { const R zr = R(64.0) * J[3].r + R(2.0) * J[4].r + R(-16.0) * J[5].r; const R zi = R(64.0) * J[3].i + R(2.0) * J[4].i + R(-16.0) * J[5].i;
      me = fma(J[3].r, zr, fma(J[3].i, zi, me)); }
    { const R zr = R(64.0) * J[4].r + R(-16.0) * J[5].r; const R zi = R(64.0) * J[4].i + R(-16.0) * J[5].i;
      me = fma(J[4].r, zr, fma(J[4].i, zi, me)); }
    { const R zr = R(64.0) * J[5].r; const R zi = R(64.0) * J[5].i;
      me = fma(J[5].r, zr, fma(J[5].i, zi, me)); }
    return me;
#undef HEL
}

template <typename R, bool SYNC, bool TC, typename S>
__device__ __noinline__ S me2_gg_ttg_impl(const S* pflat, S mt, S gs, void* slot, void* cta, int hpart,
                                       int hparts)
{
    constexpr int NEXT = Me_gg_ttg::NEXT, NHEL = Me_gg_ttg::NHEL, NGLUON = Me_gg_ttg::NGLUON;
    constexpr double COLOUR_DEN = Me_gg_ttg::COLOUR_DEN, AVG = Me_gg_ttg::AVG, SYM = Me_gg_ttg::SYM;
    S p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    Me_gg_ttg::Inv<R> local;   // used when the caller has no shared-memory slot
    Me_gg_ttg::Inv<R>& v = slot ? *static_cast<Me_gg_ttg::Inv<R>*>(slot) : local;
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const S kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const S kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const S kd4[4] = {-p[4][0], -p[4][1], -p[4][2], -p[4][3]};
    const S kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    const S kd5[4] = {kd1[0] + kd4[0], kd1[1] + kd4[1], kd1[2] + kd4[2], kd1[3] + kd4[3]};
    const S kd6[4] = {kd2[0] + kd4[0], kd2[1] + kd4[1], kd2[2] + kd4[2], kd2[3] + kd4[3]};
    const S kd7[4] = {kd1[0] + kd2[0] + kd4[0], kd1[1] + kd2[1] + kd4[1], kd1[2] + kd2[2] + kd4[2], kd1[3] + kd2[3] + kd4[3]};
    for (int c = 0; c < 4; ++c) v.K[0][c] = R(kd1[c]);
    for (int c = 0; c < 4; ++c) v.K[1][c] = R(kd2[c]);
    for (int c = 0; c < 4; ++c) v.K[2][c] = R(kd3[c]);
    for (int c = 0; c < 4; ++c) v.K[3][c] = R(kd4[c]);
    for (int c = 0; c < 4; ++c) v.K[4][c] = R(kd5[c]);
    for (int c = 0; c < 4; ++c) v.K[5][c] = R(kd6[c]);
    for (int c = 0; c < 4; ++c) v.K[6][c] = R(kd7[c]);
    for (int c = 0; c < 4; ++c) v.p3[c] = R(p[2][c]);
    v.iG[0] = R(1.0 / mdot(kd3, kd3));
    v.iG[1] = R(1.0 / mdot(kd5, kd5));
    v.iG[2] = R(1.0 / mdot(kd6, kd6));
    v.iG[3] = R(1.0 / mdot(kd7, kd7));
    { const S q[4] = {p[2][0] - kd1[0], p[2][1] - kd1[1], p[2][2] - kd1[2], p[2][3] - kd1[3]};
      v.iQ[0] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd2[0], p[2][1] - kd2[1], p[2][2] - kd2[2], p[2][3] - kd2[3]};
      v.iQ[1] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd3[0], p[2][1] - kd3[1], p[2][2] - kd3[2], p[2][3] - kd3[3]};
      v.iQ[2] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd4[0], p[2][1] - kd4[1], p[2][2] - kd4[2], p[2][3] - kd4[3]};
      v.iQ[3] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd5[0], p[2][1] - kd5[1], p[2][2] - kd5[2], p[2][3] - kd5[3]};
      v.iQ[4] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd6[0], p[2][1] - kd6[1], p[2][2] - kd6[2], p[2][3] - kd6[3]};
      v.iQ[5] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { S a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[4], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[2][j] = R(a[j]); v.e2[2][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
    // Parity: flipping every helicity leaves the colour-summed |M_h|^2 of these
    // tree amplitudes unchanged, so the sum over all helicities is twice the
    // sum over the configurations with the first gluon at helicity +1.
    R acc = R(0);
#pragma unroll 1
    for (int ih = 1 + 2 * hpart; ih < NHEL; ih += 2 * hparts) {
        static_assert(!TC, "no tensor-core colour sum for this colour basis");
        acc += hel_gg_ttg<R>(v, ih);
        if (SYNC) __syncthreads();
    }
    acc *= R(2);
    S gk = S(1.0);
    for (int i = 0; i < NGLUON; ++i) gk = gk * (gs * gs);
    return S(acc) / COLOUR_DEN * gk * AVG * SYM;
}

template <typename R, bool SYNC, bool TC, typename S>
__device__ S Me_gg_ttg::me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt,
    typename NoDeduce<S>::type gs, void* slot, void* cta, int hpart, int hparts)
{
    return me2_gg_ttg_impl<R, SYNC, TC, S>(&p[0][0], mt, gs, slot, cta, hpart, hparts);
}

// the prologue of me2 alone: the event's helicity-independent pieces into v
template <typename R>
__device__ __forceinline__ void inv_gg_ttg(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,
                                       Me_gg_ttg::Inv<R>& v)
{
    using S = typename Widen<R>::type;
    constexpr int NEXT = Me_gg_ttg::NEXT;
    S p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const S kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const S kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const S kd4[4] = {-p[4][0], -p[4][1], -p[4][2], -p[4][3]};
    const S kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    const S kd5[4] = {kd1[0] + kd4[0], kd1[1] + kd4[1], kd1[2] + kd4[2], kd1[3] + kd4[3]};
    const S kd6[4] = {kd2[0] + kd4[0], kd2[1] + kd4[1], kd2[2] + kd4[2], kd2[3] + kd4[3]};
    const S kd7[4] = {kd1[0] + kd2[0] + kd4[0], kd1[1] + kd2[1] + kd4[1], kd1[2] + kd2[2] + kd4[2], kd1[3] + kd2[3] + kd4[3]};
    for (int c = 0; c < 4; ++c) v.K[0][c] = R(kd1[c]);
    for (int c = 0; c < 4; ++c) v.K[1][c] = R(kd2[c]);
    for (int c = 0; c < 4; ++c) v.K[2][c] = R(kd3[c]);
    for (int c = 0; c < 4; ++c) v.K[3][c] = R(kd4[c]);
    for (int c = 0; c < 4; ++c) v.K[4][c] = R(kd5[c]);
    for (int c = 0; c < 4; ++c) v.K[5][c] = R(kd6[c]);
    for (int c = 0; c < 4; ++c) v.K[6][c] = R(kd7[c]);
    for (int c = 0; c < 4; ++c) v.p3[c] = R(p[2][c]);
    v.iG[0] = R(1.0 / mdot(kd3, kd3));
    v.iG[1] = R(1.0 / mdot(kd5, kd5));
    v.iG[2] = R(1.0 / mdot(kd6, kd6));
    v.iG[3] = R(1.0 / mdot(kd7, kd7));
    { const S q[4] = {p[2][0] - kd1[0], p[2][1] - kd1[1], p[2][2] - kd1[2], p[2][3] - kd1[3]};
      v.iQ[0] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd2[0], p[2][1] - kd2[1], p[2][2] - kd2[2], p[2][3] - kd2[3]};
      v.iQ[1] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd3[0], p[2][1] - kd3[1], p[2][2] - kd3[2], p[2][3] - kd3[3]};
      v.iQ[2] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd4[0], p[2][1] - kd4[1], p[2][2] - kd4[2], p[2][3] - kd4[3]};
      v.iQ[3] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd5[0], p[2][1] - kd5[1], p[2][2] - kd5[2], p[2][3] - kd5[3]};
      v.iQ[4] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd6[0], p[2][1] - kd6[1], p[2][2] - kd6[2], p[2][3] - kd6[3]};
      v.iQ[5] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { S a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[4], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[2][j] = R(a[j]); v.e2[2][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
}

// Helicity profile: the averaged |M_h|^2 of every one of the NHEL helicity configurations
// (ih bit i: helicity of external particle i, set = +1), parity mirrors included, so that
// out[ih] sums to me2 and out[ih] = out[ih ^ (NHEL - 1)] tests the parity halving of me2
template <typename R>
__device__ void hel_profile_gg_ttg(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,
                                   typename Widen<R>::type gs, Me_gg_ttg::Inv<R>& v, double* out)
{
    using S = typename Widen<R>::type;
    inv_gg_ttg<R>(pflat, mt, v);
    S gk = S(1.0);
    for (int i = 0; i < Me_gg_ttg::NGLUON; ++i) gk = gk * (gs * gs);
    for (int ih = 0; ih < Me_gg_ttg::NHEL; ++ih)
        out[ih] = val(S(hel_gg_ttg<R>(v, ih)) / Me_gg_ttg::COLOUR_DEN * gk * Me_gg_ttg::AVG * Me_gg_ttg::SYM);
}
template <typename R>
__device__ void Me_gg_ttg::hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,
                                  typename Widen<R>::type gs, double* out)
{
    Me_gg_ttg::Inv<R> v;
    hel_profile_gg_ttg<R>(&p[0][0], mt, gs, v, out);
}
}  // namespace mf

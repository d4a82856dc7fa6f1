// Generated by paper_2105_10529_gb300/gen/qcd_diagrams.py -- do not edit.
// gg_ttgg: 123 Feynman diagrams (159 amplitudes with the four-gluon
// colour structures counted apart), 24 colour flows, 64 helicities.
// Wavefunction/vertex calls per helicity: {'vvv': 18, 'vvvv': 4, 'ffv_row': 26, 'ffv_col': 8, 'ffv_amp': 114, 'vvv_amp': 27, 'vvvv_amp': 6, 'ffv_cur': 1}
#pragma once
#include "mf_helas.cuh"
#include "mf_tc.cuh"
namespace mf {
// 54 C: the colour matrix times its common denominator, for the tensor-core colour sum
static __constant__ short colour54_gg_ttgg[576] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};
struct Me_gg_ttgg {
  static constexpr int NEXT = 6;
  static constexpr int NCOL = 24;
  static constexpr int NHEL = 64;
  static constexpr int NGLUON = 4;
  static constexpr int NDIAG = 123;
  static constexpr double COLOUR_DEN = 54.0;
  static constexpr double AVG = 1.0 / 256.0;
  static constexpr double SYM = 0.5;
  // colour sum on the tensor cores available (a dense 24 x 24 contraction)
  static constexpr bool TC_COLOUR = true;
  __device__ static const short* colour54() { return colour54_gg_ttgg; }
  // helicity-independent per-event pieces
  // per-thread slot: internal momenta, FP64-computed inverse denominators,
  // polarisation bases and spinor pieces of the event (kept in shared memory)
  template <typename R> struct Inv {
    R K[15][4]; R p3[4]; R iG[11]; R iQ[14];
    R e1[4][3]; R e2[4][3]; FermionBasis<R> fb3, fb4; R mt;
    cx<R> jamp[24];   // colour-flow amplitudes of the helicity being summed
    float pad[1];
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
  // warp-per-event schedule: the helicity-independent words of Inv (everything before jamp),
  // filled for one event by one thread (inv), then read by the 32 lanes of a warp, each
  // evaluating one of the 32 helicities of the parity-halved sum (hel_j, colour flows in
  // caller storage, no colour sum)
  static constexpr int INV_WORDS = 134;
  template <typename R>
  __device__ static void inv(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt, Inv<R>& v);
  // hel_j reads the warp's record at REC_OFF + (threadIdx.x / 32) REC_STRIDE bytes and keeps the
  // thread's colour flows at threadIdx.x JROW words, both from the start of dynamic shared memory
  template <typename R, int JROW, int REC_OFF, int REC_STRIDE>
  __device__ static void hel_j(int ih);
};

// one helicity configuration: amplitudes, colour flows and (CSUM) the colour sum;
// out of line so that its register allocation sees only one helicity
template <typename R, bool CSUM = true>
__device__ __noinline__ R hel_gg_ttgg(const Me_gg_ttgg::Inv<R>& v, int ih)
{
    constexpr int NCOL = Me_gg_ttgg::NCOL;
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
    W4<R> g3; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[3][j]); b[j] = ldv(v.e2[3][j]); }
      g3 = ext_gluon(a, b, HEL(5), true); }
    const W4<R> ub3 = ext_ubar(load_basis(v.fb3), HEL(2));
    const W4<R> v4 = ext_v(load_basis(v.fb4), HEL(3));
    const R k1_1[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k2_2[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w3 = vvv_cur(g0, g1, k1_1, k2_2, ldv(v.iG[0]));
    const R k1_4[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k4_5[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w6 = vvv_cur(g0, g2, k1_4, k4_5, ldv(v.iG[1]));
    const R k1_7[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k8_8[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w9 = vvv_cur(g0, g3, k1_7, k8_8, ldv(v.iG[4]));
    const R k2_10[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k4_11[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w12 = vvv_cur(g1, g2, k2_10, k4_11, ldv(v.iG[2]));
    const R k2_13[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k8_14[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w15 = vvv_cur(g1, g3, k2_13, k8_14, ldv(v.iG[5]));
    const R k4_16[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k8_17[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w18 = vvv_cur(g2, g3, k4_16, k8_17, ldv(v.iG[7]));
    const R q1_19[4] = {ldv(v.p3[0]) - ldv(v.K[0][0]), ldv(v.p3[1]) - ldv(v.K[0][1]), ldv(v.p3[2]) - ldv(v.K[0][2]), ldv(v.p3[3]) - ldv(v.K[0][3])};
    const W4<R> w20 = ffv_row(ub3, g0, q1_19, ldv(v.mt), ldv(v.iQ[0]));
    const R q3_21[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w22 = ffv_row(w20, g1, q3_21, ldv(v.mt), ldv(v.iQ[2]));
    const R q7_24[4] = {ldv(v.p3[0]) - ldv(v.K[6][0]), ldv(v.p3[1]) - ldv(v.K[6][1]), ldv(v.p3[2]) - ldv(v.K[6][2]), ldv(v.p3[3]) - ldv(v.K[6][3])};
    const W4<R> w23 = ffv_col(g3, v4, q7_24, ldv(v.mt), ldv(v.iQ[6]));
    const cx<R> a1 = ffv_amp(w22, w23, g2);
    jadd_mi(jamp[0], a1);
    const R q11_26[4] = {ldv(v.p3[0]) - ldv(v.K[10][0]), ldv(v.p3[1]) - ldv(v.K[10][1]), ldv(v.p3[2]) - ldv(v.K[10][2]), ldv(v.p3[3]) - ldv(v.K[10][3])};
    const W4<R> w25 = ffv_col(g2, v4, q11_26, ldv(v.mt), ldv(v.iQ[10]));
    const cx<R> a2 = ffv_amp(w22, w25, g3);
    jadd_mi(jamp[1], a2);
    const cx<R> a3 = ffv_amp(w22, v4, w18);
    jadd_mi(jamp[0], a3);
    jadd_pi(jamp[1], a3);
    const R q5_27[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w28 = ffv_row(w20, g2, q5_27, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a4 = ffv_amp(w28, w23, g1);
    jadd_mi(jamp[2], a4);
    const R q13_30[4] = {ldv(v.p3[0]) - ldv(v.K[12][0]), ldv(v.p3[1]) - ldv(v.K[12][1]), ldv(v.p3[2]) - ldv(v.K[12][2]), ldv(v.p3[3]) - ldv(v.K[12][3])};
    const W4<R> w29 = ffv_col(g1, v4, q13_30, ldv(v.mt), ldv(v.iQ[12]));
    const cx<R> a5 = ffv_amp(w28, w29, g3);
    jadd_mi(jamp[3], a5);
    const cx<R> a6 = ffv_amp(w28, v4, w15);
    jadd_mi(jamp[2], a6);
    jadd_pi(jamp[3], a6);
    const R q9_31[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w32 = ffv_row(w20, g3, q9_31, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a7 = ffv_amp(w32, w25, g1);
    jadd_mi(jamp[4], a7);
    const cx<R> a8 = ffv_amp(w32, w29, g2);
    jadd_mi(jamp[5], a8);
    const cx<R> a9 = ffv_amp(w32, v4, w12);
    jadd_mi(jamp[4], a9);
    jadd_pi(jamp[5], a9);
    const cx<R> a10 = ffv_amp(w20, w23, w12);
    jadd_mi(jamp[0], a10);
    jadd_pi(jamp[2], a10);
    const cx<R> a11 = ffv_amp(w20, w25, w15);
    jadd_mi(jamp[1], a11);
    jadd_pi(jamp[4], a11);
    const cx<R> a12 = ffv_amp(w20, w29, w18);
    jadd_mi(jamp[3], a12);
    jadd_pi(jamp[5], a12);
    const R q2_33[4] = {ldv(v.p3[0]) - ldv(v.K[1][0]), ldv(v.p3[1]) - ldv(v.K[1][1]), ldv(v.p3[2]) - ldv(v.K[1][2]), ldv(v.p3[3]) - ldv(v.K[1][3])};
    const W4<R> w34 = ffv_row(ub3, g1, q2_33, ldv(v.mt), ldv(v.iQ[1]));
    const R q3_35[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w36 = ffv_row(w34, g0, q3_35, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a13 = ffv_amp(w36, w23, g2);
    jadd_mi(jamp[6], a13);
    const cx<R> a14 = ffv_amp(w36, w25, g3);
    jadd_mi(jamp[7], a14);
    const cx<R> a15 = ffv_amp(w36, v4, w18);
    jadd_mi(jamp[6], a15);
    jadd_pi(jamp[7], a15);
    const R q6_37[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w38 = ffv_row(w34, g2, q6_37, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a16 = ffv_amp(w38, w23, g0);
    jadd_mi(jamp[8], a16);
    const R q14_40[4] = {ldv(v.p3[0]) - ldv(v.K[13][0]), ldv(v.p3[1]) - ldv(v.K[13][1]), ldv(v.p3[2]) - ldv(v.K[13][2]), ldv(v.p3[3]) - ldv(v.K[13][3])};
    const W4<R> w39 = ffv_col(g0, v4, q14_40, ldv(v.mt), ldv(v.iQ[13]));
    const cx<R> a17 = ffv_amp(w38, w39, g3);
    jadd_mi(jamp[9], a17);
    const cx<R> a18 = ffv_amp(w38, v4, w9);
    jadd_mi(jamp[8], a18);
    jadd_pi(jamp[9], a18);
    const R q10_41[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w42 = ffv_row(w34, g3, q10_41, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a19 = ffv_amp(w42, w25, g0);
    jadd_mi(jamp[10], a19);
    const cx<R> a20 = ffv_amp(w42, w39, g2);
    jadd_mi(jamp[11], a20);
    const cx<R> a21 = ffv_amp(w42, v4, w6);
    jadd_mi(jamp[10], a21);
    jadd_pi(jamp[11], a21);
    const cx<R> a22 = ffv_amp(w34, w23, w6);
    jadd_mi(jamp[6], a22);
    jadd_pi(jamp[8], a22);
    const cx<R> a23 = ffv_amp(w34, w25, w9);
    jadd_mi(jamp[7], a23);
    jadd_pi(jamp[10], a23);
    const cx<R> a24 = ffv_amp(w34, w39, w18);
    jadd_mi(jamp[9], a24);
    jadd_pi(jamp[11], a24);
    const R q4_43[4] = {ldv(v.p3[0]) - ldv(v.K[3][0]), ldv(v.p3[1]) - ldv(v.K[3][1]), ldv(v.p3[2]) - ldv(v.K[3][2]), ldv(v.p3[3]) - ldv(v.K[3][3])};
    const W4<R> w44 = ffv_row(ub3, g2, q4_43, ldv(v.mt), ldv(v.iQ[3]));
    const R q5_45[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w46 = ffv_row(w44, g0, q5_45, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a25 = ffv_amp(w46, w23, g1);
    jadd_mi(jamp[12], a25);
    const cx<R> a26 = ffv_amp(w46, w29, g3);
    jadd_mi(jamp[13], a26);
    const cx<R> a27 = ffv_amp(w46, v4, w15);
    jadd_mi(jamp[12], a27);
    jadd_pi(jamp[13], a27);
    const R q6_47[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w48 = ffv_row(w44, g1, q6_47, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a28 = ffv_amp(w48, w23, g0);
    jadd_mi(jamp[14], a28);
    const cx<R> a29 = ffv_amp(w48, w39, g3);
    jadd_mi(jamp[15], a29);
    const cx<R> a30 = ffv_amp(w48, v4, w9);
    jadd_mi(jamp[14], a30);
    jadd_pi(jamp[15], a30);
    const R q12_49[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w50 = ffv_row(w44, g3, q12_49, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a31 = ffv_amp(w50, w29, g0);
    jadd_mi(jamp[16], a31);
    const cx<R> a32 = ffv_amp(w50, w39, g1);
    jadd_mi(jamp[17], a32);
    const cx<R> a33 = ffv_amp(w50, v4, w3);
    jadd_mi(jamp[16], a33);
    jadd_pi(jamp[17], a33);
    const cx<R> a34 = ffv_amp(w44, w23, w3);
    jadd_mi(jamp[12], a34);
    jadd_pi(jamp[14], a34);
    const cx<R> a35 = ffv_amp(w44, w29, w9);
    jadd_mi(jamp[13], a35);
    jadd_pi(jamp[16], a35);
    const cx<R> a36 = ffv_amp(w44, w39, w15);
    jadd_mi(jamp[15], a36);
    jadd_pi(jamp[17], a36);
    const R q8_51[4] = {ldv(v.p3[0]) - ldv(v.K[7][0]), ldv(v.p3[1]) - ldv(v.K[7][1]), ldv(v.p3[2]) - ldv(v.K[7][2]), ldv(v.p3[3]) - ldv(v.K[7][3])};
    const W4<R> w52 = ffv_row(ub3, g3, q8_51, ldv(v.mt), ldv(v.iQ[7]));
    const R q9_53[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w54 = ffv_row(w52, g0, q9_53, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a37 = ffv_amp(w54, w25, g1);
    jadd_mi(jamp[18], a37);
    const cx<R> a38 = ffv_amp(w54, w29, g2);
    jadd_mi(jamp[19], a38);
    const cx<R> a39 = ffv_amp(w54, v4, w12);
    jadd_mi(jamp[18], a39);
    jadd_pi(jamp[19], a39);
    const R q10_55[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w56 = ffv_row(w52, g1, q10_55, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a40 = ffv_amp(w56, w25, g0);
    jadd_mi(jamp[20], a40);
    const cx<R> a41 = ffv_amp(w56, w39, g2);
    jadd_mi(jamp[21], a41);
    const cx<R> a42 = ffv_amp(w56, v4, w6);
    jadd_mi(jamp[20], a42);
    jadd_pi(jamp[21], a42);
    const R q12_57[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w58 = ffv_row(w52, g2, q12_57, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a43 = ffv_amp(w58, w29, g0);
    jadd_mi(jamp[22], a43);
    const cx<R> a44 = ffv_amp(w58, w39, g1);
    jadd_mi(jamp[23], a44);
    const cx<R> a45 = ffv_amp(w58, v4, w3);
    jadd_mi(jamp[22], a45);
    jadd_pi(jamp[23], a45);
    const cx<R> a46 = ffv_amp(w52, w25, w3);
    jadd_mi(jamp[18], a46);
    jadd_pi(jamp[20], a46);
    const cx<R> a47 = ffv_amp(w52, w29, w6);
    jadd_mi(jamp[19], a47);
    jadd_pi(jamp[22], a47);
    const cx<R> a48 = ffv_amp(w52, w39, w12);
    jadd_mi(jamp[21], a48);
    jadd_pi(jamp[23], a48);
    const R q3_59[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w60 = ffv_row(ub3, w3, q3_59, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a49 = ffv_amp(w60, w23, g2);
    jadd_mi(jamp[0], a49);
    jadd_pi(jamp[6], a49);
    const cx<R> a50 = ffv_amp(w60, w25, g3);
    jadd_mi(jamp[1], a50);
    jadd_pi(jamp[7], a50);
    const cx<R> a51 = ffv_amp(w60, v4, w18);
    jadd_mi(jamp[0], a51);
    jadd_pi(jamp[1], a51);
    jadd_pi(jamp[6], a51);
    jadd_mi(jamp[7], a51);
    const R q5_61[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w62 = ffv_row(ub3, w6, q5_61, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a52 = ffv_amp(w62, w23, g1);
    jadd_mi(jamp[2], a52);
    jadd_pi(jamp[12], a52);
    const cx<R> a53 = ffv_amp(w62, w29, g3);
    jadd_mi(jamp[3], a53);
    jadd_pi(jamp[13], a53);
    const cx<R> a54 = ffv_amp(w62, v4, w15);
    jadd_mi(jamp[2], a54);
    jadd_pi(jamp[3], a54);
    jadd_pi(jamp[12], a54);
    jadd_mi(jamp[13], a54);
    const R q9_63[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w64 = ffv_row(ub3, w9, q9_63, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a55 = ffv_amp(w64, w25, g1);
    jadd_mi(jamp[4], a55);
    jadd_pi(jamp[18], a55);
    const cx<R> a56 = ffv_amp(w64, w29, g2);
    jadd_mi(jamp[5], a56);
    jadd_pi(jamp[19], a56);
    const cx<R> a57 = ffv_amp(w64, v4, w12);
    jadd_mi(jamp[4], a57);
    jadd_pi(jamp[5], a57);
    jadd_pi(jamp[18], a57);
    jadd_mi(jamp[19], a57);
    const R q6_65[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w66 = ffv_row(ub3, w12, q6_65, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a58 = ffv_amp(w66, w23, g0);
    jadd_mi(jamp[8], a58);
    jadd_pi(jamp[14], a58);
    const cx<R> a59 = ffv_amp(w66, w39, g3);
    jadd_mi(jamp[9], a59);
    jadd_pi(jamp[15], a59);
    const cx<R> a60 = ffv_amp(w66, v4, w9);
    jadd_mi(jamp[8], a60);
    jadd_pi(jamp[9], a60);
    jadd_pi(jamp[14], a60);
    jadd_mi(jamp[15], a60);
    const R q10_67[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w68 = ffv_row(ub3, w15, q10_67, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a61 = ffv_amp(w68, w25, g0);
    jadd_mi(jamp[10], a61);
    jadd_pi(jamp[20], a61);
    const cx<R> a62 = ffv_amp(w68, w39, g2);
    jadd_mi(jamp[11], a62);
    jadd_pi(jamp[21], a62);
    const cx<R> a63 = ffv_amp(w68, v4, w6);
    jadd_mi(jamp[10], a63);
    jadd_pi(jamp[11], a63);
    jadd_pi(jamp[20], a63);
    jadd_mi(jamp[21], a63);
    const R q12_69[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w70 = ffv_row(ub3, w18, q12_69, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a64 = ffv_amp(w70, w29, g0);
    jadd_mi(jamp[16], a64);
    jadd_pi(jamp[22], a64);
    const cx<R> a65 = ffv_amp(w70, w39, g1);
    jadd_mi(jamp[17], a65);
    jadd_pi(jamp[23], a65);
    const cx<R> a66 = ffv_amp(w70, v4, w3);
    jadd_mi(jamp[16], a66);
    jadd_pi(jamp[17], a66);
    jadd_pi(jamp[22], a66);
    jadd_mi(jamp[23], a66);
    const W4<R> jq = ffv_cur(ub3, v4, ldv(v.iG[10]));
    {
    const R q7_72[4] = {ldv(v.p3[0]) - ldv(v.K[6][0]), ldv(v.p3[1]) - ldv(v.K[6][1]), ldv(v.p3[2]) - ldv(v.K[6][2]), ldv(v.p3[3]) - ldv(v.K[6][3])};
    const W4<R> w71 = ffv_col(g3, v4, q7_72, ldv(v.mt), ldv(v.iQ[6]));
    const R q8_73[4] = {ldv(v.p3[0]) - ldv(v.K[7][0]), ldv(v.p3[1]) - ldv(v.K[7][1]), ldv(v.p3[2]) - ldv(v.K[7][2]), ldv(v.p3[3]) - ldv(v.K[7][3])};
    const W4<R> w74 = ffv_row(ub3, g3, q8_73, ldv(v.mt), ldv(v.iQ[7]));
    {
    const R k1_75[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k6_76[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const W4<R> w77 = vvv_cur(g0, w12, k1_75, k6_76, ldv(v.iG[3]));
    const cx<R> a67 = ffv_amp(w74, v4, w77);
    jadd_mi(jamp[18], a67);
    jadd_pi(jamp[19], a67);
    jadd_pi(jamp[21], a67);
    jadd_mi(jamp[23], a67);
    const cx<R> a68 = ffv_amp(ub3, w71, w77);
    jadd_mi(jamp[0], a68);
    jadd_pi(jamp[2], a68);
    jadd_pi(jamp[8], a68);
    jadd_mi(jamp[14], a68);
    const R k7_78[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_79[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_80[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_80[4] = {-k15_80[0], -k15_80[1], -k15_80[2], -k15_80[3]};
    const cx<R> a69 = vvv_amp(w77, g3, jq, k7_78, k8_79, nkk15_80);
    jadd_mi(jamp[0], a69);
    jadd_pi(jamp[2], a69);
    jadd_pi(jamp[8], a69);
    jadd_mi(jamp[14], a69);
    jadd_pi(jamp[18], a69);
    jadd_mi(jamp[19], a69);
    jadd_mi(jamp[21], a69);
    jadd_pi(jamp[23], a69);
    }
    {
    const R k3_81[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k4_82[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w83 = vvv_cur(w3, g2, k3_81, k4_82, ldv(v.iG[3]));
    const cx<R> a70 = ffv_amp(w74, v4, w83);
    jadd_mi(jamp[18], a70);
    jadd_pi(jamp[20], a70);
    jadd_pi(jamp[22], a70);
    jadd_mi(jamp[23], a70);
    const cx<R> a71 = ffv_amp(ub3, w71, w83);
    jadd_mi(jamp[0], a71);
    jadd_pi(jamp[6], a71);
    jadd_pi(jamp[12], a71);
    jadd_mi(jamp[14], a71);
    const R k7_84[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_85[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_86[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_86[4] = {-k15_86[0], -k15_86[1], -k15_86[2], -k15_86[3]};
    const cx<R> a72 = vvv_amp(w83, g3, jq, k7_84, k8_85, nkk15_86);
    jadd_mi(jamp[0], a72);
    jadd_pi(jamp[6], a72);
    jadd_pi(jamp[12], a72);
    jadd_mi(jamp[14], a72);
    jadd_pi(jamp[18], a72);
    jadd_mi(jamp[20], a72);
    jadd_mi(jamp[22], a72);
    jadd_pi(jamp[23], a72);
    }
    {
    const R k5_87[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k2_88[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w89 = vvv_cur(w6, g1, k5_87, k2_88, ldv(v.iG[3]));
    const cx<R> a73 = ffv_amp(w74, v4, w89);
    jadd_mi(jamp[19], a73);
    jadd_pi(jamp[20], a73);
    jadd_mi(jamp[21], a73);
    jadd_pi(jamp[22], a73);
    const cx<R> a74 = ffv_amp(ub3, w71, w89);
    jadd_mi(jamp[2], a74);
    jadd_pi(jamp[6], a74);
    jadd_mi(jamp[8], a74);
    jadd_pi(jamp[12], a74);
    const R k7_90[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_91[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_92[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_92[4] = {-k15_92[0], -k15_92[1], -k15_92[2], -k15_92[3]};
    const cx<R> a75 = vvv_amp(w89, g3, jq, k7_90, k8_91, nkk15_92);
    jadd_mi(jamp[2], a75);
    jadd_pi(jamp[6], a75);
    jadd_mi(jamp[8], a75);
    jadd_pi(jamp[12], a75);
    jadd_pi(jamp[19], a75);
    jadd_mi(jamp[20], a75);
    jadd_pi(jamp[21], a75);
    jadd_mi(jamp[22], a75);
    }
    {
    W4<R> w93, w94, w95;
    vvvv_cur(g0, g1, g2, ldv(v.iG[3]), w93, w94, w95);
    const cx<R> a76 = ffv_amp(w74, v4, w93);
    jadd_mi(jamp[18], a76);
    jadd_pi(jamp[20], a76);
    jadd_pi(jamp[22], a76);
    jadd_mi(jamp[23], a76);
    const cx<R> a77 = ffv_amp(ub3, w71, w93);
    jadd_mi(jamp[0], a77);
    jadd_pi(jamp[6], a77);
    jadd_pi(jamp[12], a77);
    jadd_mi(jamp[14], a77);
    const R k7_96[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_97[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_98[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_98[4] = {-k15_98[0], -k15_98[1], -k15_98[2], -k15_98[3]};
    const cx<R> a78 = vvv_amp(w93, g3, jq, k7_96, k8_97, nkk15_98);
    jadd_mi(jamp[0], a78);
    jadd_pi(jamp[6], a78);
    jadd_pi(jamp[12], a78);
    jadd_mi(jamp[14], a78);
    jadd_pi(jamp[18], a78);
    jadd_mi(jamp[20], a78);
    jadd_mi(jamp[22], a78);
    jadd_pi(jamp[23], a78);
    const cx<R> a79 = ffv_amp(w74, v4, w94);
    jadd_mi(jamp[19], a79);
    jadd_pi(jamp[20], a79);
    jadd_mi(jamp[21], a79);
    jadd_pi(jamp[22], a79);
    const cx<R> a80 = ffv_amp(ub3, w71, w94);
    jadd_mi(jamp[2], a80);
    jadd_pi(jamp[6], a80);
    jadd_mi(jamp[8], a80);
    jadd_pi(jamp[12], a80);
    const R k7_99[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_100[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_101[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_101[4] = {-k15_101[0], -k15_101[1], -k15_101[2], -k15_101[3]};
    const cx<R> a81 = vvv_amp(w94, g3, jq, k7_99, k8_100, nkk15_101);
    jadd_mi(jamp[2], a81);
    jadd_pi(jamp[6], a81);
    jadd_mi(jamp[8], a81);
    jadd_pi(jamp[12], a81);
    jadd_pi(jamp[19], a81);
    jadd_mi(jamp[20], a81);
    jadd_pi(jamp[21], a81);
    jadd_mi(jamp[22], a81);
    const cx<R> a82 = ffv_amp(w74, v4, w95);
    jadd_pi(jamp[18], a82);
    jadd_mi(jamp[19], a82);
    jadd_mi(jamp[21], a82);
    jadd_pi(jamp[23], a82);
    const cx<R> a83 = ffv_amp(ub3, w71, w95);
    jadd_pi(jamp[0], a83);
    jadd_mi(jamp[2], a83);
    jadd_mi(jamp[8], a83);
    jadd_pi(jamp[14], a83);
    const R k7_102[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_103[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_104[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_104[4] = {-k15_104[0], -k15_104[1], -k15_104[2], -k15_104[3]};
    const cx<R> a84 = vvv_amp(w95, g3, jq, k7_102, k8_103, nkk15_104);
    jadd_pi(jamp[0], a84);
    jadd_mi(jamp[2], a84);
    jadd_mi(jamp[8], a84);
    jadd_pi(jamp[14], a84);
    jadd_mi(jamp[18], a84);
    jadd_pi(jamp[19], a84);
    jadd_pi(jamp[21], a84);
    jadd_mi(jamp[23], a84);
    }
    }
    {
    const R q11_106[4] = {ldv(v.p3[0]) - ldv(v.K[10][0]), ldv(v.p3[1]) - ldv(v.K[10][1]), ldv(v.p3[2]) - ldv(v.K[10][2]), ldv(v.p3[3]) - ldv(v.K[10][3])};
    const W4<R> w105 = ffv_col(g2, v4, q11_106, ldv(v.mt), ldv(v.iQ[10]));
    const R q4_107[4] = {ldv(v.p3[0]) - ldv(v.K[3][0]), ldv(v.p3[1]) - ldv(v.K[3][1]), ldv(v.p3[2]) - ldv(v.K[3][2]), ldv(v.p3[3]) - ldv(v.K[3][3])};
    const W4<R> w108 = ffv_row(ub3, g2, q4_107, ldv(v.mt), ldv(v.iQ[3]));
    {
    const R k1_109[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k10_110[4] = {ldv(v.K[9][0]), ldv(v.K[9][1]), ldv(v.K[9][2]), ldv(v.K[9][3])};
    const W4<R> w111 = vvv_cur(g0, w15, k1_109, k10_110, ldv(v.iG[6]));
    const cx<R> a85 = ffv_amp(w108, v4, w111);
    jadd_mi(jamp[12], a85);
    jadd_pi(jamp[13], a85);
    jadd_pi(jamp[15], a85);
    jadd_mi(jamp[17], a85);
    const cx<R> a86 = ffv_amp(ub3, w105, w111);
    jadd_mi(jamp[1], a86);
    jadd_pi(jamp[4], a86);
    jadd_pi(jamp[10], a86);
    jadd_mi(jamp[20], a86);
    const R k11_112[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_113[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_114[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_114[4] = {-k15_114[0], -k15_114[1], -k15_114[2], -k15_114[3]};
    const cx<R> a87 = vvv_amp(w111, g2, jq, k11_112, k4_113, nkk15_114);
    jadd_mi(jamp[1], a87);
    jadd_pi(jamp[4], a87);
    jadd_pi(jamp[10], a87);
    jadd_pi(jamp[12], a87);
    jadd_mi(jamp[13], a87);
    jadd_mi(jamp[15], a87);
    jadd_pi(jamp[17], a87);
    jadd_mi(jamp[20], a87);
    }
    {
    const R k3_115[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k8_116[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w117 = vvv_cur(w3, g3, k3_115, k8_116, ldv(v.iG[6]));
    const cx<R> a88 = ffv_amp(w108, v4, w117);
    jadd_mi(jamp[12], a88);
    jadd_pi(jamp[14], a88);
    jadd_pi(jamp[16], a88);
    jadd_mi(jamp[17], a88);
    const cx<R> a89 = ffv_amp(ub3, w105, w117);
    jadd_mi(jamp[1], a89);
    jadd_pi(jamp[7], a89);
    jadd_pi(jamp[18], a89);
    jadd_mi(jamp[20], a89);
    const R k11_118[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_119[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_120[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_120[4] = {-k15_120[0], -k15_120[1], -k15_120[2], -k15_120[3]};
    const cx<R> a90 = vvv_amp(w117, g2, jq, k11_118, k4_119, nkk15_120);
    jadd_mi(jamp[1], a90);
    jadd_pi(jamp[7], a90);
    jadd_pi(jamp[12], a90);
    jadd_mi(jamp[14], a90);
    jadd_mi(jamp[16], a90);
    jadd_pi(jamp[17], a90);
    jadd_pi(jamp[18], a90);
    jadd_mi(jamp[20], a90);
    }
    {
    const R k9_121[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k2_122[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w123 = vvv_cur(w9, g1, k9_121, k2_122, ldv(v.iG[6]));
    const cx<R> a91 = ffv_amp(w108, v4, w123);
    jadd_mi(jamp[13], a91);
    jadd_pi(jamp[14], a91);
    jadd_mi(jamp[15], a91);
    jadd_pi(jamp[16], a91);
    const cx<R> a92 = ffv_amp(ub3, w105, w123);
    jadd_mi(jamp[4], a92);
    jadd_pi(jamp[7], a92);
    jadd_mi(jamp[10], a92);
    jadd_pi(jamp[18], a92);
    const R k11_124[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_125[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_126[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_126[4] = {-k15_126[0], -k15_126[1], -k15_126[2], -k15_126[3]};
    const cx<R> a93 = vvv_amp(w123, g2, jq, k11_124, k4_125, nkk15_126);
    jadd_mi(jamp[4], a93);
    jadd_pi(jamp[7], a93);
    jadd_mi(jamp[10], a93);
    jadd_pi(jamp[13], a93);
    jadd_mi(jamp[14], a93);
    jadd_pi(jamp[15], a93);
    jadd_mi(jamp[16], a93);
    jadd_pi(jamp[18], a93);
    }
    {
    W4<R> w127, w128, w129;
    vvvv_cur(g0, g1, g3, ldv(v.iG[6]), w127, w128, w129);
    const cx<R> a94 = ffv_amp(w108, v4, w127);
    jadd_mi(jamp[12], a94);
    jadd_pi(jamp[14], a94);
    jadd_pi(jamp[16], a94);
    jadd_mi(jamp[17], a94);
    const cx<R> a95 = ffv_amp(ub3, w105, w127);
    jadd_mi(jamp[1], a95);
    jadd_pi(jamp[7], a95);
    jadd_pi(jamp[18], a95);
    jadd_mi(jamp[20], a95);
    const R k11_130[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_131[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_132[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_132[4] = {-k15_132[0], -k15_132[1], -k15_132[2], -k15_132[3]};
    const cx<R> a96 = vvv_amp(w127, g2, jq, k11_130, k4_131, nkk15_132);
    jadd_mi(jamp[1], a96);
    jadd_pi(jamp[7], a96);
    jadd_pi(jamp[12], a96);
    jadd_mi(jamp[14], a96);
    jadd_mi(jamp[16], a96);
    jadd_pi(jamp[17], a96);
    jadd_pi(jamp[18], a96);
    jadd_mi(jamp[20], a96);
    const cx<R> a97 = ffv_amp(w108, v4, w128);
    jadd_mi(jamp[13], a97);
    jadd_pi(jamp[14], a97);
    jadd_mi(jamp[15], a97);
    jadd_pi(jamp[16], a97);
    const cx<R> a98 = ffv_amp(ub3, w105, w128);
    jadd_mi(jamp[4], a98);
    jadd_pi(jamp[7], a98);
    jadd_mi(jamp[10], a98);
    jadd_pi(jamp[18], a98);
    const R k11_133[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_134[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_135[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_135[4] = {-k15_135[0], -k15_135[1], -k15_135[2], -k15_135[3]};
    const cx<R> a99 = vvv_amp(w128, g2, jq, k11_133, k4_134, nkk15_135);
    jadd_mi(jamp[4], a99);
    jadd_pi(jamp[7], a99);
    jadd_mi(jamp[10], a99);
    jadd_pi(jamp[13], a99);
    jadd_mi(jamp[14], a99);
    jadd_pi(jamp[15], a99);
    jadd_mi(jamp[16], a99);
    jadd_pi(jamp[18], a99);
    const cx<R> a100 = ffv_amp(w108, v4, w129);
    jadd_pi(jamp[12], a100);
    jadd_mi(jamp[13], a100);
    jadd_mi(jamp[15], a100);
    jadd_pi(jamp[17], a100);
    const cx<R> a101 = ffv_amp(ub3, w105, w129);
    jadd_pi(jamp[1], a101);
    jadd_mi(jamp[4], a101);
    jadd_mi(jamp[10], a101);
    jadd_pi(jamp[20], a101);
    const R k11_136[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_137[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_138[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_138[4] = {-k15_138[0], -k15_138[1], -k15_138[2], -k15_138[3]};
    const cx<R> a102 = vvv_amp(w129, g2, jq, k11_136, k4_137, nkk15_138);
    jadd_pi(jamp[1], a102);
    jadd_mi(jamp[4], a102);
    jadd_mi(jamp[10], a102);
    jadd_mi(jamp[12], a102);
    jadd_pi(jamp[13], a102);
    jadd_pi(jamp[15], a102);
    jadd_mi(jamp[17], a102);
    jadd_pi(jamp[20], a102);
    }
    }
    {
    const R q13_140[4] = {ldv(v.p3[0]) - ldv(v.K[12][0]), ldv(v.p3[1]) - ldv(v.K[12][1]), ldv(v.p3[2]) - ldv(v.K[12][2]), ldv(v.p3[3]) - ldv(v.K[12][3])};
    const W4<R> w139 = ffv_col(g1, v4, q13_140, ldv(v.mt), ldv(v.iQ[12]));
    const R q2_141[4] = {ldv(v.p3[0]) - ldv(v.K[1][0]), ldv(v.p3[1]) - ldv(v.K[1][1]), ldv(v.p3[2]) - ldv(v.K[1][2]), ldv(v.p3[3]) - ldv(v.K[1][3])};
    const W4<R> w142 = ffv_row(ub3, g1, q2_141, ldv(v.mt), ldv(v.iQ[1]));
    {
    const R k1_143[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k12_144[4] = {ldv(v.K[11][0]), ldv(v.K[11][1]), ldv(v.K[11][2]), ldv(v.K[11][3])};
    const W4<R> w145 = vvv_cur(g0, w18, k1_143, k12_144, ldv(v.iG[8]));
    const cx<R> a103 = ffv_amp(w142, v4, w145);
    jadd_mi(jamp[6], a103);
    jadd_pi(jamp[7], a103);
    jadd_pi(jamp[9], a103);
    jadd_mi(jamp[11], a103);
    const cx<R> a104 = ffv_amp(ub3, w139, w145);
    jadd_mi(jamp[3], a104);
    jadd_pi(jamp[5], a104);
    jadd_pi(jamp[16], a104);
    jadd_mi(jamp[22], a104);
    const R k13_146[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_147[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_148[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_148[4] = {-k15_148[0], -k15_148[1], -k15_148[2], -k15_148[3]};
    const cx<R> a105 = vvv_amp(w145, g1, jq, k13_146, k2_147, nkk15_148);
    jadd_mi(jamp[3], a105);
    jadd_pi(jamp[5], a105);
    jadd_pi(jamp[6], a105);
    jadd_mi(jamp[7], a105);
    jadd_mi(jamp[9], a105);
    jadd_pi(jamp[11], a105);
    jadd_pi(jamp[16], a105);
    jadd_mi(jamp[22], a105);
    }
    {
    const R k5_149[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k8_150[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w151 = vvv_cur(w6, g3, k5_149, k8_150, ldv(v.iG[8]));
    const cx<R> a106 = ffv_amp(w142, v4, w151);
    jadd_mi(jamp[6], a106);
    jadd_pi(jamp[8], a106);
    jadd_pi(jamp[10], a106);
    jadd_mi(jamp[11], a106);
    const cx<R> a107 = ffv_amp(ub3, w139, w151);
    jadd_mi(jamp[3], a107);
    jadd_pi(jamp[13], a107);
    jadd_pi(jamp[19], a107);
    jadd_mi(jamp[22], a107);
    const R k13_152[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_153[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_154[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_154[4] = {-k15_154[0], -k15_154[1], -k15_154[2], -k15_154[3]};
    const cx<R> a108 = vvv_amp(w151, g1, jq, k13_152, k2_153, nkk15_154);
    jadd_mi(jamp[3], a108);
    jadd_pi(jamp[6], a108);
    jadd_mi(jamp[8], a108);
    jadd_mi(jamp[10], a108);
    jadd_pi(jamp[11], a108);
    jadd_pi(jamp[13], a108);
    jadd_pi(jamp[19], a108);
    jadd_mi(jamp[22], a108);
    }
    {
    const R k9_155[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k4_156[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w157 = vvv_cur(w9, g2, k9_155, k4_156, ldv(v.iG[8]));
    const cx<R> a109 = ffv_amp(w142, v4, w157);
    jadd_mi(jamp[7], a109);
    jadd_pi(jamp[8], a109);
    jadd_mi(jamp[9], a109);
    jadd_pi(jamp[10], a109);
    const cx<R> a110 = ffv_amp(ub3, w139, w157);
    jadd_mi(jamp[5], a110);
    jadd_pi(jamp[13], a110);
    jadd_mi(jamp[16], a110);
    jadd_pi(jamp[19], a110);
    const R k13_158[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_159[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_160[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_160[4] = {-k15_160[0], -k15_160[1], -k15_160[2], -k15_160[3]};
    const cx<R> a111 = vvv_amp(w157, g1, jq, k13_158, k2_159, nkk15_160);
    jadd_mi(jamp[5], a111);
    jadd_pi(jamp[7], a111);
    jadd_mi(jamp[8], a111);
    jadd_pi(jamp[9], a111);
    jadd_mi(jamp[10], a111);
    jadd_pi(jamp[13], a111);
    jadd_mi(jamp[16], a111);
    jadd_pi(jamp[19], a111);
    }
    {
    W4<R> w161, w162, w163;
    vvvv_cur(g0, g2, g3, ldv(v.iG[8]), w161, w162, w163);
    const cx<R> a112 = ffv_amp(w142, v4, w161);
    jadd_mi(jamp[6], a112);
    jadd_pi(jamp[8], a112);
    jadd_pi(jamp[10], a112);
    jadd_mi(jamp[11], a112);
    const cx<R> a113 = ffv_amp(ub3, w139, w161);
    jadd_mi(jamp[3], a113);
    jadd_pi(jamp[13], a113);
    jadd_pi(jamp[19], a113);
    jadd_mi(jamp[22], a113);
    const R k13_164[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_165[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_166[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_166[4] = {-k15_166[0], -k15_166[1], -k15_166[2], -k15_166[3]};
    const cx<R> a114 = vvv_amp(w161, g1, jq, k13_164, k2_165, nkk15_166);
    jadd_mi(jamp[3], a114);
    jadd_pi(jamp[6], a114);
    jadd_mi(jamp[8], a114);
    jadd_mi(jamp[10], a114);
    jadd_pi(jamp[11], a114);
    jadd_pi(jamp[13], a114);
    jadd_pi(jamp[19], a114);
    jadd_mi(jamp[22], a114);
    const cx<R> a115 = ffv_amp(w142, v4, w162);
    jadd_mi(jamp[7], a115);
    jadd_pi(jamp[8], a115);
    jadd_mi(jamp[9], a115);
    jadd_pi(jamp[10], a115);
    const cx<R> a116 = ffv_amp(ub3, w139, w162);
    jadd_mi(jamp[5], a116);
    jadd_pi(jamp[13], a116);
    jadd_mi(jamp[16], a116);
    jadd_pi(jamp[19], a116);
    const R k13_167[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_168[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_169[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_169[4] = {-k15_169[0], -k15_169[1], -k15_169[2], -k15_169[3]};
    const cx<R> a117 = vvv_amp(w162, g1, jq, k13_167, k2_168, nkk15_169);
    jadd_mi(jamp[5], a117);
    jadd_pi(jamp[7], a117);
    jadd_mi(jamp[8], a117);
    jadd_pi(jamp[9], a117);
    jadd_mi(jamp[10], a117);
    jadd_pi(jamp[13], a117);
    jadd_mi(jamp[16], a117);
    jadd_pi(jamp[19], a117);
    const cx<R> a118 = ffv_amp(w142, v4, w163);
    jadd_pi(jamp[6], a118);
    jadd_mi(jamp[7], a118);
    jadd_mi(jamp[9], a118);
    jadd_pi(jamp[11], a118);
    const cx<R> a119 = ffv_amp(ub3, w139, w163);
    jadd_pi(jamp[3], a119);
    jadd_mi(jamp[5], a119);
    jadd_mi(jamp[16], a119);
    jadd_pi(jamp[22], a119);
    const R k13_170[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_171[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_172[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_172[4] = {-k15_172[0], -k15_172[1], -k15_172[2], -k15_172[3]};
    const cx<R> a120 = vvv_amp(w163, g1, jq, k13_170, k2_171, nkk15_172);
    jadd_pi(jamp[3], a120);
    jadd_mi(jamp[5], a120);
    jadd_mi(jamp[6], a120);
    jadd_pi(jamp[7], a120);
    jadd_pi(jamp[9], a120);
    jadd_mi(jamp[11], a120);
    jadd_mi(jamp[16], a120);
    jadd_pi(jamp[22], a120);
    }
    }
    {
    const R q14_174[4] = {ldv(v.p3[0]) - ldv(v.K[13][0]), ldv(v.p3[1]) - ldv(v.K[13][1]), ldv(v.p3[2]) - ldv(v.K[13][2]), ldv(v.p3[3]) - ldv(v.K[13][3])};
    const W4<R> w173 = ffv_col(g0, v4, q14_174, ldv(v.mt), ldv(v.iQ[13]));
    const R q1_175[4] = {ldv(v.p3[0]) - ldv(v.K[0][0]), ldv(v.p3[1]) - ldv(v.K[0][1]), ldv(v.p3[2]) - ldv(v.K[0][2]), ldv(v.p3[3]) - ldv(v.K[0][3])};
    const W4<R> w176 = ffv_row(ub3, g0, q1_175, ldv(v.mt), ldv(v.iQ[0]));
    {
    const R k2_177[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k12_178[4] = {ldv(v.K[11][0]), ldv(v.K[11][1]), ldv(v.K[11][2]), ldv(v.K[11][3])};
    const W4<R> w179 = vvv_cur(g1, w18, k2_177, k12_178, ldv(v.iG[9]));
    const cx<R> a121 = ffv_amp(w176, v4, w179);
    jadd_mi(jamp[0], a121);
    jadd_pi(jamp[1], a121);
    jadd_pi(jamp[3], a121);
    jadd_mi(jamp[5], a121);
    const cx<R> a122 = ffv_amp(ub3, w173, w179);
    jadd_mi(jamp[9], a122);
    jadd_pi(jamp[11], a122);
    jadd_pi(jamp[17], a122);
    jadd_mi(jamp[23], a122);
    const R k1_180[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_181[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_182[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_182[4] = {-k15_182[0], -k15_182[1], -k15_182[2], -k15_182[3]};
    const cx<R> a123 = vvv_amp(g0, w179, jq, k1_180, k14_181, nkk15_182);
    jadd_mi(jamp[0], a123);
    jadd_pi(jamp[1], a123);
    jadd_pi(jamp[3], a123);
    jadd_mi(jamp[5], a123);
    jadd_pi(jamp[9], a123);
    jadd_mi(jamp[11], a123);
    jadd_mi(jamp[17], a123);
    jadd_pi(jamp[23], a123);
    }
    {
    const R k6_183[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const R k8_184[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w185 = vvv_cur(w12, g3, k6_183, k8_184, ldv(v.iG[9]));
    const cx<R> a124 = ffv_amp(w176, v4, w185);
    jadd_mi(jamp[0], a124);
    jadd_pi(jamp[2], a124);
    jadd_pi(jamp[4], a124);
    jadd_mi(jamp[5], a124);
    const cx<R> a125 = ffv_amp(ub3, w173, w185);
    jadd_mi(jamp[9], a125);
    jadd_pi(jamp[15], a125);
    jadd_pi(jamp[21], a125);
    jadd_mi(jamp[23], a125);
    const R k1_186[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_187[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_188[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_188[4] = {-k15_188[0], -k15_188[1], -k15_188[2], -k15_188[3]};
    const cx<R> a126 = vvv_amp(g0, w185, jq, k1_186, k14_187, nkk15_188);
    jadd_mi(jamp[0], a126);
    jadd_pi(jamp[2], a126);
    jadd_pi(jamp[4], a126);
    jadd_mi(jamp[5], a126);
    jadd_pi(jamp[9], a126);
    jadd_mi(jamp[15], a126);
    jadd_mi(jamp[21], a126);
    jadd_pi(jamp[23], a126);
    }
    {
    const R k10_189[4] = {ldv(v.K[9][0]), ldv(v.K[9][1]), ldv(v.K[9][2]), ldv(v.K[9][3])};
    const R k4_190[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w191 = vvv_cur(w15, g2, k10_189, k4_190, ldv(v.iG[9]));
    const cx<R> a127 = ffv_amp(w176, v4, w191);
    jadd_mi(jamp[1], a127);
    jadd_pi(jamp[2], a127);
    jadd_mi(jamp[3], a127);
    jadd_pi(jamp[4], a127);
    const cx<R> a128 = ffv_amp(ub3, w173, w191);
    jadd_mi(jamp[11], a128);
    jadd_pi(jamp[15], a128);
    jadd_mi(jamp[17], a128);
    jadd_pi(jamp[21], a128);
    const R k1_192[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_193[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_194[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_194[4] = {-k15_194[0], -k15_194[1], -k15_194[2], -k15_194[3]};
    const cx<R> a129 = vvv_amp(g0, w191, jq, k1_192, k14_193, nkk15_194);
    jadd_mi(jamp[1], a129);
    jadd_pi(jamp[2], a129);
    jadd_mi(jamp[3], a129);
    jadd_pi(jamp[4], a129);
    jadd_pi(jamp[11], a129);
    jadd_mi(jamp[15], a129);
    jadd_pi(jamp[17], a129);
    jadd_mi(jamp[21], a129);
    }
    {
    W4<R> w195, w196, w197;
    vvvv_cur(g1, g2, g3, ldv(v.iG[9]), w195, w196, w197);
    const cx<R> a130 = ffv_amp(w176, v4, w195);
    jadd_mi(jamp[0], a130);
    jadd_pi(jamp[2], a130);
    jadd_pi(jamp[4], a130);
    jadd_mi(jamp[5], a130);
    const cx<R> a131 = ffv_amp(ub3, w173, w195);
    jadd_mi(jamp[9], a131);
    jadd_pi(jamp[15], a131);
    jadd_pi(jamp[21], a131);
    jadd_mi(jamp[23], a131);
    const R k1_198[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_199[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_200[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_200[4] = {-k15_200[0], -k15_200[1], -k15_200[2], -k15_200[3]};
    const cx<R> a132 = vvv_amp(g0, w195, jq, k1_198, k14_199, nkk15_200);
    jadd_mi(jamp[0], a132);
    jadd_pi(jamp[2], a132);
    jadd_pi(jamp[4], a132);
    jadd_mi(jamp[5], a132);
    jadd_pi(jamp[9], a132);
    jadd_mi(jamp[15], a132);
    jadd_mi(jamp[21], a132);
    jadd_pi(jamp[23], a132);
    const cx<R> a133 = ffv_amp(w176, v4, w196);
    jadd_mi(jamp[1], a133);
    jadd_pi(jamp[2], a133);
    jadd_mi(jamp[3], a133);
    jadd_pi(jamp[4], a133);
    const cx<R> a134 = ffv_amp(ub3, w173, w196);
    jadd_mi(jamp[11], a134);
    jadd_pi(jamp[15], a134);
    jadd_mi(jamp[17], a134);
    jadd_pi(jamp[21], a134);
    const R k1_201[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_202[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_203[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_203[4] = {-k15_203[0], -k15_203[1], -k15_203[2], -k15_203[3]};
    const cx<R> a135 = vvv_amp(g0, w196, jq, k1_201, k14_202, nkk15_203);
    jadd_mi(jamp[1], a135);
    jadd_pi(jamp[2], a135);
    jadd_mi(jamp[3], a135);
    jadd_pi(jamp[4], a135);
    jadd_pi(jamp[11], a135);
    jadd_mi(jamp[15], a135);
    jadd_pi(jamp[17], a135);
    jadd_mi(jamp[21], a135);
    const cx<R> a136 = ffv_amp(w176, v4, w197);
    jadd_pi(jamp[0], a136);
    jadd_mi(jamp[1], a136);
    jadd_mi(jamp[3], a136);
    jadd_pi(jamp[5], a136);
    const cx<R> a137 = ffv_amp(ub3, w173, w197);
    jadd_pi(jamp[9], a137);
    jadd_mi(jamp[11], a137);
    jadd_mi(jamp[17], a137);
    jadd_pi(jamp[23], a137);
    const R k1_204[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_205[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_206[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_206[4] = {-k15_206[0], -k15_206[1], -k15_206[2], -k15_206[3]};
    const cx<R> a138 = vvv_amp(g0, w197, jq, k1_204, k14_205, nkk15_206);
    jadd_pi(jamp[0], a138);
    jadd_mi(jamp[1], a138);
    jadd_mi(jamp[3], a138);
    jadd_pi(jamp[5], a138);
    jadd_mi(jamp[9], a138);
    jadd_pi(jamp[11], a138);
    jadd_pi(jamp[17], a138);
    jadd_mi(jamp[23], a138);
    }
    }
    const R k3_207[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k12_208[4] = {ldv(v.K[11][0]), ldv(v.K[11][1]), ldv(v.K[11][2]), ldv(v.K[11][3])};
    const R k15_209[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_209[4] = {-k15_209[0], -k15_209[1], -k15_209[2], -k15_209[3]};
    const cx<R> a139 = vvv_amp(w3, w18, jq, k3_207, k12_208, nkk15_209);
    jadd_mi(jamp[0], a139);
    jadd_pi(jamp[1], a139);
    jadd_pi(jamp[6], a139);
    jadd_mi(jamp[7], a139);
    jadd_pi(jamp[16], a139);
    jadd_mi(jamp[17], a139);
    jadd_mi(jamp[22], a139);
    jadd_pi(jamp[23], a139);
    const R k5_210[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k10_211[4] = {ldv(v.K[9][0]), ldv(v.K[9][1]), ldv(v.K[9][2]), ldv(v.K[9][3])};
    const R k15_212[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_212[4] = {-k15_212[0], -k15_212[1], -k15_212[2], -k15_212[3]};
    const cx<R> a140 = vvv_amp(w6, w15, jq, k5_210, k10_211, nkk15_212);
    jadd_mi(jamp[2], a140);
    jadd_pi(jamp[3], a140);
    jadd_pi(jamp[10], a140);
    jadd_mi(jamp[11], a140);
    jadd_pi(jamp[12], a140);
    jadd_mi(jamp[13], a140);
    jadd_mi(jamp[20], a140);
    jadd_pi(jamp[21], a140);
    const R k9_213[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k6_214[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const R k15_215[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_215[4] = {-k15_215[0], -k15_215[1], -k15_215[2], -k15_215[3]};
    const cx<R> a141 = vvv_amp(w9, w12, jq, k9_213, k6_214, nkk15_215);
    jadd_mi(jamp[4], a141);
    jadd_pi(jamp[5], a141);
    jadd_pi(jamp[8], a141);
    jadd_mi(jamp[9], a141);
    jadd_mi(jamp[14], a141);
    jadd_pi(jamp[15], a141);
    jadd_pi(jamp[18], a141);
    jadd_mi(jamp[19], a141);
    cx<R> a142, a143, a144;
    vvvv_amp(g0, g1, w18, jq, a142, a143, a144);
    jadd_mi(jamp[0], a142);
    jadd_pi(jamp[1], a142);
    jadd_pi(jamp[6], a142);
    jadd_mi(jamp[7], a142);
    jadd_pi(jamp[16], a142);
    jadd_mi(jamp[17], a142);
    jadd_mi(jamp[22], a142);
    jadd_pi(jamp[23], a142);
    jadd_mi(jamp[3], a143);
    jadd_pi(jamp[5], a143);
    jadd_pi(jamp[6], a143);
    jadd_mi(jamp[7], a143);
    jadd_mi(jamp[9], a143);
    jadd_pi(jamp[11], a143);
    jadd_pi(jamp[16], a143);
    jadd_mi(jamp[22], a143);
    jadd_pi(jamp[0], a144);
    jadd_mi(jamp[1], a144);
    jadd_mi(jamp[3], a144);
    jadd_pi(jamp[5], a144);
    jadd_mi(jamp[9], a144);
    jadd_pi(jamp[11], a144);
    jadd_pi(jamp[17], a144);
    jadd_mi(jamp[23], a144);
    cx<R> a145, a146, a147;
    vvvv_amp(g0, w12, g3, jq, a145, a146, a147);
    jadd_mi(jamp[0], a145);
    jadd_pi(jamp[2], a145);
    jadd_pi(jamp[8], a145);
    jadd_mi(jamp[14], a145);
    jadd_pi(jamp[18], a145);
    jadd_mi(jamp[19], a145);
    jadd_mi(jamp[21], a145);
    jadd_pi(jamp[23], a145);
    jadd_mi(jamp[4], a146);
    jadd_pi(jamp[5], a146);
    jadd_pi(jamp[8], a146);
    jadd_mi(jamp[9], a146);
    jadd_mi(jamp[14], a146);
    jadd_pi(jamp[15], a146);
    jadd_pi(jamp[18], a146);
    jadd_mi(jamp[19], a146);
    jadd_pi(jamp[0], a147);
    jadd_mi(jamp[2], a147);
    jadd_mi(jamp[4], a147);
    jadd_pi(jamp[5], a147);
    jadd_mi(jamp[9], a147);
    jadd_pi(jamp[15], a147);
    jadd_pi(jamp[21], a147);
    jadd_mi(jamp[23], a147);
    cx<R> a148, a149, a150;
    vvvv_amp(g0, w15, g2, jq, a148, a149, a150);
    jadd_mi(jamp[1], a148);
    jadd_pi(jamp[4], a148);
    jadd_pi(jamp[10], a148);
    jadd_pi(jamp[12], a148);
    jadd_mi(jamp[13], a148);
    jadd_mi(jamp[15], a148);
    jadd_pi(jamp[17], a148);
    jadd_mi(jamp[20], a148);
    jadd_mi(jamp[2], a149);
    jadd_pi(jamp[3], a149);
    jadd_pi(jamp[10], a149);
    jadd_mi(jamp[11], a149);
    jadd_pi(jamp[12], a149);
    jadd_mi(jamp[13], a149);
    jadd_mi(jamp[20], a149);
    jadd_pi(jamp[21], a149);
    jadd_pi(jamp[1], a150);
    jadd_mi(jamp[2], a150);
    jadd_pi(jamp[3], a150);
    jadd_mi(jamp[4], a150);
    jadd_mi(jamp[11], a150);
    jadd_pi(jamp[15], a150);
    jadd_mi(jamp[17], a150);
    jadd_pi(jamp[21], a150);
    cx<R> a151, a152, a153;
    vvvv_amp(w3, g2, g3, jq, a151, a152, a153);
    jadd_mi(jamp[0], a151);
    jadd_pi(jamp[6], a151);
    jadd_pi(jamp[12], a151);
    jadd_mi(jamp[14], a151);
    jadd_pi(jamp[18], a151);
    jadd_mi(jamp[20], a151);
    jadd_mi(jamp[22], a151);
    jadd_pi(jamp[23], a151);
    jadd_mi(jamp[1], a152);
    jadd_pi(jamp[7], a152);
    jadd_pi(jamp[12], a152);
    jadd_mi(jamp[14], a152);
    jadd_mi(jamp[16], a152);
    jadd_pi(jamp[17], a152);
    jadd_pi(jamp[18], a152);
    jadd_mi(jamp[20], a152);
    jadd_pi(jamp[0], a153);
    jadd_mi(jamp[1], a153);
    jadd_mi(jamp[6], a153);
    jadd_pi(jamp[7], a153);
    jadd_mi(jamp[16], a153);
    jadd_pi(jamp[17], a153);
    jadd_pi(jamp[22], a153);
    jadd_mi(jamp[23], a153);
    cx<R> a154, a155, a156;
    vvvv_amp(w6, g1, g3, jq, a154, a155, a156);
    jadd_mi(jamp[2], a154);
    jadd_pi(jamp[6], a154);
    jadd_mi(jamp[8], a154);
    jadd_pi(jamp[12], a154);
    jadd_pi(jamp[19], a154);
    jadd_mi(jamp[20], a154);
    jadd_pi(jamp[21], a154);
    jadd_mi(jamp[22], a154);
    jadd_mi(jamp[3], a155);
    jadd_pi(jamp[6], a155);
    jadd_mi(jamp[8], a155);
    jadd_mi(jamp[10], a155);
    jadd_pi(jamp[11], a155);
    jadd_pi(jamp[13], a155);
    jadd_pi(jamp[19], a155);
    jadd_mi(jamp[22], a155);
    jadd_pi(jamp[2], a156);
    jadd_mi(jamp[3], a156);
    jadd_mi(jamp[10], a156);
    jadd_pi(jamp[11], a156);
    jadd_mi(jamp[12], a156);
    jadd_pi(jamp[13], a156);
    jadd_pi(jamp[20], a156);
    jadd_mi(jamp[21], a156);
    cx<R> a157, a158, a159;
    vvvv_amp(w9, g1, g2, jq, a157, a158, a159);
    jadd_mi(jamp[4], a157);
    jadd_pi(jamp[7], a157);
    jadd_mi(jamp[10], a157);
    jadd_pi(jamp[13], a157);
    jadd_mi(jamp[14], a157);
    jadd_pi(jamp[15], a157);
    jadd_mi(jamp[16], a157);
    jadd_pi(jamp[18], a157);
    jadd_mi(jamp[5], a158);
    jadd_pi(jamp[7], a158);
    jadd_mi(jamp[8], a158);
    jadd_pi(jamp[9], a158);
    jadd_mi(jamp[10], a158);
    jadd_pi(jamp[13], a158);
    jadd_mi(jamp[16], a158);
    jadd_pi(jamp[19], a158);
    jadd_pi(jamp[4], a159);
    jadd_mi(jamp[5], a159);
    jadd_mi(jamp[8], a159);
    jadd_pi(jamp[9], a159);
    jadd_pi(jamp[14], a159);
    jadd_mi(jamp[15], a159);
    jadd_mi(jamp[18], a159);
    jadd_pi(jamp[19], a159);
    if constexpr (!CSUM) return R(0);   // the caller sums the colour flows left in the slot
    cx<R> J[NCOL];
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) J[c] = mkc(vget(jamp[c].r), vget(jamp[c].i));
    R me = R(0);
    { const R zr = R(512.0) * J[0].r + R(-128.0) * J[1].r + R(-128.0) * J[2].r + R(16.0) * J[3].r + R(16.0) * J[4].r + R(160.0) * J[5].r + R(-128.0) * J[6].r + R(16.0) * J[7].r + R(16.0) * J[8].r + R(-2.0) * J[9].r + R(-2.0) * J[10].r + R(-20.0) * J[11].r + R(16.0) * J[12].r + R(-2.0) * J[13].r + R(160.0) * J[14].r + R(-20.0) * J[15].r + R(142.0) * J[16].r + R(124.0) * J[17].r + R(-2.0) * J[18].r + R(-20.0) * J[19].r + R(-20.0) * J[20].r + R(124.0) * J[21].r + R(124.0) * J[22].r + R(-56.0) * J[23].r; const R zi = R(512.0) * J[0].i + R(-128.0) * J[1].i + R(-128.0) * J[2].i + R(16.0) * J[3].i + R(16.0) * J[4].i + R(160.0) * J[5].i + R(-128.0) * J[6].i + R(16.0) * J[7].i + R(16.0) * J[8].i + R(-2.0) * J[9].i + R(-2.0) * J[10].i + R(-20.0) * J[11].i + R(16.0) * J[12].i + R(-2.0) * J[13].i + R(160.0) * J[14].i + R(-20.0) * J[15].i + R(142.0) * J[16].i + R(124.0) * J[17].i + R(-2.0) * J[18].i + R(-20.0) * J[19].i + R(-20.0) * J[20].i + R(124.0) * J[21].i + R(124.0) * J[22].i + R(-56.0) * J[23].i;
      me = fma(J[0].r, zr, fma(J[0].i, zi, me)); }
    { const R zr = R(512.0) * J[1].r + R(16.0) * J[2].r + R(160.0) * J[3].r + R(-128.0) * J[4].r + R(16.0) * J[5].r + R(16.0) * J[6].r + R(-128.0) * J[7].r + R(-2.0) * J[8].r + R(-20.0) * J[9].r + R(16.0) * J[10].r + R(-2.0) * J[11].r + R(-2.0) * J[12].r + R(-20.0) * J[13].r + R(-20.0) * J[14].r + R(124.0) * J[15].r + R(124.0) * J[16].r + R(-56.0) * J[17].r + R(16.0) * J[18].r + R(-2.0) * J[19].r + R(160.0) * J[20].r + R(-20.0) * J[21].r + R(142.0) * J[22].r + R(124.0) * J[23].r; const R zi = R(512.0) * J[1].i + R(16.0) * J[2].i + R(160.0) * J[3].i + R(-128.0) * J[4].i + R(16.0) * J[5].i + R(16.0) * J[6].i + R(-128.0) * J[7].i + R(-2.0) * J[8].i + R(-20.0) * J[9].i + R(16.0) * J[10].i + R(-2.0) * J[11].i + R(-2.0) * J[12].i + R(-20.0) * J[13].i + R(-20.0) * J[14].i + R(124.0) * J[15].i + R(124.0) * J[16].i + R(-56.0) * J[17].i + R(16.0) * J[18].i + R(-2.0) * J[19].i + R(160.0) * J[20].i + R(-20.0) * J[21].i + R(142.0) * J[22].i + R(124.0) * J[23].i;
      me = fma(J[1].r, zr, fma(J[1].i, zi, me)); }
    { const R zr = R(512.0) * J[2].r + R(-128.0) * J[3].r + R(160.0) * J[4].r + R(16.0) * J[5].r + R(16.0) * J[6].r + R(-2.0) * J[7].r + R(160.0) * J[8].r + R(-20.0) * J[9].r + R(142.0) * J[10].r + R(124.0) * J[11].r + R(-128.0) * J[12].r + R(16.0) * J[13].r + R(16.0) * J[14].r + R(-2.0) * J[15].r + R(-2.0) * J[16].r + R(-20.0) * J[17].r + R(-20.0) * J[18].r + R(-2.0) * J[19].r + R(124.0) * J[20].r + R(-56.0) * J[21].r + R(-20.0) * J[22].r + R(124.0) * J[23].r; const R zi = R(512.0) * J[2].i + R(-128.0) * J[3].i + R(160.0) * J[4].i + R(16.0) * J[5].i + R(16.0) * J[6].i + R(-2.0) * J[7].i + R(160.0) * J[8].i + R(-20.0) * J[9].i + R(142.0) * J[10].i + R(124.0) * J[11].i + R(-128.0) * J[12].i + R(16.0) * J[13].i + R(16.0) * J[14].i + R(-2.0) * J[15].i + R(-2.0) * J[16].i + R(-20.0) * J[17].i + R(-20.0) * J[18].i + R(-2.0) * J[19].i + R(124.0) * J[20].i + R(-56.0) * J[21].i + R(-20.0) * J[22].i + R(124.0) * J[23].i;
      me = fma(J[2].r, zr, fma(J[2].i, zi, me)); }
    { const R zr = R(512.0) * J[3].r + R(16.0) * J[4].r + R(-128.0) * J[5].r + R(-2.0) * J[6].r + R(-20.0) * J[7].r + R(-20.0) * J[8].r + R(124.0) * J[9].r + R(124.0) * J[10].r + R(-56.0) * J[11].r + R(16.0) * J[12].r + R(-128.0) * J[13].r + R(-2.0) * J[14].r + R(-20.0) * J[15].r + R(16.0) * J[16].r + R(-2.0) * J[17].r + R(-2.0) * J[18].r + R(16.0) * J[19].r + R(142.0) * J[20].r + R(124.0) * J[21].r + R(160.0) * J[22].r + R(-20.0) * J[23].r; const R zi = R(512.0) * J[3].i + R(16.0) * J[4].i + R(-128.0) * J[5].i + R(-2.0) * J[6].i + R(-20.0) * J[7].i + R(-20.0) * J[8].i + R(124.0) * J[9].i + R(124.0) * J[10].i + R(-56.0) * J[11].i + R(16.0) * J[12].i + R(-128.0) * J[13].i + R(-2.0) * J[14].i + R(-20.0) * J[15].i + R(16.0) * J[16].i + R(-2.0) * J[17].i + R(-2.0) * J[18].i + R(16.0) * J[19].i + R(142.0) * J[20].i + R(124.0) * J[21].i + R(160.0) * J[22].i + R(-20.0) * J[23].i;
      me = fma(J[3].r, zr, fma(J[3].i, zi, me)); }
    { const R zr = R(512.0) * J[4].r + R(-128.0) * J[5].r + R(-2.0) * J[6].r + R(16.0) * J[7].r + R(142.0) * J[8].r + R(124.0) * J[9].r + R(160.0) * J[10].r + R(-20.0) * J[11].r + R(-20.0) * J[12].r + R(-2.0) * J[13].r + R(124.0) * J[14].r + R(-56.0) * J[15].r + R(-20.0) * J[16].r + R(124.0) * J[17].r + R(-128.0) * J[18].r + R(16.0) * J[19].r + R(16.0) * J[20].r + R(-2.0) * J[21].r + R(-2.0) * J[22].r + R(-20.0) * J[23].r; const R zi = R(512.0) * J[4].i + R(-128.0) * J[5].i + R(-2.0) * J[6].i + R(16.0) * J[7].i + R(142.0) * J[8].i + R(124.0) * J[9].i + R(160.0) * J[10].i + R(-20.0) * J[11].i + R(-20.0) * J[12].i + R(-2.0) * J[13].i + R(124.0) * J[14].i + R(-56.0) * J[15].i + R(-20.0) * J[16].i + R(124.0) * J[17].i + R(-128.0) * J[18].i + R(16.0) * J[19].i + R(16.0) * J[20].i + R(-2.0) * J[21].i + R(-2.0) * J[22].i + R(-20.0) * J[23].i;
      me = fma(J[4].r, zr, fma(J[4].i, zi, me)); }
    { const R zr = R(512.0) * J[5].r + R(-20.0) * J[6].r + R(-2.0) * J[7].r + R(124.0) * J[8].r + R(-56.0) * J[9].r + R(-20.0) * J[10].r + R(124.0) * J[11].r + R(-2.0) * J[12].r + R(16.0) * J[13].r + R(142.0) * J[14].r + R(124.0) * J[15].r + R(160.0) * J[16].r + R(-20.0) * J[17].r + R(16.0) * J[18].r + R(-128.0) * J[19].r + R(-2.0) * J[20].r + R(-20.0) * J[21].r + R(16.0) * J[22].r + R(-2.0) * J[23].r; const R zi = R(512.0) * J[5].i + R(-20.0) * J[6].i + R(-2.0) * J[7].i + R(124.0) * J[8].i + R(-56.0) * J[9].i + R(-20.0) * J[10].i + R(124.0) * J[11].i + R(-2.0) * J[12].i + R(16.0) * J[13].i + R(142.0) * J[14].i + R(124.0) * J[15].i + R(160.0) * J[16].i + R(-20.0) * J[17].i + R(16.0) * J[18].i + R(-128.0) * J[19].i + R(-2.0) * J[20].i + R(-20.0) * J[21].i + R(16.0) * J[22].i + R(-2.0) * J[23].i;
      me = fma(J[5].r, zr, fma(J[5].i, zi, me)); }
    { const R zr = R(512.0) * J[6].r + R(-128.0) * J[7].r + R(-128.0) * J[8].r + R(16.0) * J[9].r + R(16.0) * J[10].r + R(160.0) * J[11].r + R(160.0) * J[12].r + R(-20.0) * J[13].r + R(16.0) * J[14].r + R(-2.0) * J[15].r + R(124.0) * J[16].r + R(142.0) * J[17].r + R(-20.0) * J[18].r + R(124.0) * J[19].r + R(-2.0) * J[20].r + R(-20.0) * J[21].r + R(-56.0) * J[22].r + R(124.0) * J[23].r; const R zi = R(512.0) * J[6].i + R(-128.0) * J[7].i + R(-128.0) * J[8].i + R(16.0) * J[9].i + R(16.0) * J[10].i + R(160.0) * J[11].i + R(160.0) * J[12].i + R(-20.0) * J[13].i + R(16.0) * J[14].i + R(-2.0) * J[15].i + R(124.0) * J[16].i + R(142.0) * J[17].i + R(-20.0) * J[18].i + R(124.0) * J[19].i + R(-2.0) * J[20].i + R(-20.0) * J[21].i + R(-56.0) * J[22].i + R(124.0) * J[23].i;
      me = fma(J[6].r, zr, fma(J[6].i, zi, me)); }
    { const R zr = R(512.0) * J[7].r + R(16.0) * J[8].r + R(160.0) * J[9].r + R(-128.0) * J[10].r + R(16.0) * J[11].r + R(-20.0) * J[12].r + R(124.0) * J[13].r + R(-2.0) * J[14].r + R(-20.0) * J[15].r + R(-56.0) * J[16].r + R(124.0) * J[17].r + R(160.0) * J[18].r + R(-20.0) * J[19].r + R(16.0) * J[20].r + R(-2.0) * J[21].r + R(124.0) * J[22].r + R(142.0) * J[23].r; const R zi = R(512.0) * J[7].i + R(16.0) * J[8].i + R(160.0) * J[9].i + R(-128.0) * J[10].i + R(16.0) * J[11].i + R(-20.0) * J[12].i + R(124.0) * J[13].i + R(-2.0) * J[14].i + R(-20.0) * J[15].i + R(-56.0) * J[16].i + R(124.0) * J[17].i + R(160.0) * J[18].i + R(-20.0) * J[19].i + R(16.0) * J[20].i + R(-2.0) * J[21].i + R(124.0) * J[22].i + R(142.0) * J[23].i;
      me = fma(J[7].r, zr, fma(J[7].i, zi, me)); }
    { const R zr = R(512.0) * J[8].r + R(-128.0) * J[9].r + R(160.0) * J[10].r + R(16.0) * J[11].r + R(16.0) * J[12].r + R(-2.0) * J[13].r + R(-128.0) * J[14].r + R(16.0) * J[15].r + R(-20.0) * J[16].r + R(-2.0) * J[17].r + R(124.0) * J[18].r + R(-56.0) * J[19].r + R(-20.0) * J[20].r + R(-2.0) * J[21].r + R(124.0) * J[22].r + R(-20.0) * J[23].r; const R zi = R(512.0) * J[8].i + R(-128.0) * J[9].i + R(160.0) * J[10].i + R(16.0) * J[11].i + R(16.0) * J[12].i + R(-2.0) * J[13].i + R(-128.0) * J[14].i + R(16.0) * J[15].i + R(-20.0) * J[16].i + R(-2.0) * J[17].i + R(124.0) * J[18].i + R(-56.0) * J[19].i + R(-20.0) * J[20].i + R(-2.0) * J[21].i + R(124.0) * J[22].i + R(-20.0) * J[23].i;
      me = fma(J[8].r, zr, fma(J[8].i, zi, me)); }
    { const R zr = R(512.0) * J[9].r + R(16.0) * J[10].r + R(-128.0) * J[11].r + R(-2.0) * J[12].r + R(-20.0) * J[13].r + R(16.0) * J[14].r + R(-128.0) * J[15].r + R(-2.0) * J[16].r + R(16.0) * J[17].r + R(142.0) * J[18].r + R(124.0) * J[19].r + R(-2.0) * J[20].r + R(16.0) * J[21].r + R(-20.0) * J[22].r + R(160.0) * J[23].r; const R zi = R(512.0) * J[9].i + R(16.0) * J[10].i + R(-128.0) * J[11].i + R(-2.0) * J[12].i + R(-20.0) * J[13].i + R(16.0) * J[14].i + R(-128.0) * J[15].i + R(-2.0) * J[16].i + R(16.0) * J[17].i + R(142.0) * J[18].i + R(124.0) * J[19].i + R(-2.0) * J[20].i + R(16.0) * J[21].i + R(-20.0) * J[22].i + R(160.0) * J[23].i;
      me = fma(J[9].r, zr, fma(J[9].i, zi, me)); }
    { const R zr = R(512.0) * J[10].r + R(-128.0) * J[11].r + R(124.0) * J[12].r + R(-56.0) * J[13].r + R(-20.0) * J[14].r + R(-2.0) * J[15].r + R(124.0) * J[16].r + R(-20.0) * J[17].r + R(16.0) * J[18].r + R(-2.0) * J[19].r + R(-128.0) * J[20].r + R(16.0) * J[21].r + R(-20.0) * J[22].r + R(-2.0) * J[23].r; const R zi = R(512.0) * J[10].i + R(-128.0) * J[11].i + R(124.0) * J[12].i + R(-56.0) * J[13].i + R(-20.0) * J[14].i + R(-2.0) * J[15].i + R(124.0) * J[16].i + R(-20.0) * J[17].i + R(16.0) * J[18].i + R(-2.0) * J[19].i + R(-128.0) * J[20].i + R(16.0) * J[21].i + R(-20.0) * J[22].i + R(-2.0) * J[23].i;
      me = fma(J[10].r, zr, fma(J[10].i, zi, me)); }
    { const R zr = R(512.0) * J[11].r + R(142.0) * J[12].r + R(124.0) * J[13].r + R(-2.0) * J[14].r + R(16.0) * J[15].r + R(-20.0) * J[16].r + R(160.0) * J[17].r + R(-2.0) * J[18].r + R(-20.0) * J[19].r + R(16.0) * J[20].r + R(-128.0) * J[21].r + R(-2.0) * J[22].r + R(16.0) * J[23].r; const R zi = R(512.0) * J[11].i + R(142.0) * J[12].i + R(124.0) * J[13].i + R(-2.0) * J[14].i + R(16.0) * J[15].i + R(-20.0) * J[16].i + R(160.0) * J[17].i + R(-2.0) * J[18].i + R(-20.0) * J[19].i + R(16.0) * J[20].i + R(-128.0) * J[21].i + R(-2.0) * J[22].i + R(16.0) * J[23].i;
      me = fma(J[11].r, zr, fma(J[11].i, zi, me)); }
    { const R zr = R(512.0) * J[12].r + R(-128.0) * J[13].r + R(-128.0) * J[14].r + R(16.0) * J[15].r + R(16.0) * J[16].r + R(160.0) * J[17].r + R(124.0) * J[18].r + R(-20.0) * J[19].r + R(-56.0) * J[20].r + R(124.0) * J[21].r + R(-2.0) * J[22].r + R(-20.0) * J[23].r; const R zi = R(512.0) * J[12].i + R(-128.0) * J[13].i + R(-128.0) * J[14].i + R(16.0) * J[15].i + R(16.0) * J[16].i + R(160.0) * J[17].i + R(124.0) * J[18].i + R(-20.0) * J[19].i + R(-56.0) * J[20].i + R(124.0) * J[21].i + R(-2.0) * J[22].i + R(-20.0) * J[23].i;
      me = fma(J[12].r, zr, fma(J[12].i, zi, me)); }
    { const R zr = R(512.0) * J[13].r + R(16.0) * J[14].r + R(160.0) * J[15].r + R(-128.0) * J[16].r + R(16.0) * J[17].r + R(-20.0) * J[18].r + R(160.0) * J[19].r + R(124.0) * J[20].r + R(142.0) * J[21].r + R(16.0) * J[22].r + R(-2.0) * J[23].r; const R zi = R(512.0) * J[13].i + R(16.0) * J[14].i + R(160.0) * J[15].i + R(-128.0) * J[16].i + R(16.0) * J[17].i + R(-20.0) * J[18].i + R(160.0) * J[19].i + R(124.0) * J[20].i + R(142.0) * J[21].i + R(16.0) * J[22].i + R(-2.0) * J[23].i;
      me = fma(J[13].r, zr, fma(J[13].i, zi, me)); }
    { const R zr = R(512.0) * J[14].r + R(-128.0) * J[15].r + R(160.0) * J[16].r + R(16.0) * J[17].r + R(-56.0) * J[18].r + R(124.0) * J[19].r + R(124.0) * J[20].r + R(-20.0) * J[21].r + R(-20.0) * J[22].r + R(-2.0) * J[23].r; const R zi = R(512.0) * J[14].i + R(-128.0) * J[15].i + R(160.0) * J[16].i + R(16.0) * J[17].i + R(-56.0) * J[18].i + R(124.0) * J[19].i + R(124.0) * J[20].i + R(-20.0) * J[21].i + R(-20.0) * J[22].i + R(-2.0) * J[23].i;
      me = fma(J[14].r, zr, fma(J[14].i, zi, me)); }
    { const R zr = R(512.0) * J[15].r + R(16.0) * J[16].r + R(-128.0) * J[17].r + R(124.0) * J[18].r + R(142.0) * J[19].r + R(-20.0) * J[20].r + R(160.0) * J[21].r + R(-2.0) * J[22].r + R(16.0) * J[23].r; const R zi = R(512.0) * J[15].i + R(16.0) * J[16].i + R(-128.0) * J[17].i + R(124.0) * J[18].i + R(142.0) * J[19].i + R(-20.0) * J[20].i + R(160.0) * J[21].i + R(-2.0) * J[22].i + R(16.0) * J[23].i;
      me = fma(J[15].r, zr, fma(J[15].i, zi, me)); }
    { const R zr = R(512.0) * J[16].r + R(-128.0) * J[17].r + R(-2.0) * J[18].r + R(16.0) * J[19].r + R(-20.0) * J[20].r + R(-2.0) * J[21].r + R(-128.0) * J[22].r + R(16.0) * J[23].r; const R zi = R(512.0) * J[16].i + R(-128.0) * J[17].i + R(-2.0) * J[18].i + R(16.0) * J[19].i + R(-20.0) * J[20].i + R(-2.0) * J[21].i + R(-128.0) * J[22].i + R(16.0) * J[23].i;
      me = fma(J[16].r, zr, fma(J[16].i, zi, me)); }
    { const R zr = R(512.0) * J[17].r + R(-20.0) * J[18].r + R(-2.0) * J[19].r + R(-2.0) * J[20].r + R(16.0) * J[21].r + R(16.0) * J[22].r + R(-128.0) * J[23].r; const R zi = R(512.0) * J[17].i + R(-20.0) * J[18].i + R(-2.0) * J[19].i + R(-2.0) * J[20].i + R(16.0) * J[21].i + R(16.0) * J[22].i + R(-128.0) * J[23].i;
      me = fma(J[17].r, zr, fma(J[17].i, zi, me)); }
    { const R zr = R(512.0) * J[18].r + R(-128.0) * J[19].r + R(-128.0) * J[20].r + R(16.0) * J[21].r + R(16.0) * J[22].r + R(160.0) * J[23].r; const R zi = R(512.0) * J[18].i + R(-128.0) * J[19].i + R(-128.0) * J[20].i + R(16.0) * J[21].i + R(16.0) * J[22].i + R(160.0) * J[23].i;
      me = fma(J[18].r, zr, fma(J[18].i, zi, me)); }
    { const R zr = R(512.0) * J[19].r + R(16.0) * J[20].r + R(160.0) * J[21].r + R(-128.0) * J[22].r + R(16.0) * J[23].r; const R zi = R(512.0) * J[19].i + R(16.0) * J[20].i + R(160.0) * J[21].i + R(-128.0) * J[22].i + R(16.0) * J[23].i;
      me = fma(J[19].r, zr, fma(J[19].i, zi, me)); }
    { const R zr = R(512.0) * J[20].r + R(-128.0) * J[21].r + R(160.0) * J[22].r + R(16.0) * J[23].r; const R zi = R(512.0) * J[20].i + R(-128.0) * J[21].i + R(160.0) * J[22].i + R(16.0) * J[23].i;
      me = fma(J[20].r, zr, fma(J[20].i, zi, me)); }
    { const R zr = R(512.0) * J[21].r + R(16.0) * J[22].r + R(-128.0) * J[23].r; const R zi = R(512.0) * J[21].i + R(16.0) * J[22].i + R(-128.0) * J[23].i;
      me = fma(J[21].r, zr, fma(J[21].i, zi, me)); }
    { const R zr = R(512.0) * J[22].r + R(-128.0) * J[23].r; const R zi = R(512.0) * J[22].i + R(-128.0) * J[23].i;
      me = fma(J[22].r, zr, fma(J[22].i, zi, me)); }
    { const R zr = R(512.0) * J[23].r; const R zi = R(512.0) * J[23].i;
      me = fma(J[23].r, zr, fma(J[23].i, zi, me)); }
    return me;
#undef HEL
}

template <typename R, bool SYNC, bool TC, typename S>
__device__ __noinline__ S me2_gg_ttgg_impl(const S* pflat, S mt, S gs, void* slot, void* cta, int hpart,
                                       int hparts)
{
    constexpr int NEXT = Me_gg_ttgg::NEXT, NHEL = Me_gg_ttgg::NHEL, NGLUON = Me_gg_ttgg::NGLUON;
    constexpr double COLOUR_DEN = Me_gg_ttgg::COLOUR_DEN, AVG = Me_gg_ttgg::AVG, SYM = Me_gg_ttgg::SYM;
    S p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    Me_gg_ttgg::Inv<R> local;   // used when the caller has no shared-memory slot
    Me_gg_ttgg::Inv<R>& v = slot ? *static_cast<Me_gg_ttgg::Inv<R>*>(slot) : local;
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const S kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const S kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const S kd4[4] = {-p[4][0], -p[4][1], -p[4][2], -p[4][3]};
    const S kd8[4] = {-p[5][0], -p[5][1], -p[5][2], -p[5][3]};
    const S kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    const S kd5[4] = {kd1[0] + kd4[0], kd1[1] + kd4[1], kd1[2] + kd4[2], kd1[3] + kd4[3]};
    const S kd6[4] = {kd2[0] + kd4[0], kd2[1] + kd4[1], kd2[2] + kd4[2], kd2[3] + kd4[3]};
    const S kd9[4] = {kd1[0] + kd8[0], kd1[1] + kd8[1], kd1[2] + kd8[2], kd1[3] + kd8[3]};
    const S kd10[4] = {kd2[0] + kd8[0], kd2[1] + kd8[1], kd2[2] + kd8[2], kd2[3] + kd8[3]};
    const S kd12[4] = {kd4[0] + kd8[0], kd4[1] + kd8[1], kd4[2] + kd8[2], kd4[3] + kd8[3]};
    const S kd7[4] = {kd1[0] + kd2[0] + kd4[0], kd1[1] + kd2[1] + kd4[1], kd1[2] + kd2[2] + kd4[2], kd1[3] + kd2[3] + kd4[3]};
    const S kd11[4] = {kd1[0] + kd2[0] + kd8[0], kd1[1] + kd2[1] + kd8[1], kd1[2] + kd2[2] + kd8[2], kd1[3] + kd2[3] + kd8[3]};
    const S kd13[4] = {kd1[0] + kd4[0] + kd8[0], kd1[1] + kd4[1] + kd8[1], kd1[2] + kd4[2] + kd8[2], kd1[3] + kd4[3] + kd8[3]};
    const S kd14[4] = {kd2[0] + kd4[0] + kd8[0], kd2[1] + kd4[1] + kd8[1], kd2[2] + kd4[2] + kd8[2], kd2[3] + kd4[3] + kd8[3]};
    const S kd15[4] = {kd1[0] + kd2[0] + kd4[0] + kd8[0], kd1[1] + kd2[1] + kd4[1] + kd8[1], kd1[2] + kd2[2] + kd4[2] + kd8[2], kd1[3] + kd2[3] + kd4[3] + kd8[3]};
    for (int c = 0; c < 4; ++c) v.K[0][c] = R(kd1[c]);
    for (int c = 0; c < 4; ++c) v.K[1][c] = R(kd2[c]);
    for (int c = 0; c < 4; ++c) v.K[2][c] = R(kd3[c]);
    for (int c = 0; c < 4; ++c) v.K[3][c] = R(kd4[c]);
    for (int c = 0; c < 4; ++c) v.K[4][c] = R(kd5[c]);
    for (int c = 0; c < 4; ++c) v.K[5][c] = R(kd6[c]);
    for (int c = 0; c < 4; ++c) v.K[6][c] = R(kd7[c]);
    for (int c = 0; c < 4; ++c) v.K[7][c] = R(kd8[c]);
    for (int c = 0; c < 4; ++c) v.K[8][c] = R(kd9[c]);
    for (int c = 0; c < 4; ++c) v.K[9][c] = R(kd10[c]);
    for (int c = 0; c < 4; ++c) v.K[10][c] = R(kd11[c]);
    for (int c = 0; c < 4; ++c) v.K[11][c] = R(kd12[c]);
    for (int c = 0; c < 4; ++c) v.K[12][c] = R(kd13[c]);
    for (int c = 0; c < 4; ++c) v.K[13][c] = R(kd14[c]);
    for (int c = 0; c < 4; ++c) v.K[14][c] = R(kd15[c]);
    for (int c = 0; c < 4; ++c) v.p3[c] = R(p[2][c]);
    v.iG[0] = R(1.0 / mdot(kd3, kd3));
    v.iG[1] = R(1.0 / mdot(kd5, kd5));
    v.iG[2] = R(1.0 / mdot(kd6, kd6));
    v.iG[3] = R(1.0 / mdot(kd7, kd7));
    v.iG[4] = R(1.0 / mdot(kd9, kd9));
    v.iG[5] = R(1.0 / mdot(kd10, kd10));
    v.iG[6] = R(1.0 / mdot(kd11, kd11));
    v.iG[7] = R(1.0 / mdot(kd12, kd12));
    v.iG[8] = R(1.0 / mdot(kd13, kd13));
    v.iG[9] = R(1.0 / mdot(kd14, kd14));
    v.iG[10] = R(1.0 / mdot(kd15, kd15));
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
    { const S q[4] = {p[2][0] - kd7[0], p[2][1] - kd7[1], p[2][2] - kd7[2], p[2][3] - kd7[3]};
      v.iQ[6] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd8[0], p[2][1] - kd8[1], p[2][2] - kd8[2], p[2][3] - kd8[3]};
      v.iQ[7] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd9[0], p[2][1] - kd9[1], p[2][2] - kd9[2], p[2][3] - kd9[3]};
      v.iQ[8] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd10[0], p[2][1] - kd10[1], p[2][2] - kd10[2], p[2][3] - kd10[3]};
      v.iQ[9] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd11[0], p[2][1] - kd11[1], p[2][2] - kd11[2], p[2][3] - kd11[3]};
      v.iQ[10] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd12[0], p[2][1] - kd12[1], p[2][2] - kd12[2], p[2][3] - kd12[3]};
      v.iQ[11] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd13[0], p[2][1] - kd13[1], p[2][2] - kd13[2], p[2][3] - kd13[3]};
      v.iQ[12] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd14[0], p[2][1] - kd14[1], p[2][2] - kd14[2], p[2][3] - kd14[3]};
      v.iQ[13] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { S a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[4], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[2][j] = R(a[j]); v.e2[2][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[5], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[3][j] = R(a[j]); v.e2[3][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
    // Parity: flipping every helicity leaves the colour-summed |M_h|^2 of these
    // tree amplitudes unchanged, so the sum over all helicities is twice the
    // sum over the configurations with the first gluon at helicity +1.
    R acc = R(0);
#pragma unroll 1
    for (int ih = 1 + 2 * hpart; ih < NHEL; ih += 2 * hparts) {
        if constexpr (TC) {
            // the colour sum synchronises the CTA itself (its barriers replace SYNC's)
            static_assert(SYNC && sizeof(R) == 4, "tensor-core colour sum: float, whole-CTA calls");
            hel_gg_ttgg<R, false>(v, ih);
            acc += tc_colour_sum<Me_gg_ttgg::NCOL>(static_cast<TcCta*>(cta),
                                                  reinterpret_cast<const volatile float*>(v.jamp));
        } else {
            acc += hel_gg_ttgg<R>(v, ih);
            if (SYNC) __syncthreads();
        }
    }
    acc *= R(2);
    S gk = S(1.0);
    for (int i = 0; i < NGLUON; ++i) gk = gk * (gs * gs);
    return S(acc) / COLOUR_DEN * gk * AVG * SYM;
}

template <typename R, bool SYNC, bool TC, typename S>
__device__ S Me_gg_ttgg::me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt,
    typename NoDeduce<S>::type gs, void* slot, void* cta, int hpart, int hparts)
{
    return me2_gg_ttgg_impl<R, SYNC, TC, S>(&p[0][0], mt, gs, slot, cta, hpart, hparts);
}

// the prologue of me2 alone: the event's helicity-independent pieces into v
template <typename R>
__device__ __forceinline__ void inv_gg_ttgg(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,
                                       Me_gg_ttgg::Inv<R>& v)
{
    using S = typename Widen<R>::type;
    constexpr int NEXT = Me_gg_ttgg::NEXT;
    S p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const S kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const S kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const S kd4[4] = {-p[4][0], -p[4][1], -p[4][2], -p[4][3]};
    const S kd8[4] = {-p[5][0], -p[5][1], -p[5][2], -p[5][3]};
    const S kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    const S kd5[4] = {kd1[0] + kd4[0], kd1[1] + kd4[1], kd1[2] + kd4[2], kd1[3] + kd4[3]};
    const S kd6[4] = {kd2[0] + kd4[0], kd2[1] + kd4[1], kd2[2] + kd4[2], kd2[3] + kd4[3]};
    const S kd9[4] = {kd1[0] + kd8[0], kd1[1] + kd8[1], kd1[2] + kd8[2], kd1[3] + kd8[3]};
    const S kd10[4] = {kd2[0] + kd8[0], kd2[1] + kd8[1], kd2[2] + kd8[2], kd2[3] + kd8[3]};
    const S kd12[4] = {kd4[0] + kd8[0], kd4[1] + kd8[1], kd4[2] + kd8[2], kd4[3] + kd8[3]};
    const S kd7[4] = {kd1[0] + kd2[0] + kd4[0], kd1[1] + kd2[1] + kd4[1], kd1[2] + kd2[2] + kd4[2], kd1[3] + kd2[3] + kd4[3]};
    const S kd11[4] = {kd1[0] + kd2[0] + kd8[0], kd1[1] + kd2[1] + kd8[1], kd1[2] + kd2[2] + kd8[2], kd1[3] + kd2[3] + kd8[3]};
    const S kd13[4] = {kd1[0] + kd4[0] + kd8[0], kd1[1] + kd4[1] + kd8[1], kd1[2] + kd4[2] + kd8[2], kd1[3] + kd4[3] + kd8[3]};
    const S kd14[4] = {kd2[0] + kd4[0] + kd8[0], kd2[1] + kd4[1] + kd8[1], kd2[2] + kd4[2] + kd8[2], kd2[3] + kd4[3] + kd8[3]};
    const S kd15[4] = {kd1[0] + kd2[0] + kd4[0] + kd8[0], kd1[1] + kd2[1] + kd4[1] + kd8[1], kd1[2] + kd2[2] + kd4[2] + kd8[2], kd1[3] + kd2[3] + kd4[3] + kd8[3]};
    for (int c = 0; c < 4; ++c) v.K[0][c] = R(kd1[c]);
    for (int c = 0; c < 4; ++c) v.K[1][c] = R(kd2[c]);
    for (int c = 0; c < 4; ++c) v.K[2][c] = R(kd3[c]);
    for (int c = 0; c < 4; ++c) v.K[3][c] = R(kd4[c]);
    for (int c = 0; c < 4; ++c) v.K[4][c] = R(kd5[c]);
    for (int c = 0; c < 4; ++c) v.K[5][c] = R(kd6[c]);
    for (int c = 0; c < 4; ++c) v.K[6][c] = R(kd7[c]);
    for (int c = 0; c < 4; ++c) v.K[7][c] = R(kd8[c]);
    for (int c = 0; c < 4; ++c) v.K[8][c] = R(kd9[c]);
    for (int c = 0; c < 4; ++c) v.K[9][c] = R(kd10[c]);
    for (int c = 0; c < 4; ++c) v.K[10][c] = R(kd11[c]);
    for (int c = 0; c < 4; ++c) v.K[11][c] = R(kd12[c]);
    for (int c = 0; c < 4; ++c) v.K[12][c] = R(kd13[c]);
    for (int c = 0; c < 4; ++c) v.K[13][c] = R(kd14[c]);
    for (int c = 0; c < 4; ++c) v.K[14][c] = R(kd15[c]);
    for (int c = 0; c < 4; ++c) v.p3[c] = R(p[2][c]);
    v.iG[0] = R(1.0 / mdot(kd3, kd3));
    v.iG[1] = R(1.0 / mdot(kd5, kd5));
    v.iG[2] = R(1.0 / mdot(kd6, kd6));
    v.iG[3] = R(1.0 / mdot(kd7, kd7));
    v.iG[4] = R(1.0 / mdot(kd9, kd9));
    v.iG[5] = R(1.0 / mdot(kd10, kd10));
    v.iG[6] = R(1.0 / mdot(kd11, kd11));
    v.iG[7] = R(1.0 / mdot(kd12, kd12));
    v.iG[8] = R(1.0 / mdot(kd13, kd13));
    v.iG[9] = R(1.0 / mdot(kd14, kd14));
    v.iG[10] = R(1.0 / mdot(kd15, kd15));
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
    { const S q[4] = {p[2][0] - kd7[0], p[2][1] - kd7[1], p[2][2] - kd7[2], p[2][3] - kd7[3]};
      v.iQ[6] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd8[0], p[2][1] - kd8[1], p[2][2] - kd8[2], p[2][3] - kd8[3]};
      v.iQ[7] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd9[0], p[2][1] - kd9[1], p[2][2] - kd9[2], p[2][3] - kd9[3]};
      v.iQ[8] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd10[0], p[2][1] - kd10[1], p[2][2] - kd10[2], p[2][3] - kd10[3]};
      v.iQ[9] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd11[0], p[2][1] - kd11[1], p[2][2] - kd11[2], p[2][3] - kd11[3]};
      v.iQ[10] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd12[0], p[2][1] - kd12[1], p[2][2] - kd12[2], p[2][3] - kd12[3]};
      v.iQ[11] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd13[0], p[2][1] - kd13[1], p[2][2] - kd13[2], p[2][3] - kd13[3]};
      v.iQ[12] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const S q[4] = {p[2][0] - kd14[0], p[2][1] - kd14[1], p[2][2] - kd14[2], p[2][3] - kd14[3]};
      v.iQ[13] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { S a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[4], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[2][j] = R(a[j]); v.e2[2][j] = R(b[j]); } }
    { S a[3], b[3]; gluon_basis(p[5], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[3][j] = R(a[j]); v.e2[3][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
}

// Helicity profile: the averaged |M_h|^2 of every one of the NHEL helicity configurations
// (ih bit i: helicity of external particle i, set = +1), parity mirrors included, so that
// out[ih] sums to me2 and out[ih] = out[ih ^ (NHEL - 1)] tests the parity halving of me2
template <typename R>
__device__ void hel_profile_gg_ttgg(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,
                                   typename Widen<R>::type gs, Me_gg_ttgg::Inv<R>& v, double* out)
{
    using S = typename Widen<R>::type;
    inv_gg_ttgg<R>(pflat, mt, v);
    S gk = S(1.0);
    for (int i = 0; i < Me_gg_ttgg::NGLUON; ++i) gk = gk * (gs * gs);
    for (int ih = 0; ih < Me_gg_ttgg::NHEL; ++ih)
        out[ih] = val(S(hel_gg_ttgg<R>(v, ih)) / Me_gg_ttgg::COLOUR_DEN * gk * Me_gg_ttgg::AVG * Me_gg_ttgg::SYM);
}
template <typename R>
__device__ void Me_gg_ttgg::hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,
                                  typename Widen<R>::type gs, double* out)
{
    Me_gg_ttgg::Inv<R> v;
    hel_profile_gg_ttgg<R>(&p[0][0], mt, gs, v, out);
}

// one helicity's colour-flow amplitudes (the same as hel_gg_ttgg, without the colour sum);
// the record and the colour-flow row sit at fixed offsets of dynamic shared memory, so that
// both addresses are shared-space offsets derived from threadIdx.x
// (R = float: the record's momenta are read 16 bytes and the colour flows
// updated 8 bytes at a time; REC_STRIDE and JROW keep them aligned)
template <typename R, int JROW, int REC_OFF, int REC_STRIDE>
__device__ __noinline__ void hel_gg_ttgg_j(int ih)
{
    constexpr int NCOL = Me_gg_ttgg::NCOL;
    static_assert(sizeof(R) == 4 && REC_OFF % 16 == 0 && REC_STRIDE % 16 == 0 && JROW % 2 == 0,
                  "aligned float records and colour-flow rows");
    extern __shared__ __align__(128) unsigned char mf_lh_smem[];
    const Me_gg_ttgg::Inv<R>& v = *reinterpret_cast<const Me_gg_ttgg::Inv<R>*>(
        mf_lh_smem + REC_OFF + (threadIdx.x >> 5) * REC_STRIDE);
    volatile cx<R>* jamp = reinterpret_cast<volatile cx<R>*>(mf_lh_smem + threadIdx.x * (JROW * sizeof(R)));
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) jzero64(jamp[c]);
    W4<R> g0; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[0][j]); b[j] = ldv(v.e2[0][j]); }
      g0 = ext_gluon(a, b, HEL(0), false); }
    W4<R> g1; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[1][j]); b[j] = ldv(v.e2[1][j]); }
      g1 = ext_gluon(a, b, HEL(1), false); }
    W4<R> g2; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[2][j]); b[j] = ldv(v.e2[2][j]); }
      g2 = ext_gluon(a, b, HEL(4), true); }
    W4<R> g3; { R a[3], b[3]; for (int j = 0; j < 3; ++j) { a[j] = ldv(v.e1[3][j]); b[j] = ldv(v.e2[3][j]); }
      g3 = ext_gluon(a, b, HEL(5), true); }
    const W4<R> ub3 = ext_ubar(load_basis(v.fb3), HEL(2));
    const W4<R> v4 = ext_v(load_basis(v.fb4), HEL(3));
    R k1_1[4]; ldv4(v.K[0], k1_1);
    R k2_2[4]; ldv4(v.K[1], k2_2);
    const W4<R> w3 = vvv_cur(g0, g1, k1_1, k2_2, ldv(v.iG[0]));
    R k1_4[4]; ldv4(v.K[0], k1_4);
    R k4_5[4]; ldv4(v.K[3], k4_5);
    const W4<R> w6 = vvv_cur(g0, g2, k1_4, k4_5, ldv(v.iG[1]));
    R k1_7[4]; ldv4(v.K[0], k1_7);
    R k8_8[4]; ldv4(v.K[7], k8_8);
    const W4<R> w9 = vvv_cur(g0, g3, k1_7, k8_8, ldv(v.iG[4]));
    R k2_10[4]; ldv4(v.K[1], k2_10);
    R k4_11[4]; ldv4(v.K[3], k4_11);
    const W4<R> w12 = vvv_cur(g1, g2, k2_10, k4_11, ldv(v.iG[2]));
    R k2_13[4]; ldv4(v.K[1], k2_13);
    R k8_14[4]; ldv4(v.K[7], k8_14);
    const W4<R> w15 = vvv_cur(g1, g3, k2_13, k8_14, ldv(v.iG[5]));
    R k4_16[4]; ldv4(v.K[3], k4_16);
    R k8_17[4]; ldv4(v.K[7], k8_17);
    const W4<R> w18 = vvv_cur(g2, g3, k4_16, k8_17, ldv(v.iG[7]));
    R q1_19[4]; ldv4_diff(v.p3, v.K[0], q1_19);
    const W4<R> w20 = ffv_row(ub3, g0, q1_19, ldv(v.mt), ldv(v.iQ[0]));
    R q3_21[4]; ldv4_diff(v.p3, v.K[2], q3_21);
    const W4<R> w22 = ffv_row(w20, g1, q3_21, ldv(v.mt), ldv(v.iQ[2]));
    R q7_24[4]; ldv4_diff(v.p3, v.K[6], q7_24);
    const W4<R> w23 = ffv_col(g3, v4, q7_24, ldv(v.mt), ldv(v.iQ[6]));
    const cx<R> a1 = ffv_amp(w22, w23, g2);
    jadd64_mi(jamp[0], a1);
    R q11_26[4]; ldv4_diff(v.p3, v.K[10], q11_26);
    const W4<R> w25 = ffv_col(g2, v4, q11_26, ldv(v.mt), ldv(v.iQ[10]));
    const cx<R> a2 = ffv_amp(w22, w25, g3);
    jadd64_mi(jamp[1], a2);
    const cx<R> a3 = ffv_amp(w22, v4, w18);
    jadd64_mi(jamp[0], a3);
    jadd64_pi(jamp[1], a3);
    R q5_27[4]; ldv4_diff(v.p3, v.K[4], q5_27);
    const W4<R> w28 = ffv_row(w20, g2, q5_27, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a4 = ffv_amp(w28, w23, g1);
    jadd64_mi(jamp[2], a4);
    R q13_30[4]; ldv4_diff(v.p3, v.K[12], q13_30);
    const W4<R> w29 = ffv_col(g1, v4, q13_30, ldv(v.mt), ldv(v.iQ[12]));
    const cx<R> a5 = ffv_amp(w28, w29, g3);
    jadd64_mi(jamp[3], a5);
    const cx<R> a6 = ffv_amp(w28, v4, w15);
    jadd64_mi(jamp[2], a6);
    jadd64_pi(jamp[3], a6);
    R q9_31[4]; ldv4_diff(v.p3, v.K[8], q9_31);
    const W4<R> w32 = ffv_row(w20, g3, q9_31, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a7 = ffv_amp(w32, w25, g1);
    jadd64_mi(jamp[4], a7);
    const cx<R> a8 = ffv_amp(w32, w29, g2);
    jadd64_mi(jamp[5], a8);
    const cx<R> a9 = ffv_amp(w32, v4, w12);
    jadd64_mi(jamp[4], a9);
    jadd64_pi(jamp[5], a9);
    const cx<R> a10 = ffv_amp(w20, w23, w12);
    jadd64_mi(jamp[0], a10);
    jadd64_pi(jamp[2], a10);
    const cx<R> a11 = ffv_amp(w20, w25, w15);
    jadd64_mi(jamp[1], a11);
    jadd64_pi(jamp[4], a11);
    const cx<R> a12 = ffv_amp(w20, w29, w18);
    jadd64_mi(jamp[3], a12);
    jadd64_pi(jamp[5], a12);
    R q2_33[4]; ldv4_diff(v.p3, v.K[1], q2_33);
    const W4<R> w34 = ffv_row(ub3, g1, q2_33, ldv(v.mt), ldv(v.iQ[1]));
    R q3_35[4]; ldv4_diff(v.p3, v.K[2], q3_35);
    const W4<R> w36 = ffv_row(w34, g0, q3_35, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a13 = ffv_amp(w36, w23, g2);
    jadd64_mi(jamp[6], a13);
    const cx<R> a14 = ffv_amp(w36, w25, g3);
    jadd64_mi(jamp[7], a14);
    const cx<R> a15 = ffv_amp(w36, v4, w18);
    jadd64_mi(jamp[6], a15);
    jadd64_pi(jamp[7], a15);
    R q6_37[4]; ldv4_diff(v.p3, v.K[5], q6_37);
    const W4<R> w38 = ffv_row(w34, g2, q6_37, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a16 = ffv_amp(w38, w23, g0);
    jadd64_mi(jamp[8], a16);
    R q14_40[4]; ldv4_diff(v.p3, v.K[13], q14_40);
    const W4<R> w39 = ffv_col(g0, v4, q14_40, ldv(v.mt), ldv(v.iQ[13]));
    const cx<R> a17 = ffv_amp(w38, w39, g3);
    jadd64_mi(jamp[9], a17);
    const cx<R> a18 = ffv_amp(w38, v4, w9);
    jadd64_mi(jamp[8], a18);
    jadd64_pi(jamp[9], a18);
    R q10_41[4]; ldv4_diff(v.p3, v.K[9], q10_41);
    const W4<R> w42 = ffv_row(w34, g3, q10_41, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a19 = ffv_amp(w42, w25, g0);
    jadd64_mi(jamp[10], a19);
    const cx<R> a20 = ffv_amp(w42, w39, g2);
    jadd64_mi(jamp[11], a20);
    const cx<R> a21 = ffv_amp(w42, v4, w6);
    jadd64_mi(jamp[10], a21);
    jadd64_pi(jamp[11], a21);
    const cx<R> a22 = ffv_amp(w34, w23, w6);
    jadd64_mi(jamp[6], a22);
    jadd64_pi(jamp[8], a22);
    const cx<R> a23 = ffv_amp(w34, w25, w9);
    jadd64_mi(jamp[7], a23);
    jadd64_pi(jamp[10], a23);
    const cx<R> a24 = ffv_amp(w34, w39, w18);
    jadd64_mi(jamp[9], a24);
    jadd64_pi(jamp[11], a24);
    R q4_43[4]; ldv4_diff(v.p3, v.K[3], q4_43);
    const W4<R> w44 = ffv_row(ub3, g2, q4_43, ldv(v.mt), ldv(v.iQ[3]));
    R q5_45[4]; ldv4_diff(v.p3, v.K[4], q5_45);
    const W4<R> w46 = ffv_row(w44, g0, q5_45, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a25 = ffv_amp(w46, w23, g1);
    jadd64_mi(jamp[12], a25);
    const cx<R> a26 = ffv_amp(w46, w29, g3);
    jadd64_mi(jamp[13], a26);
    const cx<R> a27 = ffv_amp(w46, v4, w15);
    jadd64_mi(jamp[12], a27);
    jadd64_pi(jamp[13], a27);
    R q6_47[4]; ldv4_diff(v.p3, v.K[5], q6_47);
    const W4<R> w48 = ffv_row(w44, g1, q6_47, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a28 = ffv_amp(w48, w23, g0);
    jadd64_mi(jamp[14], a28);
    const cx<R> a29 = ffv_amp(w48, w39, g3);
    jadd64_mi(jamp[15], a29);
    const cx<R> a30 = ffv_amp(w48, v4, w9);
    jadd64_mi(jamp[14], a30);
    jadd64_pi(jamp[15], a30);
    R q12_49[4]; ldv4_diff(v.p3, v.K[11], q12_49);
    const W4<R> w50 = ffv_row(w44, g3, q12_49, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a31 = ffv_amp(w50, w29, g0);
    jadd64_mi(jamp[16], a31);
    const cx<R> a32 = ffv_amp(w50, w39, g1);
    jadd64_mi(jamp[17], a32);
    const cx<R> a33 = ffv_amp(w50, v4, w3);
    jadd64_mi(jamp[16], a33);
    jadd64_pi(jamp[17], a33);
    const cx<R> a34 = ffv_amp(w44, w23, w3);
    jadd64_mi(jamp[12], a34);
    jadd64_pi(jamp[14], a34);
    const cx<R> a35 = ffv_amp(w44, w29, w9);
    jadd64_mi(jamp[13], a35);
    jadd64_pi(jamp[16], a35);
    const cx<R> a36 = ffv_amp(w44, w39, w15);
    jadd64_mi(jamp[15], a36);
    jadd64_pi(jamp[17], a36);
    R q8_51[4]; ldv4_diff(v.p3, v.K[7], q8_51);
    const W4<R> w52 = ffv_row(ub3, g3, q8_51, ldv(v.mt), ldv(v.iQ[7]));
    R q9_53[4]; ldv4_diff(v.p3, v.K[8], q9_53);
    const W4<R> w54 = ffv_row(w52, g0, q9_53, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a37 = ffv_amp(w54, w25, g1);
    jadd64_mi(jamp[18], a37);
    const cx<R> a38 = ffv_amp(w54, w29, g2);
    jadd64_mi(jamp[19], a38);
    const cx<R> a39 = ffv_amp(w54, v4, w12);
    jadd64_mi(jamp[18], a39);
    jadd64_pi(jamp[19], a39);
    R q10_55[4]; ldv4_diff(v.p3, v.K[9], q10_55);
    const W4<R> w56 = ffv_row(w52, g1, q10_55, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a40 = ffv_amp(w56, w25, g0);
    jadd64_mi(jamp[20], a40);
    const cx<R> a41 = ffv_amp(w56, w39, g2);
    jadd64_mi(jamp[21], a41);
    const cx<R> a42 = ffv_amp(w56, v4, w6);
    jadd64_mi(jamp[20], a42);
    jadd64_pi(jamp[21], a42);
    R q12_57[4]; ldv4_diff(v.p3, v.K[11], q12_57);
    const W4<R> w58 = ffv_row(w52, g2, q12_57, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a43 = ffv_amp(w58, w29, g0);
    jadd64_mi(jamp[22], a43);
    const cx<R> a44 = ffv_amp(w58, w39, g1);
    jadd64_mi(jamp[23], a44);
    const cx<R> a45 = ffv_amp(w58, v4, w3);
    jadd64_mi(jamp[22], a45);
    jadd64_pi(jamp[23], a45);
    const cx<R> a46 = ffv_amp(w52, w25, w3);
    jadd64_mi(jamp[18], a46);
    jadd64_pi(jamp[20], a46);
    const cx<R> a47 = ffv_amp(w52, w29, w6);
    jadd64_mi(jamp[19], a47);
    jadd64_pi(jamp[22], a47);
    const cx<R> a48 = ffv_amp(w52, w39, w12);
    jadd64_mi(jamp[21], a48);
    jadd64_pi(jamp[23], a48);
    R q3_59[4]; ldv4_diff(v.p3, v.K[2], q3_59);
    const W4<R> w60 = ffv_row(ub3, w3, q3_59, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a49 = ffv_amp(w60, w23, g2);
    jadd64_mi(jamp[0], a49);
    jadd64_pi(jamp[6], a49);
    const cx<R> a50 = ffv_amp(w60, w25, g3);
    jadd64_mi(jamp[1], a50);
    jadd64_pi(jamp[7], a50);
    const cx<R> a51 = ffv_amp(w60, v4, w18);
    jadd64_mi(jamp[0], a51);
    jadd64_pi(jamp[1], a51);
    jadd64_pi(jamp[6], a51);
    jadd64_mi(jamp[7], a51);
    R q5_61[4]; ldv4_diff(v.p3, v.K[4], q5_61);
    const W4<R> w62 = ffv_row(ub3, w6, q5_61, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a52 = ffv_amp(w62, w23, g1);
    jadd64_mi(jamp[2], a52);
    jadd64_pi(jamp[12], a52);
    const cx<R> a53 = ffv_amp(w62, w29, g3);
    jadd64_mi(jamp[3], a53);
    jadd64_pi(jamp[13], a53);
    const cx<R> a54 = ffv_amp(w62, v4, w15);
    jadd64_mi(jamp[2], a54);
    jadd64_pi(jamp[3], a54);
    jadd64_pi(jamp[12], a54);
    jadd64_mi(jamp[13], a54);
    R q9_63[4]; ldv4_diff(v.p3, v.K[8], q9_63);
    const W4<R> w64 = ffv_row(ub3, w9, q9_63, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a55 = ffv_amp(w64, w25, g1);
    jadd64_mi(jamp[4], a55);
    jadd64_pi(jamp[18], a55);
    const cx<R> a56 = ffv_amp(w64, w29, g2);
    jadd64_mi(jamp[5], a56);
    jadd64_pi(jamp[19], a56);
    const cx<R> a57 = ffv_amp(w64, v4, w12);
    jadd64_mi(jamp[4], a57);
    jadd64_pi(jamp[5], a57);
    jadd64_pi(jamp[18], a57);
    jadd64_mi(jamp[19], a57);
    R q6_65[4]; ldv4_diff(v.p3, v.K[5], q6_65);
    const W4<R> w66 = ffv_row(ub3, w12, q6_65, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a58 = ffv_amp(w66, w23, g0);
    jadd64_mi(jamp[8], a58);
    jadd64_pi(jamp[14], a58);
    const cx<R> a59 = ffv_amp(w66, w39, g3);
    jadd64_mi(jamp[9], a59);
    jadd64_pi(jamp[15], a59);
    const cx<R> a60 = ffv_amp(w66, v4, w9);
    jadd64_mi(jamp[8], a60);
    jadd64_pi(jamp[9], a60);
    jadd64_pi(jamp[14], a60);
    jadd64_mi(jamp[15], a60);
    R q10_67[4]; ldv4_diff(v.p3, v.K[9], q10_67);
    const W4<R> w68 = ffv_row(ub3, w15, q10_67, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a61 = ffv_amp(w68, w25, g0);
    jadd64_mi(jamp[10], a61);
    jadd64_pi(jamp[20], a61);
    const cx<R> a62 = ffv_amp(w68, w39, g2);
    jadd64_mi(jamp[11], a62);
    jadd64_pi(jamp[21], a62);
    const cx<R> a63 = ffv_amp(w68, v4, w6);
    jadd64_mi(jamp[10], a63);
    jadd64_pi(jamp[11], a63);
    jadd64_pi(jamp[20], a63);
    jadd64_mi(jamp[21], a63);
    R q12_69[4]; ldv4_diff(v.p3, v.K[11], q12_69);
    const W4<R> w70 = ffv_row(ub3, w18, q12_69, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a64 = ffv_amp(w70, w29, g0);
    jadd64_mi(jamp[16], a64);
    jadd64_pi(jamp[22], a64);
    const cx<R> a65 = ffv_amp(w70, w39, g1);
    jadd64_mi(jamp[17], a65);
    jadd64_pi(jamp[23], a65);
    const cx<R> a66 = ffv_amp(w70, v4, w3);
    jadd64_mi(jamp[16], a66);
    jadd64_pi(jamp[17], a66);
    jadd64_pi(jamp[22], a66);
    jadd64_mi(jamp[23], a66);
    const W4<R> jq = ffv_cur(ub3, v4, ldv(v.iG[10]));
    {
    R q7_72[4]; ldv4_diff(v.p3, v.K[6], q7_72);
    const W4<R> w71 = ffv_col(g3, v4, q7_72, ldv(v.mt), ldv(v.iQ[6]));
    R q8_73[4]; ldv4_diff(v.p3, v.K[7], q8_73);
    const W4<R> w74 = ffv_row(ub3, g3, q8_73, ldv(v.mt), ldv(v.iQ[7]));
    {
    R k1_75[4]; ldv4(v.K[0], k1_75);
    R k6_76[4]; ldv4(v.K[5], k6_76);
    const W4<R> w77 = vvv_cur(g0, w12, k1_75, k6_76, ldv(v.iG[3]));
    const cx<R> a67 = ffv_amp(w74, v4, w77);
    jadd64_mi(jamp[18], a67);
    jadd64_pi(jamp[19], a67);
    jadd64_pi(jamp[21], a67);
    jadd64_mi(jamp[23], a67);
    const cx<R> a68 = ffv_amp(ub3, w71, w77);
    jadd64_mi(jamp[0], a68);
    jadd64_pi(jamp[2], a68);
    jadd64_pi(jamp[8], a68);
    jadd64_mi(jamp[14], a68);
    R k7_78[4]; ldv4(v.K[6], k7_78);
    R k8_79[4]; ldv4(v.K[7], k8_79);
    R k15_80[4]; ldv4(v.K[14], k15_80);
    const R nkk15_80[4] = {-k15_80[0], -k15_80[1], -k15_80[2], -k15_80[3]};
    const cx<R> a69 = vvv_amp(w77, g3, jq, k7_78, k8_79, nkk15_80);
    jadd64_mi(jamp[0], a69);
    jadd64_pi(jamp[2], a69);
    jadd64_pi(jamp[8], a69);
    jadd64_mi(jamp[14], a69);
    jadd64_pi(jamp[18], a69);
    jadd64_mi(jamp[19], a69);
    jadd64_mi(jamp[21], a69);
    jadd64_pi(jamp[23], a69);
    }
    {
    R k3_81[4]; ldv4(v.K[2], k3_81);
    R k4_82[4]; ldv4(v.K[3], k4_82);
    const W4<R> w83 = vvv_cur(w3, g2, k3_81, k4_82, ldv(v.iG[3]));
    const cx<R> a70 = ffv_amp(w74, v4, w83);
    jadd64_mi(jamp[18], a70);
    jadd64_pi(jamp[20], a70);
    jadd64_pi(jamp[22], a70);
    jadd64_mi(jamp[23], a70);
    const cx<R> a71 = ffv_amp(ub3, w71, w83);
    jadd64_mi(jamp[0], a71);
    jadd64_pi(jamp[6], a71);
    jadd64_pi(jamp[12], a71);
    jadd64_mi(jamp[14], a71);
    R k7_84[4]; ldv4(v.K[6], k7_84);
    R k8_85[4]; ldv4(v.K[7], k8_85);
    R k15_86[4]; ldv4(v.K[14], k15_86);
    const R nkk15_86[4] = {-k15_86[0], -k15_86[1], -k15_86[2], -k15_86[3]};
    const cx<R> a72 = vvv_amp(w83, g3, jq, k7_84, k8_85, nkk15_86);
    jadd64_mi(jamp[0], a72);
    jadd64_pi(jamp[6], a72);
    jadd64_pi(jamp[12], a72);
    jadd64_mi(jamp[14], a72);
    jadd64_pi(jamp[18], a72);
    jadd64_mi(jamp[20], a72);
    jadd64_mi(jamp[22], a72);
    jadd64_pi(jamp[23], a72);
    }
    {
    R k5_87[4]; ldv4(v.K[4], k5_87);
    R k2_88[4]; ldv4(v.K[1], k2_88);
    const W4<R> w89 = vvv_cur(w6, g1, k5_87, k2_88, ldv(v.iG[3]));
    const cx<R> a73 = ffv_amp(w74, v4, w89);
    jadd64_mi(jamp[19], a73);
    jadd64_pi(jamp[20], a73);
    jadd64_mi(jamp[21], a73);
    jadd64_pi(jamp[22], a73);
    const cx<R> a74 = ffv_amp(ub3, w71, w89);
    jadd64_mi(jamp[2], a74);
    jadd64_pi(jamp[6], a74);
    jadd64_mi(jamp[8], a74);
    jadd64_pi(jamp[12], a74);
    R k7_90[4]; ldv4(v.K[6], k7_90);
    R k8_91[4]; ldv4(v.K[7], k8_91);
    R k15_92[4]; ldv4(v.K[14], k15_92);
    const R nkk15_92[4] = {-k15_92[0], -k15_92[1], -k15_92[2], -k15_92[3]};
    const cx<R> a75 = vvv_amp(w89, g3, jq, k7_90, k8_91, nkk15_92);
    jadd64_mi(jamp[2], a75);
    jadd64_pi(jamp[6], a75);
    jadd64_mi(jamp[8], a75);
    jadd64_pi(jamp[12], a75);
    jadd64_pi(jamp[19], a75);
    jadd64_mi(jamp[20], a75);
    jadd64_pi(jamp[21], a75);
    jadd64_mi(jamp[22], a75);
    }
    {
    W4<R> w93, w94, w95;
    vvvv_cur(g0, g1, g2, ldv(v.iG[3]), w93, w94, w95);
    const cx<R> a76 = ffv_amp(w74, v4, w93);
    jadd64_mi(jamp[18], a76);
    jadd64_pi(jamp[20], a76);
    jadd64_pi(jamp[22], a76);
    jadd64_mi(jamp[23], a76);
    const cx<R> a77 = ffv_amp(ub3, w71, w93);
    jadd64_mi(jamp[0], a77);
    jadd64_pi(jamp[6], a77);
    jadd64_pi(jamp[12], a77);
    jadd64_mi(jamp[14], a77);
    R k7_96[4]; ldv4(v.K[6], k7_96);
    R k8_97[4]; ldv4(v.K[7], k8_97);
    R k15_98[4]; ldv4(v.K[14], k15_98);
    const R nkk15_98[4] = {-k15_98[0], -k15_98[1], -k15_98[2], -k15_98[3]};
    const cx<R> a78 = vvv_amp(w93, g3, jq, k7_96, k8_97, nkk15_98);
    jadd64_mi(jamp[0], a78);
    jadd64_pi(jamp[6], a78);
    jadd64_pi(jamp[12], a78);
    jadd64_mi(jamp[14], a78);
    jadd64_pi(jamp[18], a78);
    jadd64_mi(jamp[20], a78);
    jadd64_mi(jamp[22], a78);
    jadd64_pi(jamp[23], a78);
    const cx<R> a79 = ffv_amp(w74, v4, w94);
    jadd64_mi(jamp[19], a79);
    jadd64_pi(jamp[20], a79);
    jadd64_mi(jamp[21], a79);
    jadd64_pi(jamp[22], a79);
    const cx<R> a80 = ffv_amp(ub3, w71, w94);
    jadd64_mi(jamp[2], a80);
    jadd64_pi(jamp[6], a80);
    jadd64_mi(jamp[8], a80);
    jadd64_pi(jamp[12], a80);
    R k7_99[4]; ldv4(v.K[6], k7_99);
    R k8_100[4]; ldv4(v.K[7], k8_100);
    R k15_101[4]; ldv4(v.K[14], k15_101);
    const R nkk15_101[4] = {-k15_101[0], -k15_101[1], -k15_101[2], -k15_101[3]};
    const cx<R> a81 = vvv_amp(w94, g3, jq, k7_99, k8_100, nkk15_101);
    jadd64_mi(jamp[2], a81);
    jadd64_pi(jamp[6], a81);
    jadd64_mi(jamp[8], a81);
    jadd64_pi(jamp[12], a81);
    jadd64_pi(jamp[19], a81);
    jadd64_mi(jamp[20], a81);
    jadd64_pi(jamp[21], a81);
    jadd64_mi(jamp[22], a81);
    const cx<R> a82 = ffv_amp(w74, v4, w95);
    jadd64_pi(jamp[18], a82);
    jadd64_mi(jamp[19], a82);
    jadd64_mi(jamp[21], a82);
    jadd64_pi(jamp[23], a82);
    const cx<R> a83 = ffv_amp(ub3, w71, w95);
    jadd64_pi(jamp[0], a83);
    jadd64_mi(jamp[2], a83);
    jadd64_mi(jamp[8], a83);
    jadd64_pi(jamp[14], a83);
    R k7_102[4]; ldv4(v.K[6], k7_102);
    R k8_103[4]; ldv4(v.K[7], k8_103);
    R k15_104[4]; ldv4(v.K[14], k15_104);
    const R nkk15_104[4] = {-k15_104[0], -k15_104[1], -k15_104[2], -k15_104[3]};
    const cx<R> a84 = vvv_amp(w95, g3, jq, k7_102, k8_103, nkk15_104);
    jadd64_pi(jamp[0], a84);
    jadd64_mi(jamp[2], a84);
    jadd64_mi(jamp[8], a84);
    jadd64_pi(jamp[14], a84);
    jadd64_mi(jamp[18], a84);
    jadd64_pi(jamp[19], a84);
    jadd64_pi(jamp[21], a84);
    jadd64_mi(jamp[23], a84);
    }
    }
    {
    R q11_106[4]; ldv4_diff(v.p3, v.K[10], q11_106);
    const W4<R> w105 = ffv_col(g2, v4, q11_106, ldv(v.mt), ldv(v.iQ[10]));
    R q4_107[4]; ldv4_diff(v.p3, v.K[3], q4_107);
    const W4<R> w108 = ffv_row(ub3, g2, q4_107, ldv(v.mt), ldv(v.iQ[3]));
    {
    R k1_109[4]; ldv4(v.K[0], k1_109);
    R k10_110[4]; ldv4(v.K[9], k10_110);
    const W4<R> w111 = vvv_cur(g0, w15, k1_109, k10_110, ldv(v.iG[6]));
    const cx<R> a85 = ffv_amp(w108, v4, w111);
    jadd64_mi(jamp[12], a85);
    jadd64_pi(jamp[13], a85);
    jadd64_pi(jamp[15], a85);
    jadd64_mi(jamp[17], a85);
    const cx<R> a86 = ffv_amp(ub3, w105, w111);
    jadd64_mi(jamp[1], a86);
    jadd64_pi(jamp[4], a86);
    jadd64_pi(jamp[10], a86);
    jadd64_mi(jamp[20], a86);
    R k11_112[4]; ldv4(v.K[10], k11_112);
    R k4_113[4]; ldv4(v.K[3], k4_113);
    R k15_114[4]; ldv4(v.K[14], k15_114);
    const R nkk15_114[4] = {-k15_114[0], -k15_114[1], -k15_114[2], -k15_114[3]};
    const cx<R> a87 = vvv_amp(w111, g2, jq, k11_112, k4_113, nkk15_114);
    jadd64_mi(jamp[1], a87);
    jadd64_pi(jamp[4], a87);
    jadd64_pi(jamp[10], a87);
    jadd64_pi(jamp[12], a87);
    jadd64_mi(jamp[13], a87);
    jadd64_mi(jamp[15], a87);
    jadd64_pi(jamp[17], a87);
    jadd64_mi(jamp[20], a87);
    }
    {
    R k3_115[4]; ldv4(v.K[2], k3_115);
    R k8_116[4]; ldv4(v.K[7], k8_116);
    const W4<R> w117 = vvv_cur(w3, g3, k3_115, k8_116, ldv(v.iG[6]));
    const cx<R> a88 = ffv_amp(w108, v4, w117);
    jadd64_mi(jamp[12], a88);
    jadd64_pi(jamp[14], a88);
    jadd64_pi(jamp[16], a88);
    jadd64_mi(jamp[17], a88);
    const cx<R> a89 = ffv_amp(ub3, w105, w117);
    jadd64_mi(jamp[1], a89);
    jadd64_pi(jamp[7], a89);
    jadd64_pi(jamp[18], a89);
    jadd64_mi(jamp[20], a89);
    R k11_118[4]; ldv4(v.K[10], k11_118);
    R k4_119[4]; ldv4(v.K[3], k4_119);
    R k15_120[4]; ldv4(v.K[14], k15_120);
    const R nkk15_120[4] = {-k15_120[0], -k15_120[1], -k15_120[2], -k15_120[3]};
    const cx<R> a90 = vvv_amp(w117, g2, jq, k11_118, k4_119, nkk15_120);
    jadd64_mi(jamp[1], a90);
    jadd64_pi(jamp[7], a90);
    jadd64_pi(jamp[12], a90);
    jadd64_mi(jamp[14], a90);
    jadd64_mi(jamp[16], a90);
    jadd64_pi(jamp[17], a90);
    jadd64_pi(jamp[18], a90);
    jadd64_mi(jamp[20], a90);
    }
    {
    R k9_121[4]; ldv4(v.K[8], k9_121);
    R k2_122[4]; ldv4(v.K[1], k2_122);
    const W4<R> w123 = vvv_cur(w9, g1, k9_121, k2_122, ldv(v.iG[6]));
    const cx<R> a91 = ffv_amp(w108, v4, w123);
    jadd64_mi(jamp[13], a91);
    jadd64_pi(jamp[14], a91);
    jadd64_mi(jamp[15], a91);
    jadd64_pi(jamp[16], a91);
    const cx<R> a92 = ffv_amp(ub3, w105, w123);
    jadd64_mi(jamp[4], a92);
    jadd64_pi(jamp[7], a92);
    jadd64_mi(jamp[10], a92);
    jadd64_pi(jamp[18], a92);
    R k11_124[4]; ldv4(v.K[10], k11_124);
    R k4_125[4]; ldv4(v.K[3], k4_125);
    R k15_126[4]; ldv4(v.K[14], k15_126);
    const R nkk15_126[4] = {-k15_126[0], -k15_126[1], -k15_126[2], -k15_126[3]};
    const cx<R> a93 = vvv_amp(w123, g2, jq, k11_124, k4_125, nkk15_126);
    jadd64_mi(jamp[4], a93);
    jadd64_pi(jamp[7], a93);
    jadd64_mi(jamp[10], a93);
    jadd64_pi(jamp[13], a93);
    jadd64_mi(jamp[14], a93);
    jadd64_pi(jamp[15], a93);
    jadd64_mi(jamp[16], a93);
    jadd64_pi(jamp[18], a93);
    }
    {
    W4<R> w127, w128, w129;
    vvvv_cur(g0, g1, g3, ldv(v.iG[6]), w127, w128, w129);
    const cx<R> a94 = ffv_amp(w108, v4, w127);
    jadd64_mi(jamp[12], a94);
    jadd64_pi(jamp[14], a94);
    jadd64_pi(jamp[16], a94);
    jadd64_mi(jamp[17], a94);
    const cx<R> a95 = ffv_amp(ub3, w105, w127);
    jadd64_mi(jamp[1], a95);
    jadd64_pi(jamp[7], a95);
    jadd64_pi(jamp[18], a95);
    jadd64_mi(jamp[20], a95);
    R k11_130[4]; ldv4(v.K[10], k11_130);
    R k4_131[4]; ldv4(v.K[3], k4_131);
    R k15_132[4]; ldv4(v.K[14], k15_132);
    const R nkk15_132[4] = {-k15_132[0], -k15_132[1], -k15_132[2], -k15_132[3]};
    const cx<R> a96 = vvv_amp(w127, g2, jq, k11_130, k4_131, nkk15_132);
    jadd64_mi(jamp[1], a96);
    jadd64_pi(jamp[7], a96);
    jadd64_pi(jamp[12], a96);
    jadd64_mi(jamp[14], a96);
    jadd64_mi(jamp[16], a96);
    jadd64_pi(jamp[17], a96);
    jadd64_pi(jamp[18], a96);
    jadd64_mi(jamp[20], a96);
    const cx<R> a97 = ffv_amp(w108, v4, w128);
    jadd64_mi(jamp[13], a97);
    jadd64_pi(jamp[14], a97);
    jadd64_mi(jamp[15], a97);
    jadd64_pi(jamp[16], a97);
    const cx<R> a98 = ffv_amp(ub3, w105, w128);
    jadd64_mi(jamp[4], a98);
    jadd64_pi(jamp[7], a98);
    jadd64_mi(jamp[10], a98);
    jadd64_pi(jamp[18], a98);
    R k11_133[4]; ldv4(v.K[10], k11_133);
    R k4_134[4]; ldv4(v.K[3], k4_134);
    R k15_135[4]; ldv4(v.K[14], k15_135);
    const R nkk15_135[4] = {-k15_135[0], -k15_135[1], -k15_135[2], -k15_135[3]};
    const cx<R> a99 = vvv_amp(w128, g2, jq, k11_133, k4_134, nkk15_135);
    jadd64_mi(jamp[4], a99);
    jadd64_pi(jamp[7], a99);
    jadd64_mi(jamp[10], a99);
    jadd64_pi(jamp[13], a99);
    jadd64_mi(jamp[14], a99);
    jadd64_pi(jamp[15], a99);
    jadd64_mi(jamp[16], a99);
    jadd64_pi(jamp[18], a99);
    const cx<R> a100 = ffv_amp(w108, v4, w129);
    jadd64_pi(jamp[12], a100);
    jadd64_mi(jamp[13], a100);
    jadd64_mi(jamp[15], a100);
    jadd64_pi(jamp[17], a100);
    const cx<R> a101 = ffv_amp(ub3, w105, w129);
    jadd64_pi(jamp[1], a101);
    jadd64_mi(jamp[4], a101);
    jadd64_mi(jamp[10], a101);
    jadd64_pi(jamp[20], a101);
    R k11_136[4]; ldv4(v.K[10], k11_136);
    R k4_137[4]; ldv4(v.K[3], k4_137);
    R k15_138[4]; ldv4(v.K[14], k15_138);
    const R nkk15_138[4] = {-k15_138[0], -k15_138[1], -k15_138[2], -k15_138[3]};
    const cx<R> a102 = vvv_amp(w129, g2, jq, k11_136, k4_137, nkk15_138);
    jadd64_pi(jamp[1], a102);
    jadd64_mi(jamp[4], a102);
    jadd64_mi(jamp[10], a102);
    jadd64_mi(jamp[12], a102);
    jadd64_pi(jamp[13], a102);
    jadd64_pi(jamp[15], a102);
    jadd64_mi(jamp[17], a102);
    jadd64_pi(jamp[20], a102);
    }
    }
    {
    R q13_140[4]; ldv4_diff(v.p3, v.K[12], q13_140);
    const W4<R> w139 = ffv_col(g1, v4, q13_140, ldv(v.mt), ldv(v.iQ[12]));
    R q2_141[4]; ldv4_diff(v.p3, v.K[1], q2_141);
    const W4<R> w142 = ffv_row(ub3, g1, q2_141, ldv(v.mt), ldv(v.iQ[1]));
    {
    R k1_143[4]; ldv4(v.K[0], k1_143);
    R k12_144[4]; ldv4(v.K[11], k12_144);
    const W4<R> w145 = vvv_cur(g0, w18, k1_143, k12_144, ldv(v.iG[8]));
    const cx<R> a103 = ffv_amp(w142, v4, w145);
    jadd64_mi(jamp[6], a103);
    jadd64_pi(jamp[7], a103);
    jadd64_pi(jamp[9], a103);
    jadd64_mi(jamp[11], a103);
    const cx<R> a104 = ffv_amp(ub3, w139, w145);
    jadd64_mi(jamp[3], a104);
    jadd64_pi(jamp[5], a104);
    jadd64_pi(jamp[16], a104);
    jadd64_mi(jamp[22], a104);
    R k13_146[4]; ldv4(v.K[12], k13_146);
    R k2_147[4]; ldv4(v.K[1], k2_147);
    R k15_148[4]; ldv4(v.K[14], k15_148);
    const R nkk15_148[4] = {-k15_148[0], -k15_148[1], -k15_148[2], -k15_148[3]};
    const cx<R> a105 = vvv_amp(w145, g1, jq, k13_146, k2_147, nkk15_148);
    jadd64_mi(jamp[3], a105);
    jadd64_pi(jamp[5], a105);
    jadd64_pi(jamp[6], a105);
    jadd64_mi(jamp[7], a105);
    jadd64_mi(jamp[9], a105);
    jadd64_pi(jamp[11], a105);
    jadd64_pi(jamp[16], a105);
    jadd64_mi(jamp[22], a105);
    }
    {
    R k5_149[4]; ldv4(v.K[4], k5_149);
    R k8_150[4]; ldv4(v.K[7], k8_150);
    const W4<R> w151 = vvv_cur(w6, g3, k5_149, k8_150, ldv(v.iG[8]));
    const cx<R> a106 = ffv_amp(w142, v4, w151);
    jadd64_mi(jamp[6], a106);
    jadd64_pi(jamp[8], a106);
    jadd64_pi(jamp[10], a106);
    jadd64_mi(jamp[11], a106);
    const cx<R> a107 = ffv_amp(ub3, w139, w151);
    jadd64_mi(jamp[3], a107);
    jadd64_pi(jamp[13], a107);
    jadd64_pi(jamp[19], a107);
    jadd64_mi(jamp[22], a107);
    R k13_152[4]; ldv4(v.K[12], k13_152);
    R k2_153[4]; ldv4(v.K[1], k2_153);
    R k15_154[4]; ldv4(v.K[14], k15_154);
    const R nkk15_154[4] = {-k15_154[0], -k15_154[1], -k15_154[2], -k15_154[3]};
    const cx<R> a108 = vvv_amp(w151, g1, jq, k13_152, k2_153, nkk15_154);
    jadd64_mi(jamp[3], a108);
    jadd64_pi(jamp[6], a108);
    jadd64_mi(jamp[8], a108);
    jadd64_mi(jamp[10], a108);
    jadd64_pi(jamp[11], a108);
    jadd64_pi(jamp[13], a108);
    jadd64_pi(jamp[19], a108);
    jadd64_mi(jamp[22], a108);
    }
    {
    R k9_155[4]; ldv4(v.K[8], k9_155);
    R k4_156[4]; ldv4(v.K[3], k4_156);
    const W4<R> w157 = vvv_cur(w9, g2, k9_155, k4_156, ldv(v.iG[8]));
    const cx<R> a109 = ffv_amp(w142, v4, w157);
    jadd64_mi(jamp[7], a109);
    jadd64_pi(jamp[8], a109);
    jadd64_mi(jamp[9], a109);
    jadd64_pi(jamp[10], a109);
    const cx<R> a110 = ffv_amp(ub3, w139, w157);
    jadd64_mi(jamp[5], a110);
    jadd64_pi(jamp[13], a110);
    jadd64_mi(jamp[16], a110);
    jadd64_pi(jamp[19], a110);
    R k13_158[4]; ldv4(v.K[12], k13_158);
    R k2_159[4]; ldv4(v.K[1], k2_159);
    R k15_160[4]; ldv4(v.K[14], k15_160);
    const R nkk15_160[4] = {-k15_160[0], -k15_160[1], -k15_160[2], -k15_160[3]};
    const cx<R> a111 = vvv_amp(w157, g1, jq, k13_158, k2_159, nkk15_160);
    jadd64_mi(jamp[5], a111);
    jadd64_pi(jamp[7], a111);
    jadd64_mi(jamp[8], a111);
    jadd64_pi(jamp[9], a111);
    jadd64_mi(jamp[10], a111);
    jadd64_pi(jamp[13], a111);
    jadd64_mi(jamp[16], a111);
    jadd64_pi(jamp[19], a111);
    }
    {
    W4<R> w161, w162, w163;
    vvvv_cur(g0, g2, g3, ldv(v.iG[8]), w161, w162, w163);
    const cx<R> a112 = ffv_amp(w142, v4, w161);
    jadd64_mi(jamp[6], a112);
    jadd64_pi(jamp[8], a112);
    jadd64_pi(jamp[10], a112);
    jadd64_mi(jamp[11], a112);
    const cx<R> a113 = ffv_amp(ub3, w139, w161);
    jadd64_mi(jamp[3], a113);
    jadd64_pi(jamp[13], a113);
    jadd64_pi(jamp[19], a113);
    jadd64_mi(jamp[22], a113);
    R k13_164[4]; ldv4(v.K[12], k13_164);
    R k2_165[4]; ldv4(v.K[1], k2_165);
    R k15_166[4]; ldv4(v.K[14], k15_166);
    const R nkk15_166[4] = {-k15_166[0], -k15_166[1], -k15_166[2], -k15_166[3]};
    const cx<R> a114 = vvv_amp(w161, g1, jq, k13_164, k2_165, nkk15_166);
    jadd64_mi(jamp[3], a114);
    jadd64_pi(jamp[6], a114);
    jadd64_mi(jamp[8], a114);
    jadd64_mi(jamp[10], a114);
    jadd64_pi(jamp[11], a114);
    jadd64_pi(jamp[13], a114);
    jadd64_pi(jamp[19], a114);
    jadd64_mi(jamp[22], a114);
    const cx<R> a115 = ffv_amp(w142, v4, w162);
    jadd64_mi(jamp[7], a115);
    jadd64_pi(jamp[8], a115);
    jadd64_mi(jamp[9], a115);
    jadd64_pi(jamp[10], a115);
    const cx<R> a116 = ffv_amp(ub3, w139, w162);
    jadd64_mi(jamp[5], a116);
    jadd64_pi(jamp[13], a116);
    jadd64_mi(jamp[16], a116);
    jadd64_pi(jamp[19], a116);
    R k13_167[4]; ldv4(v.K[12], k13_167);
    R k2_168[4]; ldv4(v.K[1], k2_168);
    R k15_169[4]; ldv4(v.K[14], k15_169);
    const R nkk15_169[4] = {-k15_169[0], -k15_169[1], -k15_169[2], -k15_169[3]};
    const cx<R> a117 = vvv_amp(w162, g1, jq, k13_167, k2_168, nkk15_169);
    jadd64_mi(jamp[5], a117);
    jadd64_pi(jamp[7], a117);
    jadd64_mi(jamp[8], a117);
    jadd64_pi(jamp[9], a117);
    jadd64_mi(jamp[10], a117);
    jadd64_pi(jamp[13], a117);
    jadd64_mi(jamp[16], a117);
    jadd64_pi(jamp[19], a117);
    const cx<R> a118 = ffv_amp(w142, v4, w163);
    jadd64_pi(jamp[6], a118);
    jadd64_mi(jamp[7], a118);
    jadd64_mi(jamp[9], a118);
    jadd64_pi(jamp[11], a118);
    const cx<R> a119 = ffv_amp(ub3, w139, w163);
    jadd64_pi(jamp[3], a119);
    jadd64_mi(jamp[5], a119);
    jadd64_mi(jamp[16], a119);
    jadd64_pi(jamp[22], a119);
    R k13_170[4]; ldv4(v.K[12], k13_170);
    R k2_171[4]; ldv4(v.K[1], k2_171);
    R k15_172[4]; ldv4(v.K[14], k15_172);
    const R nkk15_172[4] = {-k15_172[0], -k15_172[1], -k15_172[2], -k15_172[3]};
    const cx<R> a120 = vvv_amp(w163, g1, jq, k13_170, k2_171, nkk15_172);
    jadd64_pi(jamp[3], a120);
    jadd64_mi(jamp[5], a120);
    jadd64_mi(jamp[6], a120);
    jadd64_pi(jamp[7], a120);
    jadd64_pi(jamp[9], a120);
    jadd64_mi(jamp[11], a120);
    jadd64_mi(jamp[16], a120);
    jadd64_pi(jamp[22], a120);
    }
    }
    {
    R q14_174[4]; ldv4_diff(v.p3, v.K[13], q14_174);
    const W4<R> w173 = ffv_col(g0, v4, q14_174, ldv(v.mt), ldv(v.iQ[13]));
    R q1_175[4]; ldv4_diff(v.p3, v.K[0], q1_175);
    const W4<R> w176 = ffv_row(ub3, g0, q1_175, ldv(v.mt), ldv(v.iQ[0]));
    {
    R k2_177[4]; ldv4(v.K[1], k2_177);
    R k12_178[4]; ldv4(v.K[11], k12_178);
    const W4<R> w179 = vvv_cur(g1, w18, k2_177, k12_178, ldv(v.iG[9]));
    const cx<R> a121 = ffv_amp(w176, v4, w179);
    jadd64_mi(jamp[0], a121);
    jadd64_pi(jamp[1], a121);
    jadd64_pi(jamp[3], a121);
    jadd64_mi(jamp[5], a121);
    const cx<R> a122 = ffv_amp(ub3, w173, w179);
    jadd64_mi(jamp[9], a122);
    jadd64_pi(jamp[11], a122);
    jadd64_pi(jamp[17], a122);
    jadd64_mi(jamp[23], a122);
    R k1_180[4]; ldv4(v.K[0], k1_180);
    R k14_181[4]; ldv4(v.K[13], k14_181);
    R k15_182[4]; ldv4(v.K[14], k15_182);
    const R nkk15_182[4] = {-k15_182[0], -k15_182[1], -k15_182[2], -k15_182[3]};
    const cx<R> a123 = vvv_amp(g0, w179, jq, k1_180, k14_181, nkk15_182);
    jadd64_mi(jamp[0], a123);
    jadd64_pi(jamp[1], a123);
    jadd64_pi(jamp[3], a123);
    jadd64_mi(jamp[5], a123);
    jadd64_pi(jamp[9], a123);
    jadd64_mi(jamp[11], a123);
    jadd64_mi(jamp[17], a123);
    jadd64_pi(jamp[23], a123);
    }
    {
    R k6_183[4]; ldv4(v.K[5], k6_183);
    R k8_184[4]; ldv4(v.K[7], k8_184);
    const W4<R> w185 = vvv_cur(w12, g3, k6_183, k8_184, ldv(v.iG[9]));
    const cx<R> a124 = ffv_amp(w176, v4, w185);
    jadd64_mi(jamp[0], a124);
    jadd64_pi(jamp[2], a124);
    jadd64_pi(jamp[4], a124);
    jadd64_mi(jamp[5], a124);
    const cx<R> a125 = ffv_amp(ub3, w173, w185);
    jadd64_mi(jamp[9], a125);
    jadd64_pi(jamp[15], a125);
    jadd64_pi(jamp[21], a125);
    jadd64_mi(jamp[23], a125);
    R k1_186[4]; ldv4(v.K[0], k1_186);
    R k14_187[4]; ldv4(v.K[13], k14_187);
    R k15_188[4]; ldv4(v.K[14], k15_188);
    const R nkk15_188[4] = {-k15_188[0], -k15_188[1], -k15_188[2], -k15_188[3]};
    const cx<R> a126 = vvv_amp(g0, w185, jq, k1_186, k14_187, nkk15_188);
    jadd64_mi(jamp[0], a126);
    jadd64_pi(jamp[2], a126);
    jadd64_pi(jamp[4], a126);
    jadd64_mi(jamp[5], a126);
    jadd64_pi(jamp[9], a126);
    jadd64_mi(jamp[15], a126);
    jadd64_mi(jamp[21], a126);
    jadd64_pi(jamp[23], a126);
    }
    {
    R k10_189[4]; ldv4(v.K[9], k10_189);
    R k4_190[4]; ldv4(v.K[3], k4_190);
    const W4<R> w191 = vvv_cur(w15, g2, k10_189, k4_190, ldv(v.iG[9]));
    const cx<R> a127 = ffv_amp(w176, v4, w191);
    jadd64_mi(jamp[1], a127);
    jadd64_pi(jamp[2], a127);
    jadd64_mi(jamp[3], a127);
    jadd64_pi(jamp[4], a127);
    const cx<R> a128 = ffv_amp(ub3, w173, w191);
    jadd64_mi(jamp[11], a128);
    jadd64_pi(jamp[15], a128);
    jadd64_mi(jamp[17], a128);
    jadd64_pi(jamp[21], a128);
    R k1_192[4]; ldv4(v.K[0], k1_192);
    R k14_193[4]; ldv4(v.K[13], k14_193);
    R k15_194[4]; ldv4(v.K[14], k15_194);
    const R nkk15_194[4] = {-k15_194[0], -k15_194[1], -k15_194[2], -k15_194[3]};
    const cx<R> a129 = vvv_amp(g0, w191, jq, k1_192, k14_193, nkk15_194);
    jadd64_mi(jamp[1], a129);
    jadd64_pi(jamp[2], a129);
    jadd64_mi(jamp[3], a129);
    jadd64_pi(jamp[4], a129);
    jadd64_pi(jamp[11], a129);
    jadd64_mi(jamp[15], a129);
    jadd64_pi(jamp[17], a129);
    jadd64_mi(jamp[21], a129);
    }
    {
    W4<R> w195, w196, w197;
    vvvv_cur(g1, g2, g3, ldv(v.iG[9]), w195, w196, w197);
    const cx<R> a130 = ffv_amp(w176, v4, w195);
    jadd64_mi(jamp[0], a130);
    jadd64_pi(jamp[2], a130);
    jadd64_pi(jamp[4], a130);
    jadd64_mi(jamp[5], a130);
    const cx<R> a131 = ffv_amp(ub3, w173, w195);
    jadd64_mi(jamp[9], a131);
    jadd64_pi(jamp[15], a131);
    jadd64_pi(jamp[21], a131);
    jadd64_mi(jamp[23], a131);
    R k1_198[4]; ldv4(v.K[0], k1_198);
    R k14_199[4]; ldv4(v.K[13], k14_199);
    R k15_200[4]; ldv4(v.K[14], k15_200);
    const R nkk15_200[4] = {-k15_200[0], -k15_200[1], -k15_200[2], -k15_200[3]};
    const cx<R> a132 = vvv_amp(g0, w195, jq, k1_198, k14_199, nkk15_200);
    jadd64_mi(jamp[0], a132);
    jadd64_pi(jamp[2], a132);
    jadd64_pi(jamp[4], a132);
    jadd64_mi(jamp[5], a132);
    jadd64_pi(jamp[9], a132);
    jadd64_mi(jamp[15], a132);
    jadd64_mi(jamp[21], a132);
    jadd64_pi(jamp[23], a132);
    const cx<R> a133 = ffv_amp(w176, v4, w196);
    jadd64_mi(jamp[1], a133);
    jadd64_pi(jamp[2], a133);
    jadd64_mi(jamp[3], a133);
    jadd64_pi(jamp[4], a133);
    const cx<R> a134 = ffv_amp(ub3, w173, w196);
    jadd64_mi(jamp[11], a134);
    jadd64_pi(jamp[15], a134);
    jadd64_mi(jamp[17], a134);
    jadd64_pi(jamp[21], a134);
    R k1_201[4]; ldv4(v.K[0], k1_201);
    R k14_202[4]; ldv4(v.K[13], k14_202);
    R k15_203[4]; ldv4(v.K[14], k15_203);
    const R nkk15_203[4] = {-k15_203[0], -k15_203[1], -k15_203[2], -k15_203[3]};
    const cx<R> a135 = vvv_amp(g0, w196, jq, k1_201, k14_202, nkk15_203);
    jadd64_mi(jamp[1], a135);
    jadd64_pi(jamp[2], a135);
    jadd64_mi(jamp[3], a135);
    jadd64_pi(jamp[4], a135);
    jadd64_pi(jamp[11], a135);
    jadd64_mi(jamp[15], a135);
    jadd64_pi(jamp[17], a135);
    jadd64_mi(jamp[21], a135);
    const cx<R> a136 = ffv_amp(w176, v4, w197);
    jadd64_pi(jamp[0], a136);
    jadd64_mi(jamp[1], a136);
    jadd64_mi(jamp[3], a136);
    jadd64_pi(jamp[5], a136);
    const cx<R> a137 = ffv_amp(ub3, w173, w197);
    jadd64_pi(jamp[9], a137);
    jadd64_mi(jamp[11], a137);
    jadd64_mi(jamp[17], a137);
    jadd64_pi(jamp[23], a137);
    R k1_204[4]; ldv4(v.K[0], k1_204);
    R k14_205[4]; ldv4(v.K[13], k14_205);
    R k15_206[4]; ldv4(v.K[14], k15_206);
    const R nkk15_206[4] = {-k15_206[0], -k15_206[1], -k15_206[2], -k15_206[3]};
    const cx<R> a138 = vvv_amp(g0, w197, jq, k1_204, k14_205, nkk15_206);
    jadd64_pi(jamp[0], a138);
    jadd64_mi(jamp[1], a138);
    jadd64_mi(jamp[3], a138);
    jadd64_pi(jamp[5], a138);
    jadd64_mi(jamp[9], a138);
    jadd64_pi(jamp[11], a138);
    jadd64_pi(jamp[17], a138);
    jadd64_mi(jamp[23], a138);
    }
    }
    R k3_207[4]; ldv4(v.K[2], k3_207);
    R k12_208[4]; ldv4(v.K[11], k12_208);
    R k15_209[4]; ldv4(v.K[14], k15_209);
    const R nkk15_209[4] = {-k15_209[0], -k15_209[1], -k15_209[2], -k15_209[3]};
    const cx<R> a139 = vvv_amp(w3, w18, jq, k3_207, k12_208, nkk15_209);
    jadd64_mi(jamp[0], a139);
    jadd64_pi(jamp[1], a139);
    jadd64_pi(jamp[6], a139);
    jadd64_mi(jamp[7], a139);
    jadd64_pi(jamp[16], a139);
    jadd64_mi(jamp[17], a139);
    jadd64_mi(jamp[22], a139);
    jadd64_pi(jamp[23], a139);
    R k5_210[4]; ldv4(v.K[4], k5_210);
    R k10_211[4]; ldv4(v.K[9], k10_211);
    R k15_212[4]; ldv4(v.K[14], k15_212);
    const R nkk15_212[4] = {-k15_212[0], -k15_212[1], -k15_212[2], -k15_212[3]};
    const cx<R> a140 = vvv_amp(w6, w15, jq, k5_210, k10_211, nkk15_212);
    jadd64_mi(jamp[2], a140);
    jadd64_pi(jamp[3], a140);
    jadd64_pi(jamp[10], a140);
    jadd64_mi(jamp[11], a140);
    jadd64_pi(jamp[12], a140);
    jadd64_mi(jamp[13], a140);
    jadd64_mi(jamp[20], a140);
    jadd64_pi(jamp[21], a140);
    R k9_213[4]; ldv4(v.K[8], k9_213);
    R k6_214[4]; ldv4(v.K[5], k6_214);
    R k15_215[4]; ldv4(v.K[14], k15_215);
    const R nkk15_215[4] = {-k15_215[0], -k15_215[1], -k15_215[2], -k15_215[3]};
    const cx<R> a141 = vvv_amp(w9, w12, jq, k9_213, k6_214, nkk15_215);
    jadd64_mi(jamp[4], a141);
    jadd64_pi(jamp[5], a141);
    jadd64_pi(jamp[8], a141);
    jadd64_mi(jamp[9], a141);
    jadd64_mi(jamp[14], a141);
    jadd64_pi(jamp[15], a141);
    jadd64_pi(jamp[18], a141);
    jadd64_mi(jamp[19], a141);
    cx<R> a142, a143, a144;
    vvvv_amp(g0, g1, w18, jq, a142, a143, a144);
    jadd64_mi(jamp[0], a142);
    jadd64_pi(jamp[1], a142);
    jadd64_pi(jamp[6], a142);
    jadd64_mi(jamp[7], a142);
    jadd64_pi(jamp[16], a142);
    jadd64_mi(jamp[17], a142);
    jadd64_mi(jamp[22], a142);
    jadd64_pi(jamp[23], a142);
    jadd64_mi(jamp[3], a143);
    jadd64_pi(jamp[5], a143);
    jadd64_pi(jamp[6], a143);
    jadd64_mi(jamp[7], a143);
    jadd64_mi(jamp[9], a143);
    jadd64_pi(jamp[11], a143);
    jadd64_pi(jamp[16], a143);
    jadd64_mi(jamp[22], a143);
    jadd64_pi(jamp[0], a144);
    jadd64_mi(jamp[1], a144);
    jadd64_mi(jamp[3], a144);
    jadd64_pi(jamp[5], a144);
    jadd64_mi(jamp[9], a144);
    jadd64_pi(jamp[11], a144);
    jadd64_pi(jamp[17], a144);
    jadd64_mi(jamp[23], a144);
    cx<R> a145, a146, a147;
    vvvv_amp(g0, w12, g3, jq, a145, a146, a147);
    jadd64_mi(jamp[0], a145);
    jadd64_pi(jamp[2], a145);
    jadd64_pi(jamp[8], a145);
    jadd64_mi(jamp[14], a145);
    jadd64_pi(jamp[18], a145);
    jadd64_mi(jamp[19], a145);
    jadd64_mi(jamp[21], a145);
    jadd64_pi(jamp[23], a145);
    jadd64_mi(jamp[4], a146);
    jadd64_pi(jamp[5], a146);
    jadd64_pi(jamp[8], a146);
    jadd64_mi(jamp[9], a146);
    jadd64_mi(jamp[14], a146);
    jadd64_pi(jamp[15], a146);
    jadd64_pi(jamp[18], a146);
    jadd64_mi(jamp[19], a146);
    jadd64_pi(jamp[0], a147);
    jadd64_mi(jamp[2], a147);
    jadd64_mi(jamp[4], a147);
    jadd64_pi(jamp[5], a147);
    jadd64_mi(jamp[9], a147);
    jadd64_pi(jamp[15], a147);
    jadd64_pi(jamp[21], a147);
    jadd64_mi(jamp[23], a147);
    cx<R> a148, a149, a150;
    vvvv_amp(g0, w15, g2, jq, a148, a149, a150);
    jadd64_mi(jamp[1], a148);
    jadd64_pi(jamp[4], a148);
    jadd64_pi(jamp[10], a148);
    jadd64_pi(jamp[12], a148);
    jadd64_mi(jamp[13], a148);
    jadd64_mi(jamp[15], a148);
    jadd64_pi(jamp[17], a148);
    jadd64_mi(jamp[20], a148);
    jadd64_mi(jamp[2], a149);
    jadd64_pi(jamp[3], a149);
    jadd64_pi(jamp[10], a149);
    jadd64_mi(jamp[11], a149);
    jadd64_pi(jamp[12], a149);
    jadd64_mi(jamp[13], a149);
    jadd64_mi(jamp[20], a149);
    jadd64_pi(jamp[21], a149);
    jadd64_pi(jamp[1], a150);
    jadd64_mi(jamp[2], a150);
    jadd64_pi(jamp[3], a150);
    jadd64_mi(jamp[4], a150);
    jadd64_mi(jamp[11], a150);
    jadd64_pi(jamp[15], a150);
    jadd64_mi(jamp[17], a150);
    jadd64_pi(jamp[21], a150);
    cx<R> a151, a152, a153;
    vvvv_amp(w3, g2, g3, jq, a151, a152, a153);
    jadd64_mi(jamp[0], a151);
    jadd64_pi(jamp[6], a151);
    jadd64_pi(jamp[12], a151);
    jadd64_mi(jamp[14], a151);
    jadd64_pi(jamp[18], a151);
    jadd64_mi(jamp[20], a151);
    jadd64_mi(jamp[22], a151);
    jadd64_pi(jamp[23], a151);
    jadd64_mi(jamp[1], a152);
    jadd64_pi(jamp[7], a152);
    jadd64_pi(jamp[12], a152);
    jadd64_mi(jamp[14], a152);
    jadd64_mi(jamp[16], a152);
    jadd64_pi(jamp[17], a152);
    jadd64_pi(jamp[18], a152);
    jadd64_mi(jamp[20], a152);
    jadd64_pi(jamp[0], a153);
    jadd64_mi(jamp[1], a153);
    jadd64_mi(jamp[6], a153);
    jadd64_pi(jamp[7], a153);
    jadd64_mi(jamp[16], a153);
    jadd64_pi(jamp[17], a153);
    jadd64_pi(jamp[22], a153);
    jadd64_mi(jamp[23], a153);
    cx<R> a154, a155, a156;
    vvvv_amp(w6, g1, g3, jq, a154, a155, a156);
    jadd64_mi(jamp[2], a154);
    jadd64_pi(jamp[6], a154);
    jadd64_mi(jamp[8], a154);
    jadd64_pi(jamp[12], a154);
    jadd64_pi(jamp[19], a154);
    jadd64_mi(jamp[20], a154);
    jadd64_pi(jamp[21], a154);
    jadd64_mi(jamp[22], a154);
    jadd64_mi(jamp[3], a155);
    jadd64_pi(jamp[6], a155);
    jadd64_mi(jamp[8], a155);
    jadd64_mi(jamp[10], a155);
    jadd64_pi(jamp[11], a155);
    jadd64_pi(jamp[13], a155);
    jadd64_pi(jamp[19], a155);
    jadd64_mi(jamp[22], a155);
    jadd64_pi(jamp[2], a156);
    jadd64_mi(jamp[3], a156);
    jadd64_mi(jamp[10], a156);
    jadd64_pi(jamp[11], a156);
    jadd64_mi(jamp[12], a156);
    jadd64_pi(jamp[13], a156);
    jadd64_pi(jamp[20], a156);
    jadd64_mi(jamp[21], a156);
    cx<R> a157, a158, a159;
    vvvv_amp(w9, g1, g2, jq, a157, a158, a159);
    jadd64_mi(jamp[4], a157);
    jadd64_pi(jamp[7], a157);
    jadd64_mi(jamp[10], a157);
    jadd64_pi(jamp[13], a157);
    jadd64_mi(jamp[14], a157);
    jadd64_pi(jamp[15], a157);
    jadd64_mi(jamp[16], a157);
    jadd64_pi(jamp[18], a157);
    jadd64_mi(jamp[5], a158);
    jadd64_pi(jamp[7], a158);
    jadd64_mi(jamp[8], a158);
    jadd64_pi(jamp[9], a158);
    jadd64_mi(jamp[10], a158);
    jadd64_pi(jamp[13], a158);
    jadd64_mi(jamp[16], a158);
    jadd64_pi(jamp[19], a158);
    jadd64_pi(jamp[4], a159);
    jadd64_mi(jamp[5], a159);
    jadd64_mi(jamp[8], a159);
    jadd64_pi(jamp[9], a159);
    jadd64_pi(jamp[14], a159);
    jadd64_mi(jamp[15], a159);
    jadd64_mi(jamp[18], a159);
    jadd64_pi(jamp[19], a159);
#undef HEL
}

template <typename R>
__device__ void Me_gg_ttgg::inv(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt, Inv<R>& v)
{
    inv_gg_ttgg<R>(&p[0][0], mt, v);
}
template <typename R, int JROW, int REC_OFF, int REC_STRIDE>
__device__ void Me_gg_ttgg::hel_j(int ih)
{
    hel_gg_ttgg_j<R, JROW, REC_OFF, REC_STRIDE>(ih);
}
}  // namespace mf

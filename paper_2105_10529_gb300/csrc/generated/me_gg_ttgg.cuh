// Generated by paper_2105_10529_gb300/gen/qcd_diagrams.py -- do not edit.
// gg_ttgg: 123 Feynman diagrams (159 amplitudes with the four-gluon
// colour structures counted apart), 24 colour flows, 64 helicities.
// Wavefunction/vertex calls per helicity: {'vvv': 18, 'vvvv': 4, 'ffv_row': 26, 'ffv_col': 8, 'ffv_amp': 114, 'vvv_amp': 27, 'vvvv_amp': 6, 'ffv_cur': 1}
#pragma once
#include "mf_helas.cuh"
namespace mf {
struct Me_gg_ttgg {
  static constexpr int NEXT = 6;
  static constexpr int NCOL = 24;
  static constexpr int NHEL = 64;
  static constexpr int NGLUON = 4;
  static constexpr int NDIAG = 123;
  static constexpr double COLOUR_DEN = 54.0;
  static constexpr double AVG = 1.0 / 256.0;
  static constexpr double SYM = 0.5;
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
  template <typename R, bool SYNC = false>
  __device__ static double me2(const double (&p)[NEXT][4], double mt, double gs, void* slot);
  template <typename R> static constexpr size_t slot_bytes() { return sizeof(Inv<R>); }
};

// one helicity configuration: amplitudes, colour flows and the colour sum;
// out of line so that its register allocation sees only one helicity
template <typename R>
__device__ __noinline__ R hel_gg_ttgg(const Me_gg_ttgg::Inv<R>& v, int ih)
{
    constexpr int NCOL = Me_gg_ttgg::NCOL;
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
    // colour-flow amplitudes accumulate in the slot (shared memory), not in registers
    volatile cx<R>* jamp = reinterpret_cast<volatile cx<R>*>(const_cast<cx<R>*>(v.jamp));
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) { jamp[c].r = R(0); jamp[c].i = R(0); }
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
    jamp[0].r += a1.i; jamp[0].i -= a1.r;
    const R q11_26[4] = {ldv(v.p3[0]) - ldv(v.K[10][0]), ldv(v.p3[1]) - ldv(v.K[10][1]), ldv(v.p3[2]) - ldv(v.K[10][2]), ldv(v.p3[3]) - ldv(v.K[10][3])};
    const W4<R> w25 = ffv_col(g2, v4, q11_26, ldv(v.mt), ldv(v.iQ[10]));
    const cx<R> a2 = ffv_amp(w22, w25, g3);
    jamp[1].r += a2.i; jamp[1].i -= a2.r;
    const cx<R> a3 = ffv_amp(w22, v4, w18);
    jamp[0].r += a3.i; jamp[0].i -= a3.r;
    jamp[1].r -= a3.i; jamp[1].i += a3.r;
    const R q5_27[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w28 = ffv_row(w20, g2, q5_27, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a4 = ffv_amp(w28, w23, g1);
    jamp[2].r += a4.i; jamp[2].i -= a4.r;
    const R q13_30[4] = {ldv(v.p3[0]) - ldv(v.K[12][0]), ldv(v.p3[1]) - ldv(v.K[12][1]), ldv(v.p3[2]) - ldv(v.K[12][2]), ldv(v.p3[3]) - ldv(v.K[12][3])};
    const W4<R> w29 = ffv_col(g1, v4, q13_30, ldv(v.mt), ldv(v.iQ[12]));
    const cx<R> a5 = ffv_amp(w28, w29, g3);
    jamp[3].r += a5.i; jamp[3].i -= a5.r;
    const cx<R> a6 = ffv_amp(w28, v4, w15);
    jamp[2].r += a6.i; jamp[2].i -= a6.r;
    jamp[3].r -= a6.i; jamp[3].i += a6.r;
    const R q9_31[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w32 = ffv_row(w20, g3, q9_31, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a7 = ffv_amp(w32, w25, g1);
    jamp[4].r += a7.i; jamp[4].i -= a7.r;
    const cx<R> a8 = ffv_amp(w32, w29, g2);
    jamp[5].r += a8.i; jamp[5].i -= a8.r;
    const cx<R> a9 = ffv_amp(w32, v4, w12);
    jamp[4].r += a9.i; jamp[4].i -= a9.r;
    jamp[5].r -= a9.i; jamp[5].i += a9.r;
    const cx<R> a10 = ffv_amp(w20, w23, w12);
    jamp[0].r += a10.i; jamp[0].i -= a10.r;
    jamp[2].r -= a10.i; jamp[2].i += a10.r;
    const cx<R> a11 = ffv_amp(w20, w25, w15);
    jamp[1].r += a11.i; jamp[1].i -= a11.r;
    jamp[4].r -= a11.i; jamp[4].i += a11.r;
    const cx<R> a12 = ffv_amp(w20, w29, w18);
    jamp[3].r += a12.i; jamp[3].i -= a12.r;
    jamp[5].r -= a12.i; jamp[5].i += a12.r;
    const R q2_33[4] = {ldv(v.p3[0]) - ldv(v.K[1][0]), ldv(v.p3[1]) - ldv(v.K[1][1]), ldv(v.p3[2]) - ldv(v.K[1][2]), ldv(v.p3[3]) - ldv(v.K[1][3])};
    const W4<R> w34 = ffv_row(ub3, g1, q2_33, ldv(v.mt), ldv(v.iQ[1]));
    const R q3_35[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w36 = ffv_row(w34, g0, q3_35, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a13 = ffv_amp(w36, w23, g2);
    jamp[6].r += a13.i; jamp[6].i -= a13.r;
    const cx<R> a14 = ffv_amp(w36, w25, g3);
    jamp[7].r += a14.i; jamp[7].i -= a14.r;
    const cx<R> a15 = ffv_amp(w36, v4, w18);
    jamp[6].r += a15.i; jamp[6].i -= a15.r;
    jamp[7].r -= a15.i; jamp[7].i += a15.r;
    const R q6_37[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w38 = ffv_row(w34, g2, q6_37, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a16 = ffv_amp(w38, w23, g0);
    jamp[8].r += a16.i; jamp[8].i -= a16.r;
    const R q14_40[4] = {ldv(v.p3[0]) - ldv(v.K[13][0]), ldv(v.p3[1]) - ldv(v.K[13][1]), ldv(v.p3[2]) - ldv(v.K[13][2]), ldv(v.p3[3]) - ldv(v.K[13][3])};
    const W4<R> w39 = ffv_col(g0, v4, q14_40, ldv(v.mt), ldv(v.iQ[13]));
    const cx<R> a17 = ffv_amp(w38, w39, g3);
    jamp[9].r += a17.i; jamp[9].i -= a17.r;
    const cx<R> a18 = ffv_amp(w38, v4, w9);
    jamp[8].r += a18.i; jamp[8].i -= a18.r;
    jamp[9].r -= a18.i; jamp[9].i += a18.r;
    const R q10_41[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w42 = ffv_row(w34, g3, q10_41, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a19 = ffv_amp(w42, w25, g0);
    jamp[10].r += a19.i; jamp[10].i -= a19.r;
    const cx<R> a20 = ffv_amp(w42, w39, g2);
    jamp[11].r += a20.i; jamp[11].i -= a20.r;
    const cx<R> a21 = ffv_amp(w42, v4, w6);
    jamp[10].r += a21.i; jamp[10].i -= a21.r;
    jamp[11].r -= a21.i; jamp[11].i += a21.r;
    const cx<R> a22 = ffv_amp(w34, w23, w6);
    jamp[6].r += a22.i; jamp[6].i -= a22.r;
    jamp[8].r -= a22.i; jamp[8].i += a22.r;
    const cx<R> a23 = ffv_amp(w34, w25, w9);
    jamp[7].r += a23.i; jamp[7].i -= a23.r;
    jamp[10].r -= a23.i; jamp[10].i += a23.r;
    const cx<R> a24 = ffv_amp(w34, w39, w18);
    jamp[9].r += a24.i; jamp[9].i -= a24.r;
    jamp[11].r -= a24.i; jamp[11].i += a24.r;
    const R q4_43[4] = {ldv(v.p3[0]) - ldv(v.K[3][0]), ldv(v.p3[1]) - ldv(v.K[3][1]), ldv(v.p3[2]) - ldv(v.K[3][2]), ldv(v.p3[3]) - ldv(v.K[3][3])};
    const W4<R> w44 = ffv_row(ub3, g2, q4_43, ldv(v.mt), ldv(v.iQ[3]));
    const R q5_45[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w46 = ffv_row(w44, g0, q5_45, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a25 = ffv_amp(w46, w23, g1);
    jamp[12].r += a25.i; jamp[12].i -= a25.r;
    const cx<R> a26 = ffv_amp(w46, w29, g3);
    jamp[13].r += a26.i; jamp[13].i -= a26.r;
    const cx<R> a27 = ffv_amp(w46, v4, w15);
    jamp[12].r += a27.i; jamp[12].i -= a27.r;
    jamp[13].r -= a27.i; jamp[13].i += a27.r;
    const R q6_47[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w48 = ffv_row(w44, g1, q6_47, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a28 = ffv_amp(w48, w23, g0);
    jamp[14].r += a28.i; jamp[14].i -= a28.r;
    const cx<R> a29 = ffv_amp(w48, w39, g3);
    jamp[15].r += a29.i; jamp[15].i -= a29.r;
    const cx<R> a30 = ffv_amp(w48, v4, w9);
    jamp[14].r += a30.i; jamp[14].i -= a30.r;
    jamp[15].r -= a30.i; jamp[15].i += a30.r;
    const R q12_49[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w50 = ffv_row(w44, g3, q12_49, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a31 = ffv_amp(w50, w29, g0);
    jamp[16].r += a31.i; jamp[16].i -= a31.r;
    const cx<R> a32 = ffv_amp(w50, w39, g1);
    jamp[17].r += a32.i; jamp[17].i -= a32.r;
    const cx<R> a33 = ffv_amp(w50, v4, w3);
    jamp[16].r += a33.i; jamp[16].i -= a33.r;
    jamp[17].r -= a33.i; jamp[17].i += a33.r;
    const cx<R> a34 = ffv_amp(w44, w23, w3);
    jamp[12].r += a34.i; jamp[12].i -= a34.r;
    jamp[14].r -= a34.i; jamp[14].i += a34.r;
    const cx<R> a35 = ffv_amp(w44, w29, w9);
    jamp[13].r += a35.i; jamp[13].i -= a35.r;
    jamp[16].r -= a35.i; jamp[16].i += a35.r;
    const cx<R> a36 = ffv_amp(w44, w39, w15);
    jamp[15].r += a36.i; jamp[15].i -= a36.r;
    jamp[17].r -= a36.i; jamp[17].i += a36.r;
    const R q8_51[4] = {ldv(v.p3[0]) - ldv(v.K[7][0]), ldv(v.p3[1]) - ldv(v.K[7][1]), ldv(v.p3[2]) - ldv(v.K[7][2]), ldv(v.p3[3]) - ldv(v.K[7][3])};
    const W4<R> w52 = ffv_row(ub3, g3, q8_51, ldv(v.mt), ldv(v.iQ[7]));
    const R q9_53[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w54 = ffv_row(w52, g0, q9_53, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a37 = ffv_amp(w54, w25, g1);
    jamp[18].r += a37.i; jamp[18].i -= a37.r;
    const cx<R> a38 = ffv_amp(w54, w29, g2);
    jamp[19].r += a38.i; jamp[19].i -= a38.r;
    const cx<R> a39 = ffv_amp(w54, v4, w12);
    jamp[18].r += a39.i; jamp[18].i -= a39.r;
    jamp[19].r -= a39.i; jamp[19].i += a39.r;
    const R q10_55[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w56 = ffv_row(w52, g1, q10_55, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a40 = ffv_amp(w56, w25, g0);
    jamp[20].r += a40.i; jamp[20].i -= a40.r;
    const cx<R> a41 = ffv_amp(w56, w39, g2);
    jamp[21].r += a41.i; jamp[21].i -= a41.r;
    const cx<R> a42 = ffv_amp(w56, v4, w6);
    jamp[20].r += a42.i; jamp[20].i -= a42.r;
    jamp[21].r -= a42.i; jamp[21].i += a42.r;
    const R q12_57[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w58 = ffv_row(w52, g2, q12_57, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a43 = ffv_amp(w58, w29, g0);
    jamp[22].r += a43.i; jamp[22].i -= a43.r;
    const cx<R> a44 = ffv_amp(w58, w39, g1);
    jamp[23].r += a44.i; jamp[23].i -= a44.r;
    const cx<R> a45 = ffv_amp(w58, v4, w3);
    jamp[22].r += a45.i; jamp[22].i -= a45.r;
    jamp[23].r -= a45.i; jamp[23].i += a45.r;
    const cx<R> a46 = ffv_amp(w52, w25, w3);
    jamp[18].r += a46.i; jamp[18].i -= a46.r;
    jamp[20].r -= a46.i; jamp[20].i += a46.r;
    const cx<R> a47 = ffv_amp(w52, w29, w6);
    jamp[19].r += a47.i; jamp[19].i -= a47.r;
    jamp[22].r -= a47.i; jamp[22].i += a47.r;
    const cx<R> a48 = ffv_amp(w52, w39, w12);
    jamp[21].r += a48.i; jamp[21].i -= a48.r;
    jamp[23].r -= a48.i; jamp[23].i += a48.r;
    const R q3_59[4] = {ldv(v.p3[0]) - ldv(v.K[2][0]), ldv(v.p3[1]) - ldv(v.K[2][1]), ldv(v.p3[2]) - ldv(v.K[2][2]), ldv(v.p3[3]) - ldv(v.K[2][3])};
    const W4<R> w60 = ffv_row(ub3, w3, q3_59, ldv(v.mt), ldv(v.iQ[2]));
    const cx<R> a49 = ffv_amp(w60, w23, g2);
    jamp[0].r += a49.i; jamp[0].i -= a49.r;
    jamp[6].r -= a49.i; jamp[6].i += a49.r;
    const cx<R> a50 = ffv_amp(w60, w25, g3);
    jamp[1].r += a50.i; jamp[1].i -= a50.r;
    jamp[7].r -= a50.i; jamp[7].i += a50.r;
    const cx<R> a51 = ffv_amp(w60, v4, w18);
    jamp[0].r += a51.i; jamp[0].i -= a51.r;
    jamp[1].r -= a51.i; jamp[1].i += a51.r;
    jamp[6].r -= a51.i; jamp[6].i += a51.r;
    jamp[7].r += a51.i; jamp[7].i -= a51.r;
    const R q5_61[4] = {ldv(v.p3[0]) - ldv(v.K[4][0]), ldv(v.p3[1]) - ldv(v.K[4][1]), ldv(v.p3[2]) - ldv(v.K[4][2]), ldv(v.p3[3]) - ldv(v.K[4][3])};
    const W4<R> w62 = ffv_row(ub3, w6, q5_61, ldv(v.mt), ldv(v.iQ[4]));
    const cx<R> a52 = ffv_amp(w62, w23, g1);
    jamp[2].r += a52.i; jamp[2].i -= a52.r;
    jamp[12].r -= a52.i; jamp[12].i += a52.r;
    const cx<R> a53 = ffv_amp(w62, w29, g3);
    jamp[3].r += a53.i; jamp[3].i -= a53.r;
    jamp[13].r -= a53.i; jamp[13].i += a53.r;
    const cx<R> a54 = ffv_amp(w62, v4, w15);
    jamp[2].r += a54.i; jamp[2].i -= a54.r;
    jamp[3].r -= a54.i; jamp[3].i += a54.r;
    jamp[12].r -= a54.i; jamp[12].i += a54.r;
    jamp[13].r += a54.i; jamp[13].i -= a54.r;
    const R q9_63[4] = {ldv(v.p3[0]) - ldv(v.K[8][0]), ldv(v.p3[1]) - ldv(v.K[8][1]), ldv(v.p3[2]) - ldv(v.K[8][2]), ldv(v.p3[3]) - ldv(v.K[8][3])};
    const W4<R> w64 = ffv_row(ub3, w9, q9_63, ldv(v.mt), ldv(v.iQ[8]));
    const cx<R> a55 = ffv_amp(w64, w25, g1);
    jamp[4].r += a55.i; jamp[4].i -= a55.r;
    jamp[18].r -= a55.i; jamp[18].i += a55.r;
    const cx<R> a56 = ffv_amp(w64, w29, g2);
    jamp[5].r += a56.i; jamp[5].i -= a56.r;
    jamp[19].r -= a56.i; jamp[19].i += a56.r;
    const cx<R> a57 = ffv_amp(w64, v4, w12);
    jamp[4].r += a57.i; jamp[4].i -= a57.r;
    jamp[5].r -= a57.i; jamp[5].i += a57.r;
    jamp[18].r -= a57.i; jamp[18].i += a57.r;
    jamp[19].r += a57.i; jamp[19].i -= a57.r;
    const R q6_65[4] = {ldv(v.p3[0]) - ldv(v.K[5][0]), ldv(v.p3[1]) - ldv(v.K[5][1]), ldv(v.p3[2]) - ldv(v.K[5][2]), ldv(v.p3[3]) - ldv(v.K[5][3])};
    const W4<R> w66 = ffv_row(ub3, w12, q6_65, ldv(v.mt), ldv(v.iQ[5]));
    const cx<R> a58 = ffv_amp(w66, w23, g0);
    jamp[8].r += a58.i; jamp[8].i -= a58.r;
    jamp[14].r -= a58.i; jamp[14].i += a58.r;
    const cx<R> a59 = ffv_amp(w66, w39, g3);
    jamp[9].r += a59.i; jamp[9].i -= a59.r;
    jamp[15].r -= a59.i; jamp[15].i += a59.r;
    const cx<R> a60 = ffv_amp(w66, v4, w9);
    jamp[8].r += a60.i; jamp[8].i -= a60.r;
    jamp[9].r -= a60.i; jamp[9].i += a60.r;
    jamp[14].r -= a60.i; jamp[14].i += a60.r;
    jamp[15].r += a60.i; jamp[15].i -= a60.r;
    const R q10_67[4] = {ldv(v.p3[0]) - ldv(v.K[9][0]), ldv(v.p3[1]) - ldv(v.K[9][1]), ldv(v.p3[2]) - ldv(v.K[9][2]), ldv(v.p3[3]) - ldv(v.K[9][3])};
    const W4<R> w68 = ffv_row(ub3, w15, q10_67, ldv(v.mt), ldv(v.iQ[9]));
    const cx<R> a61 = ffv_amp(w68, w25, g0);
    jamp[10].r += a61.i; jamp[10].i -= a61.r;
    jamp[20].r -= a61.i; jamp[20].i += a61.r;
    const cx<R> a62 = ffv_amp(w68, w39, g2);
    jamp[11].r += a62.i; jamp[11].i -= a62.r;
    jamp[21].r -= a62.i; jamp[21].i += a62.r;
    const cx<R> a63 = ffv_amp(w68, v4, w6);
    jamp[10].r += a63.i; jamp[10].i -= a63.r;
    jamp[11].r -= a63.i; jamp[11].i += a63.r;
    jamp[20].r -= a63.i; jamp[20].i += a63.r;
    jamp[21].r += a63.i; jamp[21].i -= a63.r;
    const R q12_69[4] = {ldv(v.p3[0]) - ldv(v.K[11][0]), ldv(v.p3[1]) - ldv(v.K[11][1]), ldv(v.p3[2]) - ldv(v.K[11][2]), ldv(v.p3[3]) - ldv(v.K[11][3])};
    const W4<R> w70 = ffv_row(ub3, w18, q12_69, ldv(v.mt), ldv(v.iQ[11]));
    const cx<R> a64 = ffv_amp(w70, w29, g0);
    jamp[16].r += a64.i; jamp[16].i -= a64.r;
    jamp[22].r -= a64.i; jamp[22].i += a64.r;
    const cx<R> a65 = ffv_amp(w70, w39, g1);
    jamp[17].r += a65.i; jamp[17].i -= a65.r;
    jamp[23].r -= a65.i; jamp[23].i += a65.r;
    const cx<R> a66 = ffv_amp(w70, v4, w3);
    jamp[16].r += a66.i; jamp[16].i -= a66.r;
    jamp[17].r -= a66.i; jamp[17].i += a66.r;
    jamp[22].r -= a66.i; jamp[22].i += a66.r;
    jamp[23].r += a66.i; jamp[23].i -= a66.r;
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
    jamp[18].r += a67.i; jamp[18].i -= a67.r;
    jamp[19].r -= a67.i; jamp[19].i += a67.r;
    jamp[21].r -= a67.i; jamp[21].i += a67.r;
    jamp[23].r += a67.i; jamp[23].i -= a67.r;
    const cx<R> a68 = ffv_amp(ub3, w71, w77);
    jamp[0].r += a68.i; jamp[0].i -= a68.r;
    jamp[2].r -= a68.i; jamp[2].i += a68.r;
    jamp[8].r -= a68.i; jamp[8].i += a68.r;
    jamp[14].r += a68.i; jamp[14].i -= a68.r;
    const R k7_78[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_79[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_80[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_80[4] = {-k15_80[0], -k15_80[1], -k15_80[2], -k15_80[3]};
    const cx<R> a69 = vvv_amp(w77, g3, jq, k7_78, k8_79, nkk15_80);
    jamp[0].r += a69.i; jamp[0].i -= a69.r;
    jamp[2].r -= a69.i; jamp[2].i += a69.r;
    jamp[8].r -= a69.i; jamp[8].i += a69.r;
    jamp[14].r += a69.i; jamp[14].i -= a69.r;
    jamp[18].r -= a69.i; jamp[18].i += a69.r;
    jamp[19].r += a69.i; jamp[19].i -= a69.r;
    jamp[21].r += a69.i; jamp[21].i -= a69.r;
    jamp[23].r -= a69.i; jamp[23].i += a69.r;
    }
    {
    const R k3_81[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k4_82[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w83 = vvv_cur(w3, g2, k3_81, k4_82, ldv(v.iG[3]));
    const cx<R> a70 = ffv_amp(w74, v4, w83);
    jamp[18].r += a70.i; jamp[18].i -= a70.r;
    jamp[20].r -= a70.i; jamp[20].i += a70.r;
    jamp[22].r -= a70.i; jamp[22].i += a70.r;
    jamp[23].r += a70.i; jamp[23].i -= a70.r;
    const cx<R> a71 = ffv_amp(ub3, w71, w83);
    jamp[0].r += a71.i; jamp[0].i -= a71.r;
    jamp[6].r -= a71.i; jamp[6].i += a71.r;
    jamp[12].r -= a71.i; jamp[12].i += a71.r;
    jamp[14].r += a71.i; jamp[14].i -= a71.r;
    const R k7_84[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_85[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_86[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_86[4] = {-k15_86[0], -k15_86[1], -k15_86[2], -k15_86[3]};
    const cx<R> a72 = vvv_amp(w83, g3, jq, k7_84, k8_85, nkk15_86);
    jamp[0].r += a72.i; jamp[0].i -= a72.r;
    jamp[6].r -= a72.i; jamp[6].i += a72.r;
    jamp[12].r -= a72.i; jamp[12].i += a72.r;
    jamp[14].r += a72.i; jamp[14].i -= a72.r;
    jamp[18].r -= a72.i; jamp[18].i += a72.r;
    jamp[20].r += a72.i; jamp[20].i -= a72.r;
    jamp[22].r += a72.i; jamp[22].i -= a72.r;
    jamp[23].r -= a72.i; jamp[23].i += a72.r;
    }
    {
    const R k5_87[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k2_88[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w89 = vvv_cur(w6, g1, k5_87, k2_88, ldv(v.iG[3]));
    const cx<R> a73 = ffv_amp(w74, v4, w89);
    jamp[19].r += a73.i; jamp[19].i -= a73.r;
    jamp[20].r -= a73.i; jamp[20].i += a73.r;
    jamp[21].r += a73.i; jamp[21].i -= a73.r;
    jamp[22].r -= a73.i; jamp[22].i += a73.r;
    const cx<R> a74 = ffv_amp(ub3, w71, w89);
    jamp[2].r += a74.i; jamp[2].i -= a74.r;
    jamp[6].r -= a74.i; jamp[6].i += a74.r;
    jamp[8].r += a74.i; jamp[8].i -= a74.r;
    jamp[12].r -= a74.i; jamp[12].i += a74.r;
    const R k7_90[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_91[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_92[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_92[4] = {-k15_92[0], -k15_92[1], -k15_92[2], -k15_92[3]};
    const cx<R> a75 = vvv_amp(w89, g3, jq, k7_90, k8_91, nkk15_92);
    jamp[2].r += a75.i; jamp[2].i -= a75.r;
    jamp[6].r -= a75.i; jamp[6].i += a75.r;
    jamp[8].r += a75.i; jamp[8].i -= a75.r;
    jamp[12].r -= a75.i; jamp[12].i += a75.r;
    jamp[19].r -= a75.i; jamp[19].i += a75.r;
    jamp[20].r += a75.i; jamp[20].i -= a75.r;
    jamp[21].r -= a75.i; jamp[21].i += a75.r;
    jamp[22].r += a75.i; jamp[22].i -= a75.r;
    }
    {
    W4<R> w93, w94, w95;
    vvvv_cur(g0, g1, g2, ldv(v.iG[3]), w93, w94, w95);
    const cx<R> a76 = ffv_amp(w74, v4, w93);
    jamp[18].r += a76.i; jamp[18].i -= a76.r;
    jamp[20].r -= a76.i; jamp[20].i += a76.r;
    jamp[22].r -= a76.i; jamp[22].i += a76.r;
    jamp[23].r += a76.i; jamp[23].i -= a76.r;
    const cx<R> a77 = ffv_amp(ub3, w71, w93);
    jamp[0].r += a77.i; jamp[0].i -= a77.r;
    jamp[6].r -= a77.i; jamp[6].i += a77.r;
    jamp[12].r -= a77.i; jamp[12].i += a77.r;
    jamp[14].r += a77.i; jamp[14].i -= a77.r;
    const R k7_96[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_97[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_98[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_98[4] = {-k15_98[0], -k15_98[1], -k15_98[2], -k15_98[3]};
    const cx<R> a78 = vvv_amp(w93, g3, jq, k7_96, k8_97, nkk15_98);
    jamp[0].r += a78.i; jamp[0].i -= a78.r;
    jamp[6].r -= a78.i; jamp[6].i += a78.r;
    jamp[12].r -= a78.i; jamp[12].i += a78.r;
    jamp[14].r += a78.i; jamp[14].i -= a78.r;
    jamp[18].r -= a78.i; jamp[18].i += a78.r;
    jamp[20].r += a78.i; jamp[20].i -= a78.r;
    jamp[22].r += a78.i; jamp[22].i -= a78.r;
    jamp[23].r -= a78.i; jamp[23].i += a78.r;
    const cx<R> a79 = ffv_amp(w74, v4, w94);
    jamp[19].r += a79.i; jamp[19].i -= a79.r;
    jamp[20].r -= a79.i; jamp[20].i += a79.r;
    jamp[21].r += a79.i; jamp[21].i -= a79.r;
    jamp[22].r -= a79.i; jamp[22].i += a79.r;
    const cx<R> a80 = ffv_amp(ub3, w71, w94);
    jamp[2].r += a80.i; jamp[2].i -= a80.r;
    jamp[6].r -= a80.i; jamp[6].i += a80.r;
    jamp[8].r += a80.i; jamp[8].i -= a80.r;
    jamp[12].r -= a80.i; jamp[12].i += a80.r;
    const R k7_99[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_100[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_101[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_101[4] = {-k15_101[0], -k15_101[1], -k15_101[2], -k15_101[3]};
    const cx<R> a81 = vvv_amp(w94, g3, jq, k7_99, k8_100, nkk15_101);
    jamp[2].r += a81.i; jamp[2].i -= a81.r;
    jamp[6].r -= a81.i; jamp[6].i += a81.r;
    jamp[8].r += a81.i; jamp[8].i -= a81.r;
    jamp[12].r -= a81.i; jamp[12].i += a81.r;
    jamp[19].r -= a81.i; jamp[19].i += a81.r;
    jamp[20].r += a81.i; jamp[20].i -= a81.r;
    jamp[21].r -= a81.i; jamp[21].i += a81.r;
    jamp[22].r += a81.i; jamp[22].i -= a81.r;
    const cx<R> a82 = ffv_amp(w74, v4, w95);
    jamp[18].r -= a82.i; jamp[18].i += a82.r;
    jamp[19].r += a82.i; jamp[19].i -= a82.r;
    jamp[21].r += a82.i; jamp[21].i -= a82.r;
    jamp[23].r -= a82.i; jamp[23].i += a82.r;
    const cx<R> a83 = ffv_amp(ub3, w71, w95);
    jamp[0].r -= a83.i; jamp[0].i += a83.r;
    jamp[2].r += a83.i; jamp[2].i -= a83.r;
    jamp[8].r += a83.i; jamp[8].i -= a83.r;
    jamp[14].r -= a83.i; jamp[14].i += a83.r;
    const R k7_102[4] = {ldv(v.K[6][0]), ldv(v.K[6][1]), ldv(v.K[6][2]), ldv(v.K[6][3])};
    const R k8_103[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const R k15_104[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_104[4] = {-k15_104[0], -k15_104[1], -k15_104[2], -k15_104[3]};
    const cx<R> a84 = vvv_amp(w95, g3, jq, k7_102, k8_103, nkk15_104);
    jamp[0].r -= a84.i; jamp[0].i += a84.r;
    jamp[2].r += a84.i; jamp[2].i -= a84.r;
    jamp[8].r += a84.i; jamp[8].i -= a84.r;
    jamp[14].r -= a84.i; jamp[14].i += a84.r;
    jamp[18].r += a84.i; jamp[18].i -= a84.r;
    jamp[19].r -= a84.i; jamp[19].i += a84.r;
    jamp[21].r -= a84.i; jamp[21].i += a84.r;
    jamp[23].r += a84.i; jamp[23].i -= a84.r;
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
    jamp[12].r += a85.i; jamp[12].i -= a85.r;
    jamp[13].r -= a85.i; jamp[13].i += a85.r;
    jamp[15].r -= a85.i; jamp[15].i += a85.r;
    jamp[17].r += a85.i; jamp[17].i -= a85.r;
    const cx<R> a86 = ffv_amp(ub3, w105, w111);
    jamp[1].r += a86.i; jamp[1].i -= a86.r;
    jamp[4].r -= a86.i; jamp[4].i += a86.r;
    jamp[10].r -= a86.i; jamp[10].i += a86.r;
    jamp[20].r += a86.i; jamp[20].i -= a86.r;
    const R k11_112[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_113[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_114[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_114[4] = {-k15_114[0], -k15_114[1], -k15_114[2], -k15_114[3]};
    const cx<R> a87 = vvv_amp(w111, g2, jq, k11_112, k4_113, nkk15_114);
    jamp[1].r += a87.i; jamp[1].i -= a87.r;
    jamp[4].r -= a87.i; jamp[4].i += a87.r;
    jamp[10].r -= a87.i; jamp[10].i += a87.r;
    jamp[12].r -= a87.i; jamp[12].i += a87.r;
    jamp[13].r += a87.i; jamp[13].i -= a87.r;
    jamp[15].r += a87.i; jamp[15].i -= a87.r;
    jamp[17].r -= a87.i; jamp[17].i += a87.r;
    jamp[20].r += a87.i; jamp[20].i -= a87.r;
    }
    {
    const R k3_115[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k8_116[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w117 = vvv_cur(w3, g3, k3_115, k8_116, ldv(v.iG[6]));
    const cx<R> a88 = ffv_amp(w108, v4, w117);
    jamp[12].r += a88.i; jamp[12].i -= a88.r;
    jamp[14].r -= a88.i; jamp[14].i += a88.r;
    jamp[16].r -= a88.i; jamp[16].i += a88.r;
    jamp[17].r += a88.i; jamp[17].i -= a88.r;
    const cx<R> a89 = ffv_amp(ub3, w105, w117);
    jamp[1].r += a89.i; jamp[1].i -= a89.r;
    jamp[7].r -= a89.i; jamp[7].i += a89.r;
    jamp[18].r -= a89.i; jamp[18].i += a89.r;
    jamp[20].r += a89.i; jamp[20].i -= a89.r;
    const R k11_118[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_119[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_120[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_120[4] = {-k15_120[0], -k15_120[1], -k15_120[2], -k15_120[3]};
    const cx<R> a90 = vvv_amp(w117, g2, jq, k11_118, k4_119, nkk15_120);
    jamp[1].r += a90.i; jamp[1].i -= a90.r;
    jamp[7].r -= a90.i; jamp[7].i += a90.r;
    jamp[12].r -= a90.i; jamp[12].i += a90.r;
    jamp[14].r += a90.i; jamp[14].i -= a90.r;
    jamp[16].r += a90.i; jamp[16].i -= a90.r;
    jamp[17].r -= a90.i; jamp[17].i += a90.r;
    jamp[18].r -= a90.i; jamp[18].i += a90.r;
    jamp[20].r += a90.i; jamp[20].i -= a90.r;
    }
    {
    const R k9_121[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k2_122[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const W4<R> w123 = vvv_cur(w9, g1, k9_121, k2_122, ldv(v.iG[6]));
    const cx<R> a91 = ffv_amp(w108, v4, w123);
    jamp[13].r += a91.i; jamp[13].i -= a91.r;
    jamp[14].r -= a91.i; jamp[14].i += a91.r;
    jamp[15].r += a91.i; jamp[15].i -= a91.r;
    jamp[16].r -= a91.i; jamp[16].i += a91.r;
    const cx<R> a92 = ffv_amp(ub3, w105, w123);
    jamp[4].r += a92.i; jamp[4].i -= a92.r;
    jamp[7].r -= a92.i; jamp[7].i += a92.r;
    jamp[10].r += a92.i; jamp[10].i -= a92.r;
    jamp[18].r -= a92.i; jamp[18].i += a92.r;
    const R k11_124[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_125[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_126[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_126[4] = {-k15_126[0], -k15_126[1], -k15_126[2], -k15_126[3]};
    const cx<R> a93 = vvv_amp(w123, g2, jq, k11_124, k4_125, nkk15_126);
    jamp[4].r += a93.i; jamp[4].i -= a93.r;
    jamp[7].r -= a93.i; jamp[7].i += a93.r;
    jamp[10].r += a93.i; jamp[10].i -= a93.r;
    jamp[13].r -= a93.i; jamp[13].i += a93.r;
    jamp[14].r += a93.i; jamp[14].i -= a93.r;
    jamp[15].r -= a93.i; jamp[15].i += a93.r;
    jamp[16].r += a93.i; jamp[16].i -= a93.r;
    jamp[18].r -= a93.i; jamp[18].i += a93.r;
    }
    {
    W4<R> w127, w128, w129;
    vvvv_cur(g0, g1, g3, ldv(v.iG[6]), w127, w128, w129);
    const cx<R> a94 = ffv_amp(w108, v4, w127);
    jamp[12].r += a94.i; jamp[12].i -= a94.r;
    jamp[14].r -= a94.i; jamp[14].i += a94.r;
    jamp[16].r -= a94.i; jamp[16].i += a94.r;
    jamp[17].r += a94.i; jamp[17].i -= a94.r;
    const cx<R> a95 = ffv_amp(ub3, w105, w127);
    jamp[1].r += a95.i; jamp[1].i -= a95.r;
    jamp[7].r -= a95.i; jamp[7].i += a95.r;
    jamp[18].r -= a95.i; jamp[18].i += a95.r;
    jamp[20].r += a95.i; jamp[20].i -= a95.r;
    const R k11_130[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_131[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_132[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_132[4] = {-k15_132[0], -k15_132[1], -k15_132[2], -k15_132[3]};
    const cx<R> a96 = vvv_amp(w127, g2, jq, k11_130, k4_131, nkk15_132);
    jamp[1].r += a96.i; jamp[1].i -= a96.r;
    jamp[7].r -= a96.i; jamp[7].i += a96.r;
    jamp[12].r -= a96.i; jamp[12].i += a96.r;
    jamp[14].r += a96.i; jamp[14].i -= a96.r;
    jamp[16].r += a96.i; jamp[16].i -= a96.r;
    jamp[17].r -= a96.i; jamp[17].i += a96.r;
    jamp[18].r -= a96.i; jamp[18].i += a96.r;
    jamp[20].r += a96.i; jamp[20].i -= a96.r;
    const cx<R> a97 = ffv_amp(w108, v4, w128);
    jamp[13].r += a97.i; jamp[13].i -= a97.r;
    jamp[14].r -= a97.i; jamp[14].i += a97.r;
    jamp[15].r += a97.i; jamp[15].i -= a97.r;
    jamp[16].r -= a97.i; jamp[16].i += a97.r;
    const cx<R> a98 = ffv_amp(ub3, w105, w128);
    jamp[4].r += a98.i; jamp[4].i -= a98.r;
    jamp[7].r -= a98.i; jamp[7].i += a98.r;
    jamp[10].r += a98.i; jamp[10].i -= a98.r;
    jamp[18].r -= a98.i; jamp[18].i += a98.r;
    const R k11_133[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_134[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_135[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_135[4] = {-k15_135[0], -k15_135[1], -k15_135[2], -k15_135[3]};
    const cx<R> a99 = vvv_amp(w128, g2, jq, k11_133, k4_134, nkk15_135);
    jamp[4].r += a99.i; jamp[4].i -= a99.r;
    jamp[7].r -= a99.i; jamp[7].i += a99.r;
    jamp[10].r += a99.i; jamp[10].i -= a99.r;
    jamp[13].r -= a99.i; jamp[13].i += a99.r;
    jamp[14].r += a99.i; jamp[14].i -= a99.r;
    jamp[15].r -= a99.i; jamp[15].i += a99.r;
    jamp[16].r += a99.i; jamp[16].i -= a99.r;
    jamp[18].r -= a99.i; jamp[18].i += a99.r;
    const cx<R> a100 = ffv_amp(w108, v4, w129);
    jamp[12].r -= a100.i; jamp[12].i += a100.r;
    jamp[13].r += a100.i; jamp[13].i -= a100.r;
    jamp[15].r += a100.i; jamp[15].i -= a100.r;
    jamp[17].r -= a100.i; jamp[17].i += a100.r;
    const cx<R> a101 = ffv_amp(ub3, w105, w129);
    jamp[1].r -= a101.i; jamp[1].i += a101.r;
    jamp[4].r += a101.i; jamp[4].i -= a101.r;
    jamp[10].r += a101.i; jamp[10].i -= a101.r;
    jamp[20].r -= a101.i; jamp[20].i += a101.r;
    const R k11_136[4] = {ldv(v.K[10][0]), ldv(v.K[10][1]), ldv(v.K[10][2]), ldv(v.K[10][3])};
    const R k4_137[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const R k15_138[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_138[4] = {-k15_138[0], -k15_138[1], -k15_138[2], -k15_138[3]};
    const cx<R> a102 = vvv_amp(w129, g2, jq, k11_136, k4_137, nkk15_138);
    jamp[1].r -= a102.i; jamp[1].i += a102.r;
    jamp[4].r += a102.i; jamp[4].i -= a102.r;
    jamp[10].r += a102.i; jamp[10].i -= a102.r;
    jamp[12].r += a102.i; jamp[12].i -= a102.r;
    jamp[13].r -= a102.i; jamp[13].i += a102.r;
    jamp[15].r -= a102.i; jamp[15].i += a102.r;
    jamp[17].r += a102.i; jamp[17].i -= a102.r;
    jamp[20].r -= a102.i; jamp[20].i += a102.r;
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
    jamp[6].r += a103.i; jamp[6].i -= a103.r;
    jamp[7].r -= a103.i; jamp[7].i += a103.r;
    jamp[9].r -= a103.i; jamp[9].i += a103.r;
    jamp[11].r += a103.i; jamp[11].i -= a103.r;
    const cx<R> a104 = ffv_amp(ub3, w139, w145);
    jamp[3].r += a104.i; jamp[3].i -= a104.r;
    jamp[5].r -= a104.i; jamp[5].i += a104.r;
    jamp[16].r -= a104.i; jamp[16].i += a104.r;
    jamp[22].r += a104.i; jamp[22].i -= a104.r;
    const R k13_146[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_147[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_148[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_148[4] = {-k15_148[0], -k15_148[1], -k15_148[2], -k15_148[3]};
    const cx<R> a105 = vvv_amp(w145, g1, jq, k13_146, k2_147, nkk15_148);
    jamp[3].r += a105.i; jamp[3].i -= a105.r;
    jamp[5].r -= a105.i; jamp[5].i += a105.r;
    jamp[6].r -= a105.i; jamp[6].i += a105.r;
    jamp[7].r += a105.i; jamp[7].i -= a105.r;
    jamp[9].r += a105.i; jamp[9].i -= a105.r;
    jamp[11].r -= a105.i; jamp[11].i += a105.r;
    jamp[16].r -= a105.i; jamp[16].i += a105.r;
    jamp[22].r += a105.i; jamp[22].i -= a105.r;
    }
    {
    const R k5_149[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k8_150[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w151 = vvv_cur(w6, g3, k5_149, k8_150, ldv(v.iG[8]));
    const cx<R> a106 = ffv_amp(w142, v4, w151);
    jamp[6].r += a106.i; jamp[6].i -= a106.r;
    jamp[8].r -= a106.i; jamp[8].i += a106.r;
    jamp[10].r -= a106.i; jamp[10].i += a106.r;
    jamp[11].r += a106.i; jamp[11].i -= a106.r;
    const cx<R> a107 = ffv_amp(ub3, w139, w151);
    jamp[3].r += a107.i; jamp[3].i -= a107.r;
    jamp[13].r -= a107.i; jamp[13].i += a107.r;
    jamp[19].r -= a107.i; jamp[19].i += a107.r;
    jamp[22].r += a107.i; jamp[22].i -= a107.r;
    const R k13_152[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_153[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_154[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_154[4] = {-k15_154[0], -k15_154[1], -k15_154[2], -k15_154[3]};
    const cx<R> a108 = vvv_amp(w151, g1, jq, k13_152, k2_153, nkk15_154);
    jamp[3].r += a108.i; jamp[3].i -= a108.r;
    jamp[6].r -= a108.i; jamp[6].i += a108.r;
    jamp[8].r += a108.i; jamp[8].i -= a108.r;
    jamp[10].r += a108.i; jamp[10].i -= a108.r;
    jamp[11].r -= a108.i; jamp[11].i += a108.r;
    jamp[13].r -= a108.i; jamp[13].i += a108.r;
    jamp[19].r -= a108.i; jamp[19].i += a108.r;
    jamp[22].r += a108.i; jamp[22].i -= a108.r;
    }
    {
    const R k9_155[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k4_156[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w157 = vvv_cur(w9, g2, k9_155, k4_156, ldv(v.iG[8]));
    const cx<R> a109 = ffv_amp(w142, v4, w157);
    jamp[7].r += a109.i; jamp[7].i -= a109.r;
    jamp[8].r -= a109.i; jamp[8].i += a109.r;
    jamp[9].r += a109.i; jamp[9].i -= a109.r;
    jamp[10].r -= a109.i; jamp[10].i += a109.r;
    const cx<R> a110 = ffv_amp(ub3, w139, w157);
    jamp[5].r += a110.i; jamp[5].i -= a110.r;
    jamp[13].r -= a110.i; jamp[13].i += a110.r;
    jamp[16].r += a110.i; jamp[16].i -= a110.r;
    jamp[19].r -= a110.i; jamp[19].i += a110.r;
    const R k13_158[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_159[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_160[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_160[4] = {-k15_160[0], -k15_160[1], -k15_160[2], -k15_160[3]};
    const cx<R> a111 = vvv_amp(w157, g1, jq, k13_158, k2_159, nkk15_160);
    jamp[5].r += a111.i; jamp[5].i -= a111.r;
    jamp[7].r -= a111.i; jamp[7].i += a111.r;
    jamp[8].r += a111.i; jamp[8].i -= a111.r;
    jamp[9].r -= a111.i; jamp[9].i += a111.r;
    jamp[10].r += a111.i; jamp[10].i -= a111.r;
    jamp[13].r -= a111.i; jamp[13].i += a111.r;
    jamp[16].r += a111.i; jamp[16].i -= a111.r;
    jamp[19].r -= a111.i; jamp[19].i += a111.r;
    }
    {
    W4<R> w161, w162, w163;
    vvvv_cur(g0, g2, g3, ldv(v.iG[8]), w161, w162, w163);
    const cx<R> a112 = ffv_amp(w142, v4, w161);
    jamp[6].r += a112.i; jamp[6].i -= a112.r;
    jamp[8].r -= a112.i; jamp[8].i += a112.r;
    jamp[10].r -= a112.i; jamp[10].i += a112.r;
    jamp[11].r += a112.i; jamp[11].i -= a112.r;
    const cx<R> a113 = ffv_amp(ub3, w139, w161);
    jamp[3].r += a113.i; jamp[3].i -= a113.r;
    jamp[13].r -= a113.i; jamp[13].i += a113.r;
    jamp[19].r -= a113.i; jamp[19].i += a113.r;
    jamp[22].r += a113.i; jamp[22].i -= a113.r;
    const R k13_164[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_165[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_166[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_166[4] = {-k15_166[0], -k15_166[1], -k15_166[2], -k15_166[3]};
    const cx<R> a114 = vvv_amp(w161, g1, jq, k13_164, k2_165, nkk15_166);
    jamp[3].r += a114.i; jamp[3].i -= a114.r;
    jamp[6].r -= a114.i; jamp[6].i += a114.r;
    jamp[8].r += a114.i; jamp[8].i -= a114.r;
    jamp[10].r += a114.i; jamp[10].i -= a114.r;
    jamp[11].r -= a114.i; jamp[11].i += a114.r;
    jamp[13].r -= a114.i; jamp[13].i += a114.r;
    jamp[19].r -= a114.i; jamp[19].i += a114.r;
    jamp[22].r += a114.i; jamp[22].i -= a114.r;
    const cx<R> a115 = ffv_amp(w142, v4, w162);
    jamp[7].r += a115.i; jamp[7].i -= a115.r;
    jamp[8].r -= a115.i; jamp[8].i += a115.r;
    jamp[9].r += a115.i; jamp[9].i -= a115.r;
    jamp[10].r -= a115.i; jamp[10].i += a115.r;
    const cx<R> a116 = ffv_amp(ub3, w139, w162);
    jamp[5].r += a116.i; jamp[5].i -= a116.r;
    jamp[13].r -= a116.i; jamp[13].i += a116.r;
    jamp[16].r += a116.i; jamp[16].i -= a116.r;
    jamp[19].r -= a116.i; jamp[19].i += a116.r;
    const R k13_167[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_168[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_169[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_169[4] = {-k15_169[0], -k15_169[1], -k15_169[2], -k15_169[3]};
    const cx<R> a117 = vvv_amp(w162, g1, jq, k13_167, k2_168, nkk15_169);
    jamp[5].r += a117.i; jamp[5].i -= a117.r;
    jamp[7].r -= a117.i; jamp[7].i += a117.r;
    jamp[8].r += a117.i; jamp[8].i -= a117.r;
    jamp[9].r -= a117.i; jamp[9].i += a117.r;
    jamp[10].r += a117.i; jamp[10].i -= a117.r;
    jamp[13].r -= a117.i; jamp[13].i += a117.r;
    jamp[16].r += a117.i; jamp[16].i -= a117.r;
    jamp[19].r -= a117.i; jamp[19].i += a117.r;
    const cx<R> a118 = ffv_amp(w142, v4, w163);
    jamp[6].r -= a118.i; jamp[6].i += a118.r;
    jamp[7].r += a118.i; jamp[7].i -= a118.r;
    jamp[9].r += a118.i; jamp[9].i -= a118.r;
    jamp[11].r -= a118.i; jamp[11].i += a118.r;
    const cx<R> a119 = ffv_amp(ub3, w139, w163);
    jamp[3].r -= a119.i; jamp[3].i += a119.r;
    jamp[5].r += a119.i; jamp[5].i -= a119.r;
    jamp[16].r += a119.i; jamp[16].i -= a119.r;
    jamp[22].r -= a119.i; jamp[22].i += a119.r;
    const R k13_170[4] = {ldv(v.K[12][0]), ldv(v.K[12][1]), ldv(v.K[12][2]), ldv(v.K[12][3])};
    const R k2_171[4] = {ldv(v.K[1][0]), ldv(v.K[1][1]), ldv(v.K[1][2]), ldv(v.K[1][3])};
    const R k15_172[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_172[4] = {-k15_172[0], -k15_172[1], -k15_172[2], -k15_172[3]};
    const cx<R> a120 = vvv_amp(w163, g1, jq, k13_170, k2_171, nkk15_172);
    jamp[3].r -= a120.i; jamp[3].i += a120.r;
    jamp[5].r += a120.i; jamp[5].i -= a120.r;
    jamp[6].r += a120.i; jamp[6].i -= a120.r;
    jamp[7].r -= a120.i; jamp[7].i += a120.r;
    jamp[9].r -= a120.i; jamp[9].i += a120.r;
    jamp[11].r += a120.i; jamp[11].i -= a120.r;
    jamp[16].r += a120.i; jamp[16].i -= a120.r;
    jamp[22].r -= a120.i; jamp[22].i += a120.r;
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
    jamp[0].r += a121.i; jamp[0].i -= a121.r;
    jamp[1].r -= a121.i; jamp[1].i += a121.r;
    jamp[3].r -= a121.i; jamp[3].i += a121.r;
    jamp[5].r += a121.i; jamp[5].i -= a121.r;
    const cx<R> a122 = ffv_amp(ub3, w173, w179);
    jamp[9].r += a122.i; jamp[9].i -= a122.r;
    jamp[11].r -= a122.i; jamp[11].i += a122.r;
    jamp[17].r -= a122.i; jamp[17].i += a122.r;
    jamp[23].r += a122.i; jamp[23].i -= a122.r;
    const R k1_180[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_181[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_182[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_182[4] = {-k15_182[0], -k15_182[1], -k15_182[2], -k15_182[3]};
    const cx<R> a123 = vvv_amp(g0, w179, jq, k1_180, k14_181, nkk15_182);
    jamp[0].r += a123.i; jamp[0].i -= a123.r;
    jamp[1].r -= a123.i; jamp[1].i += a123.r;
    jamp[3].r -= a123.i; jamp[3].i += a123.r;
    jamp[5].r += a123.i; jamp[5].i -= a123.r;
    jamp[9].r -= a123.i; jamp[9].i += a123.r;
    jamp[11].r += a123.i; jamp[11].i -= a123.r;
    jamp[17].r += a123.i; jamp[17].i -= a123.r;
    jamp[23].r -= a123.i; jamp[23].i += a123.r;
    }
    {
    const R k6_183[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const R k8_184[4] = {ldv(v.K[7][0]), ldv(v.K[7][1]), ldv(v.K[7][2]), ldv(v.K[7][3])};
    const W4<R> w185 = vvv_cur(w12, g3, k6_183, k8_184, ldv(v.iG[9]));
    const cx<R> a124 = ffv_amp(w176, v4, w185);
    jamp[0].r += a124.i; jamp[0].i -= a124.r;
    jamp[2].r -= a124.i; jamp[2].i += a124.r;
    jamp[4].r -= a124.i; jamp[4].i += a124.r;
    jamp[5].r += a124.i; jamp[5].i -= a124.r;
    const cx<R> a125 = ffv_amp(ub3, w173, w185);
    jamp[9].r += a125.i; jamp[9].i -= a125.r;
    jamp[15].r -= a125.i; jamp[15].i += a125.r;
    jamp[21].r -= a125.i; jamp[21].i += a125.r;
    jamp[23].r += a125.i; jamp[23].i -= a125.r;
    const R k1_186[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_187[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_188[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_188[4] = {-k15_188[0], -k15_188[1], -k15_188[2], -k15_188[3]};
    const cx<R> a126 = vvv_amp(g0, w185, jq, k1_186, k14_187, nkk15_188);
    jamp[0].r += a126.i; jamp[0].i -= a126.r;
    jamp[2].r -= a126.i; jamp[2].i += a126.r;
    jamp[4].r -= a126.i; jamp[4].i += a126.r;
    jamp[5].r += a126.i; jamp[5].i -= a126.r;
    jamp[9].r -= a126.i; jamp[9].i += a126.r;
    jamp[15].r += a126.i; jamp[15].i -= a126.r;
    jamp[21].r += a126.i; jamp[21].i -= a126.r;
    jamp[23].r -= a126.i; jamp[23].i += a126.r;
    }
    {
    const R k10_189[4] = {ldv(v.K[9][0]), ldv(v.K[9][1]), ldv(v.K[9][2]), ldv(v.K[9][3])};
    const R k4_190[4] = {ldv(v.K[3][0]), ldv(v.K[3][1]), ldv(v.K[3][2]), ldv(v.K[3][3])};
    const W4<R> w191 = vvv_cur(w15, g2, k10_189, k4_190, ldv(v.iG[9]));
    const cx<R> a127 = ffv_amp(w176, v4, w191);
    jamp[1].r += a127.i; jamp[1].i -= a127.r;
    jamp[2].r -= a127.i; jamp[2].i += a127.r;
    jamp[3].r += a127.i; jamp[3].i -= a127.r;
    jamp[4].r -= a127.i; jamp[4].i += a127.r;
    const cx<R> a128 = ffv_amp(ub3, w173, w191);
    jamp[11].r += a128.i; jamp[11].i -= a128.r;
    jamp[15].r -= a128.i; jamp[15].i += a128.r;
    jamp[17].r += a128.i; jamp[17].i -= a128.r;
    jamp[21].r -= a128.i; jamp[21].i += a128.r;
    const R k1_192[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_193[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_194[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_194[4] = {-k15_194[0], -k15_194[1], -k15_194[2], -k15_194[3]};
    const cx<R> a129 = vvv_amp(g0, w191, jq, k1_192, k14_193, nkk15_194);
    jamp[1].r += a129.i; jamp[1].i -= a129.r;
    jamp[2].r -= a129.i; jamp[2].i += a129.r;
    jamp[3].r += a129.i; jamp[3].i -= a129.r;
    jamp[4].r -= a129.i; jamp[4].i += a129.r;
    jamp[11].r -= a129.i; jamp[11].i += a129.r;
    jamp[15].r += a129.i; jamp[15].i -= a129.r;
    jamp[17].r -= a129.i; jamp[17].i += a129.r;
    jamp[21].r += a129.i; jamp[21].i -= a129.r;
    }
    {
    W4<R> w195, w196, w197;
    vvvv_cur(g1, g2, g3, ldv(v.iG[9]), w195, w196, w197);
    const cx<R> a130 = ffv_amp(w176, v4, w195);
    jamp[0].r += a130.i; jamp[0].i -= a130.r;
    jamp[2].r -= a130.i; jamp[2].i += a130.r;
    jamp[4].r -= a130.i; jamp[4].i += a130.r;
    jamp[5].r += a130.i; jamp[5].i -= a130.r;
    const cx<R> a131 = ffv_amp(ub3, w173, w195);
    jamp[9].r += a131.i; jamp[9].i -= a131.r;
    jamp[15].r -= a131.i; jamp[15].i += a131.r;
    jamp[21].r -= a131.i; jamp[21].i += a131.r;
    jamp[23].r += a131.i; jamp[23].i -= a131.r;
    const R k1_198[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_199[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_200[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_200[4] = {-k15_200[0], -k15_200[1], -k15_200[2], -k15_200[3]};
    const cx<R> a132 = vvv_amp(g0, w195, jq, k1_198, k14_199, nkk15_200);
    jamp[0].r += a132.i; jamp[0].i -= a132.r;
    jamp[2].r -= a132.i; jamp[2].i += a132.r;
    jamp[4].r -= a132.i; jamp[4].i += a132.r;
    jamp[5].r += a132.i; jamp[5].i -= a132.r;
    jamp[9].r -= a132.i; jamp[9].i += a132.r;
    jamp[15].r += a132.i; jamp[15].i -= a132.r;
    jamp[21].r += a132.i; jamp[21].i -= a132.r;
    jamp[23].r -= a132.i; jamp[23].i += a132.r;
    const cx<R> a133 = ffv_amp(w176, v4, w196);
    jamp[1].r += a133.i; jamp[1].i -= a133.r;
    jamp[2].r -= a133.i; jamp[2].i += a133.r;
    jamp[3].r += a133.i; jamp[3].i -= a133.r;
    jamp[4].r -= a133.i; jamp[4].i += a133.r;
    const cx<R> a134 = ffv_amp(ub3, w173, w196);
    jamp[11].r += a134.i; jamp[11].i -= a134.r;
    jamp[15].r -= a134.i; jamp[15].i += a134.r;
    jamp[17].r += a134.i; jamp[17].i -= a134.r;
    jamp[21].r -= a134.i; jamp[21].i += a134.r;
    const R k1_201[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_202[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_203[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_203[4] = {-k15_203[0], -k15_203[1], -k15_203[2], -k15_203[3]};
    const cx<R> a135 = vvv_amp(g0, w196, jq, k1_201, k14_202, nkk15_203);
    jamp[1].r += a135.i; jamp[1].i -= a135.r;
    jamp[2].r -= a135.i; jamp[2].i += a135.r;
    jamp[3].r += a135.i; jamp[3].i -= a135.r;
    jamp[4].r -= a135.i; jamp[4].i += a135.r;
    jamp[11].r -= a135.i; jamp[11].i += a135.r;
    jamp[15].r += a135.i; jamp[15].i -= a135.r;
    jamp[17].r -= a135.i; jamp[17].i += a135.r;
    jamp[21].r += a135.i; jamp[21].i -= a135.r;
    const cx<R> a136 = ffv_amp(w176, v4, w197);
    jamp[0].r -= a136.i; jamp[0].i += a136.r;
    jamp[1].r += a136.i; jamp[1].i -= a136.r;
    jamp[3].r += a136.i; jamp[3].i -= a136.r;
    jamp[5].r -= a136.i; jamp[5].i += a136.r;
    const cx<R> a137 = ffv_amp(ub3, w173, w197);
    jamp[9].r -= a137.i; jamp[9].i += a137.r;
    jamp[11].r += a137.i; jamp[11].i -= a137.r;
    jamp[17].r += a137.i; jamp[17].i -= a137.r;
    jamp[23].r -= a137.i; jamp[23].i += a137.r;
    const R k1_204[4] = {ldv(v.K[0][0]), ldv(v.K[0][1]), ldv(v.K[0][2]), ldv(v.K[0][3])};
    const R k14_205[4] = {ldv(v.K[13][0]), ldv(v.K[13][1]), ldv(v.K[13][2]), ldv(v.K[13][3])};
    const R k15_206[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_206[4] = {-k15_206[0], -k15_206[1], -k15_206[2], -k15_206[3]};
    const cx<R> a138 = vvv_amp(g0, w197, jq, k1_204, k14_205, nkk15_206);
    jamp[0].r -= a138.i; jamp[0].i += a138.r;
    jamp[1].r += a138.i; jamp[1].i -= a138.r;
    jamp[3].r += a138.i; jamp[3].i -= a138.r;
    jamp[5].r -= a138.i; jamp[5].i += a138.r;
    jamp[9].r += a138.i; jamp[9].i -= a138.r;
    jamp[11].r -= a138.i; jamp[11].i += a138.r;
    jamp[17].r -= a138.i; jamp[17].i += a138.r;
    jamp[23].r += a138.i; jamp[23].i -= a138.r;
    }
    }
    const R k3_207[4] = {ldv(v.K[2][0]), ldv(v.K[2][1]), ldv(v.K[2][2]), ldv(v.K[2][3])};
    const R k12_208[4] = {ldv(v.K[11][0]), ldv(v.K[11][1]), ldv(v.K[11][2]), ldv(v.K[11][3])};
    const R k15_209[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_209[4] = {-k15_209[0], -k15_209[1], -k15_209[2], -k15_209[3]};
    const cx<R> a139 = vvv_amp(w3, w18, jq, k3_207, k12_208, nkk15_209);
    jamp[0].r += a139.i; jamp[0].i -= a139.r;
    jamp[1].r -= a139.i; jamp[1].i += a139.r;
    jamp[6].r -= a139.i; jamp[6].i += a139.r;
    jamp[7].r += a139.i; jamp[7].i -= a139.r;
    jamp[16].r -= a139.i; jamp[16].i += a139.r;
    jamp[17].r += a139.i; jamp[17].i -= a139.r;
    jamp[22].r += a139.i; jamp[22].i -= a139.r;
    jamp[23].r -= a139.i; jamp[23].i += a139.r;
    const R k5_210[4] = {ldv(v.K[4][0]), ldv(v.K[4][1]), ldv(v.K[4][2]), ldv(v.K[4][3])};
    const R k10_211[4] = {ldv(v.K[9][0]), ldv(v.K[9][1]), ldv(v.K[9][2]), ldv(v.K[9][3])};
    const R k15_212[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_212[4] = {-k15_212[0], -k15_212[1], -k15_212[2], -k15_212[3]};
    const cx<R> a140 = vvv_amp(w6, w15, jq, k5_210, k10_211, nkk15_212);
    jamp[2].r += a140.i; jamp[2].i -= a140.r;
    jamp[3].r -= a140.i; jamp[3].i += a140.r;
    jamp[10].r -= a140.i; jamp[10].i += a140.r;
    jamp[11].r += a140.i; jamp[11].i -= a140.r;
    jamp[12].r -= a140.i; jamp[12].i += a140.r;
    jamp[13].r += a140.i; jamp[13].i -= a140.r;
    jamp[20].r += a140.i; jamp[20].i -= a140.r;
    jamp[21].r -= a140.i; jamp[21].i += a140.r;
    const R k9_213[4] = {ldv(v.K[8][0]), ldv(v.K[8][1]), ldv(v.K[8][2]), ldv(v.K[8][3])};
    const R k6_214[4] = {ldv(v.K[5][0]), ldv(v.K[5][1]), ldv(v.K[5][2]), ldv(v.K[5][3])};
    const R k15_215[4] = {ldv(v.K[14][0]), ldv(v.K[14][1]), ldv(v.K[14][2]), ldv(v.K[14][3])};
    const R nkk15_215[4] = {-k15_215[0], -k15_215[1], -k15_215[2], -k15_215[3]};
    const cx<R> a141 = vvv_amp(w9, w12, jq, k9_213, k6_214, nkk15_215);
    jamp[4].r += a141.i; jamp[4].i -= a141.r;
    jamp[5].r -= a141.i; jamp[5].i += a141.r;
    jamp[8].r -= a141.i; jamp[8].i += a141.r;
    jamp[9].r += a141.i; jamp[9].i -= a141.r;
    jamp[14].r += a141.i; jamp[14].i -= a141.r;
    jamp[15].r -= a141.i; jamp[15].i += a141.r;
    jamp[18].r -= a141.i; jamp[18].i += a141.r;
    jamp[19].r += a141.i; jamp[19].i -= a141.r;
    cx<R> a142, a143, a144;
    vvvv_amp(g0, g1, w18, jq, a142, a143, a144);
    jamp[0].r += a142.i; jamp[0].i -= a142.r;
    jamp[1].r -= a142.i; jamp[1].i += a142.r;
    jamp[6].r -= a142.i; jamp[6].i += a142.r;
    jamp[7].r += a142.i; jamp[7].i -= a142.r;
    jamp[16].r -= a142.i; jamp[16].i += a142.r;
    jamp[17].r += a142.i; jamp[17].i -= a142.r;
    jamp[22].r += a142.i; jamp[22].i -= a142.r;
    jamp[23].r -= a142.i; jamp[23].i += a142.r;
    jamp[3].r += a143.i; jamp[3].i -= a143.r;
    jamp[5].r -= a143.i; jamp[5].i += a143.r;
    jamp[6].r -= a143.i; jamp[6].i += a143.r;
    jamp[7].r += a143.i; jamp[7].i -= a143.r;
    jamp[9].r += a143.i; jamp[9].i -= a143.r;
    jamp[11].r -= a143.i; jamp[11].i += a143.r;
    jamp[16].r -= a143.i; jamp[16].i += a143.r;
    jamp[22].r += a143.i; jamp[22].i -= a143.r;
    jamp[0].r -= a144.i; jamp[0].i += a144.r;
    jamp[1].r += a144.i; jamp[1].i -= a144.r;
    jamp[3].r += a144.i; jamp[3].i -= a144.r;
    jamp[5].r -= a144.i; jamp[5].i += a144.r;
    jamp[9].r += a144.i; jamp[9].i -= a144.r;
    jamp[11].r -= a144.i; jamp[11].i += a144.r;
    jamp[17].r -= a144.i; jamp[17].i += a144.r;
    jamp[23].r += a144.i; jamp[23].i -= a144.r;
    cx<R> a145, a146, a147;
    vvvv_amp(g0, w12, g3, jq, a145, a146, a147);
    jamp[0].r += a145.i; jamp[0].i -= a145.r;
    jamp[2].r -= a145.i; jamp[2].i += a145.r;
    jamp[8].r -= a145.i; jamp[8].i += a145.r;
    jamp[14].r += a145.i; jamp[14].i -= a145.r;
    jamp[18].r -= a145.i; jamp[18].i += a145.r;
    jamp[19].r += a145.i; jamp[19].i -= a145.r;
    jamp[21].r += a145.i; jamp[21].i -= a145.r;
    jamp[23].r -= a145.i; jamp[23].i += a145.r;
    jamp[4].r += a146.i; jamp[4].i -= a146.r;
    jamp[5].r -= a146.i; jamp[5].i += a146.r;
    jamp[8].r -= a146.i; jamp[8].i += a146.r;
    jamp[9].r += a146.i; jamp[9].i -= a146.r;
    jamp[14].r += a146.i; jamp[14].i -= a146.r;
    jamp[15].r -= a146.i; jamp[15].i += a146.r;
    jamp[18].r -= a146.i; jamp[18].i += a146.r;
    jamp[19].r += a146.i; jamp[19].i -= a146.r;
    jamp[0].r -= a147.i; jamp[0].i += a147.r;
    jamp[2].r += a147.i; jamp[2].i -= a147.r;
    jamp[4].r += a147.i; jamp[4].i -= a147.r;
    jamp[5].r -= a147.i; jamp[5].i += a147.r;
    jamp[9].r += a147.i; jamp[9].i -= a147.r;
    jamp[15].r -= a147.i; jamp[15].i += a147.r;
    jamp[21].r -= a147.i; jamp[21].i += a147.r;
    jamp[23].r += a147.i; jamp[23].i -= a147.r;
    cx<R> a148, a149, a150;
    vvvv_amp(g0, w15, g2, jq, a148, a149, a150);
    jamp[1].r += a148.i; jamp[1].i -= a148.r;
    jamp[4].r -= a148.i; jamp[4].i += a148.r;
    jamp[10].r -= a148.i; jamp[10].i += a148.r;
    jamp[12].r -= a148.i; jamp[12].i += a148.r;
    jamp[13].r += a148.i; jamp[13].i -= a148.r;
    jamp[15].r += a148.i; jamp[15].i -= a148.r;
    jamp[17].r -= a148.i; jamp[17].i += a148.r;
    jamp[20].r += a148.i; jamp[20].i -= a148.r;
    jamp[2].r += a149.i; jamp[2].i -= a149.r;
    jamp[3].r -= a149.i; jamp[3].i += a149.r;
    jamp[10].r -= a149.i; jamp[10].i += a149.r;
    jamp[11].r += a149.i; jamp[11].i -= a149.r;
    jamp[12].r -= a149.i; jamp[12].i += a149.r;
    jamp[13].r += a149.i; jamp[13].i -= a149.r;
    jamp[20].r += a149.i; jamp[20].i -= a149.r;
    jamp[21].r -= a149.i; jamp[21].i += a149.r;
    jamp[1].r -= a150.i; jamp[1].i += a150.r;
    jamp[2].r += a150.i; jamp[2].i -= a150.r;
    jamp[3].r -= a150.i; jamp[3].i += a150.r;
    jamp[4].r += a150.i; jamp[4].i -= a150.r;
    jamp[11].r += a150.i; jamp[11].i -= a150.r;
    jamp[15].r -= a150.i; jamp[15].i += a150.r;
    jamp[17].r += a150.i; jamp[17].i -= a150.r;
    jamp[21].r -= a150.i; jamp[21].i += a150.r;
    cx<R> a151, a152, a153;
    vvvv_amp(w3, g2, g3, jq, a151, a152, a153);
    jamp[0].r += a151.i; jamp[0].i -= a151.r;
    jamp[6].r -= a151.i; jamp[6].i += a151.r;
    jamp[12].r -= a151.i; jamp[12].i += a151.r;
    jamp[14].r += a151.i; jamp[14].i -= a151.r;
    jamp[18].r -= a151.i; jamp[18].i += a151.r;
    jamp[20].r += a151.i; jamp[20].i -= a151.r;
    jamp[22].r += a151.i; jamp[22].i -= a151.r;
    jamp[23].r -= a151.i; jamp[23].i += a151.r;
    jamp[1].r += a152.i; jamp[1].i -= a152.r;
    jamp[7].r -= a152.i; jamp[7].i += a152.r;
    jamp[12].r -= a152.i; jamp[12].i += a152.r;
    jamp[14].r += a152.i; jamp[14].i -= a152.r;
    jamp[16].r += a152.i; jamp[16].i -= a152.r;
    jamp[17].r -= a152.i; jamp[17].i += a152.r;
    jamp[18].r -= a152.i; jamp[18].i += a152.r;
    jamp[20].r += a152.i; jamp[20].i -= a152.r;
    jamp[0].r -= a153.i; jamp[0].i += a153.r;
    jamp[1].r += a153.i; jamp[1].i -= a153.r;
    jamp[6].r += a153.i; jamp[6].i -= a153.r;
    jamp[7].r -= a153.i; jamp[7].i += a153.r;
    jamp[16].r += a153.i; jamp[16].i -= a153.r;
    jamp[17].r -= a153.i; jamp[17].i += a153.r;
    jamp[22].r -= a153.i; jamp[22].i += a153.r;
    jamp[23].r += a153.i; jamp[23].i -= a153.r;
    cx<R> a154, a155, a156;
    vvvv_amp(w6, g1, g3, jq, a154, a155, a156);
    jamp[2].r += a154.i; jamp[2].i -= a154.r;
    jamp[6].r -= a154.i; jamp[6].i += a154.r;
    jamp[8].r += a154.i; jamp[8].i -= a154.r;
    jamp[12].r -= a154.i; jamp[12].i += a154.r;
    jamp[19].r -= a154.i; jamp[19].i += a154.r;
    jamp[20].r += a154.i; jamp[20].i -= a154.r;
    jamp[21].r -= a154.i; jamp[21].i += a154.r;
    jamp[22].r += a154.i; jamp[22].i -= a154.r;
    jamp[3].r += a155.i; jamp[3].i -= a155.r;
    jamp[6].r -= a155.i; jamp[6].i += a155.r;
    jamp[8].r += a155.i; jamp[8].i -= a155.r;
    jamp[10].r += a155.i; jamp[10].i -= a155.r;
    jamp[11].r -= a155.i; jamp[11].i += a155.r;
    jamp[13].r -= a155.i; jamp[13].i += a155.r;
    jamp[19].r -= a155.i; jamp[19].i += a155.r;
    jamp[22].r += a155.i; jamp[22].i -= a155.r;
    jamp[2].r -= a156.i; jamp[2].i += a156.r;
    jamp[3].r += a156.i; jamp[3].i -= a156.r;
    jamp[10].r += a156.i; jamp[10].i -= a156.r;
    jamp[11].r -= a156.i; jamp[11].i += a156.r;
    jamp[12].r += a156.i; jamp[12].i -= a156.r;
    jamp[13].r -= a156.i; jamp[13].i += a156.r;
    jamp[20].r -= a156.i; jamp[20].i += a156.r;
    jamp[21].r += a156.i; jamp[21].i -= a156.r;
    cx<R> a157, a158, a159;
    vvvv_amp(w9, g1, g2, jq, a157, a158, a159);
    jamp[4].r += a157.i; jamp[4].i -= a157.r;
    jamp[7].r -= a157.i; jamp[7].i += a157.r;
    jamp[10].r += a157.i; jamp[10].i -= a157.r;
    jamp[13].r -= a157.i; jamp[13].i += a157.r;
    jamp[14].r += a157.i; jamp[14].i -= a157.r;
    jamp[15].r -= a157.i; jamp[15].i += a157.r;
    jamp[16].r += a157.i; jamp[16].i -= a157.r;
    jamp[18].r -= a157.i; jamp[18].i += a157.r;
    jamp[5].r += a158.i; jamp[5].i -= a158.r;
    jamp[7].r -= a158.i; jamp[7].i += a158.r;
    jamp[8].r += a158.i; jamp[8].i -= a158.r;
    jamp[9].r -= a158.i; jamp[9].i += a158.r;
    jamp[10].r += a158.i; jamp[10].i -= a158.r;
    jamp[13].r -= a158.i; jamp[13].i += a158.r;
    jamp[16].r += a158.i; jamp[16].i -= a158.r;
    jamp[19].r -= a158.i; jamp[19].i += a158.r;
    jamp[4].r -= a159.i; jamp[4].i += a159.r;
    jamp[5].r += a159.i; jamp[5].i -= a159.r;
    jamp[8].r += a159.i; jamp[8].i -= a159.r;
    jamp[9].r -= a159.i; jamp[9].i += a159.r;
    jamp[14].r -= a159.i; jamp[14].i += a159.r;
    jamp[15].r += a159.i; jamp[15].i -= a159.r;
    jamp[18].r += a159.i; jamp[18].i -= a159.r;
    jamp[19].r -= a159.i; jamp[19].i += a159.r;
    cx<R> J[NCOL];
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) J[c] = mkc(R(jamp[c].r), R(jamp[c].i));
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

template <typename R, bool SYNC>
__device__ __noinline__ double me2_gg_ttgg_impl(const double* pflat, double mt, double gs, void* slot)
{
    constexpr int NEXT = Me_gg_ttgg::NEXT, NHEL = Me_gg_ttgg::NHEL, NGLUON = Me_gg_ttgg::NGLUON;
    constexpr double COLOUR_DEN = Me_gg_ttgg::COLOUR_DEN, AVG = Me_gg_ttgg::AVG, SYM = Me_gg_ttgg::SYM;
    double p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    Me_gg_ttgg::Inv<R> local;   // used when the caller has no shared-memory slot
    Me_gg_ttgg::Inv<R>& v = slot ? *static_cast<Me_gg_ttgg::Inv<R>*>(slot) : local;
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const double kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const double kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const double kd4[4] = {-p[4][0], -p[4][1], -p[4][2], -p[4][3]};
    const double kd8[4] = {-p[5][0], -p[5][1], -p[5][2], -p[5][3]};
    const double kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    const double kd5[4] = {kd1[0] + kd4[0], kd1[1] + kd4[1], kd1[2] + kd4[2], kd1[3] + kd4[3]};
    const double kd6[4] = {kd2[0] + kd4[0], kd2[1] + kd4[1], kd2[2] + kd4[2], kd2[3] + kd4[3]};
    const double kd9[4] = {kd1[0] + kd8[0], kd1[1] + kd8[1], kd1[2] + kd8[2], kd1[3] + kd8[3]};
    const double kd10[4] = {kd2[0] + kd8[0], kd2[1] + kd8[1], kd2[2] + kd8[2], kd2[3] + kd8[3]};
    const double kd12[4] = {kd4[0] + kd8[0], kd4[1] + kd8[1], kd4[2] + kd8[2], kd4[3] + kd8[3]};
    const double kd7[4] = {kd1[0] + kd2[0] + kd4[0], kd1[1] + kd2[1] + kd4[1], kd1[2] + kd2[2] + kd4[2], kd1[3] + kd2[3] + kd4[3]};
    const double kd11[4] = {kd1[0] + kd2[0] + kd8[0], kd1[1] + kd2[1] + kd8[1], kd1[2] + kd2[2] + kd8[2], kd1[3] + kd2[3] + kd8[3]};
    const double kd13[4] = {kd1[0] + kd4[0] + kd8[0], kd1[1] + kd4[1] + kd8[1], kd1[2] + kd4[2] + kd8[2], kd1[3] + kd4[3] + kd8[3]};
    const double kd14[4] = {kd2[0] + kd4[0] + kd8[0], kd2[1] + kd4[1] + kd8[1], kd2[2] + kd4[2] + kd8[2], kd2[3] + kd4[3] + kd8[3]};
    const double kd15[4] = {kd1[0] + kd2[0] + kd4[0] + kd8[0], kd1[1] + kd2[1] + kd4[1] + kd8[1], kd1[2] + kd2[2] + kd4[2] + kd8[2], kd1[3] + kd2[3] + kd4[3] + kd8[3]};
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
    { const double q[4] = {p[2][0] - kd1[0], p[2][1] - kd1[1], p[2][2] - kd1[2], p[2][3] - kd1[3]};
      v.iQ[0] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd2[0], p[2][1] - kd2[1], p[2][2] - kd2[2], p[2][3] - kd2[3]};
      v.iQ[1] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd3[0], p[2][1] - kd3[1], p[2][2] - kd3[2], p[2][3] - kd3[3]};
      v.iQ[2] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd4[0], p[2][1] - kd4[1], p[2][2] - kd4[2], p[2][3] - kd4[3]};
      v.iQ[3] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd5[0], p[2][1] - kd5[1], p[2][2] - kd5[2], p[2][3] - kd5[3]};
      v.iQ[4] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd6[0], p[2][1] - kd6[1], p[2][2] - kd6[2], p[2][3] - kd6[3]};
      v.iQ[5] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd7[0], p[2][1] - kd7[1], p[2][2] - kd7[2], p[2][3] - kd7[3]};
      v.iQ[6] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd8[0], p[2][1] - kd8[1], p[2][2] - kd8[2], p[2][3] - kd8[3]};
      v.iQ[7] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd9[0], p[2][1] - kd9[1], p[2][2] - kd9[2], p[2][3] - kd9[3]};
      v.iQ[8] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd10[0], p[2][1] - kd10[1], p[2][2] - kd10[2], p[2][3] - kd10[3]};
      v.iQ[9] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd11[0], p[2][1] - kd11[1], p[2][2] - kd11[2], p[2][3] - kd11[3]};
      v.iQ[10] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd12[0], p[2][1] - kd12[1], p[2][2] - kd12[2], p[2][3] - kd12[3]};
      v.iQ[11] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd13[0], p[2][1] - kd13[1], p[2][2] - kd13[2], p[2][3] - kd13[3]};
      v.iQ[12] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd14[0], p[2][1] - kd14[1], p[2][2] - kd14[2], p[2][3] - kd14[3]};
      v.iQ[13] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { double a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { double a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    { double a[3], b[3]; gluon_basis(p[4], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[2][j] = R(a[j]); v.e2[2][j] = R(b[j]); } }
    { double a[3], b[3]; gluon_basis(p[5], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[3][j] = R(a[j]); v.e2[3][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
    // Parity: flipping every helicity leaves the colour-summed |M_h|^2 of these
    // tree amplitudes unchanged, so the sum over all helicities is twice the
    // sum over the configurations with the first gluon at helicity +1.
    R acc = R(0);
#pragma unroll 1
    for (int ih = 1; ih < NHEL; ih += 2) {
        acc += hel_gg_ttgg<R>(v, ih);
        if (SYNC) __syncthreads();
    }
    acc *= R(2);
    double gk = 1.0;
    for (int i = 0; i < NGLUON; ++i) gk *= gs * gs;
    return double(acc) / COLOUR_DEN * gk * AVG * SYM;
}

template <typename R, bool SYNC>
__device__ double Me_gg_ttgg::me2(const double (&p)[NEXT][4], double mt, double gs, void* slot)
{
    return me2_gg_ttgg_impl<R, SYNC>(&p[0][0], mt, gs, slot);
}
}  // namespace mf

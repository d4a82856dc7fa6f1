// Generated by paper_2105_10529_gb300/gen/qcd_diagrams.py -- do not edit.
// gg_tt: 3 Feynman diagrams (3 amplitudes with the four-gluon
// colour structures counted apart), 2 colour flows, 16 helicities.
// Wavefunction/vertex calls per helicity: {'vvv': 0, 'vvvv': 0, 'ffv_row': 0, 'ffv_col': 2, 'ffv_amp': 2, 'vvv_amp': 1, 'vvvv_amp': 0, 'ffv_cur': 1}
#pragma once
#include "mf_helas.cuh"
namespace mf {
struct Me_gg_tt {
  static constexpr int NEXT = 4;
  static constexpr int NCOL = 2;
  static constexpr int NHEL = 16;
  static constexpr int NGLUON = 2;
  static constexpr int NDIAG = 3;
  static constexpr double COLOUR_DEN = 3.0;
  static constexpr double AVG = 1.0 / 256.0;
  static constexpr double SYM = 1.0;
  // helicity-independent per-event pieces
  template <typename R> struct Inv {
    R kr[2][4]; R p3r[4]; R iG[1]; R iQ[2];
    R e1[2][3]; R e2[2][3]; FermionBasis<R> fb3, fb4; R mt;
  };
  // averaged |M|^2 (spin/colour average and identical-particle factor included);
  // p: momenta (E,px,py,pz) incoming first: g, g, t, tbar, g...
  template <typename R>
  __device__ static double me2(const double (&p)[NEXT][4], double mt, double gs);
};

// one helicity configuration: amplitudes, colour flows and the colour sum;
// out of line so that its register allocation sees only one helicity
template <typename R>
__device__ __noinline__ R hel_gg_tt(const Me_gg_tt::Inv<R>& v, int ih)
{
    constexpr int NCOL = Me_gg_tt::NCOL;
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
    cx<R> jamp[NCOL];
    #pragma unroll
    for (int c = 0; c < NCOL; ++c) jamp[c] = mkc(R(0), R(0));
    const W4<R> g0 = ext_gluon(v.e1[0], v.e2[0], HEL(0), false);
    const W4<R> g1 = ext_gluon(v.e1[1], v.e2[1], HEL(1), false);
    const W4<R> ub3 = ext_ubar(v.fb3, HEL(2));
    const W4<R> v4 = ext_v(v.fb4, HEL(3));
    const R q1_2[4] = {v.p3r[0] - (v.kr[0][0]), v.p3r[1] - (v.kr[0][1]), v.p3r[2] - (v.kr[0][2]), v.p3r[3] - (v.kr[0][3])};
    const W4<R> w1 = ffv_col(g1, v4, q1_2, v.mt, v.iQ[0]);
    const cx<R> a1 = ffv_amp(ub3, w1, g0);
    jamp[0].r += a1.i; jamp[0].i -= a1.r;
    const R q2_4[4] = {v.p3r[0] - (v.kr[1][0]), v.p3r[1] - (v.kr[1][1]), v.p3r[2] - (v.kr[1][2]), v.p3r[3] - (v.kr[1][3])};
    const W4<R> w3 = ffv_col(g0, v4, q2_4, v.mt, v.iQ[1]);
    const cx<R> a2 = ffv_amp(ub3, w3, g1);
    jamp[1].r += a2.i; jamp[1].i -= a2.r;
    const W4<R> jq = ffv_cur(ub3, v4, v.iG[0]);
    const R k1_5[4] = {v.kr[0][0], v.kr[0][1], v.kr[0][2], v.kr[0][3]};
    const R k2_6[4] = {v.kr[1][0], v.kr[1][1], v.kr[1][2], v.kr[1][3]};
    const R k3_7[4] = {v.kr[0][0] + v.kr[1][0], v.kr[0][1] + v.kr[1][1], v.kr[0][2] + v.kr[1][2], v.kr[0][3] + v.kr[1][3]};
    const R nkk3_7[4] = {-k3_7[0], -k3_7[1], -k3_7[2], -k3_7[3]};
    const cx<R> a3 = vvv_amp(g0, g1, jq, k1_5, k2_6, nkk3_7);
    jamp[0].r += a3.i; jamp[0].i -= a3.r;
    jamp[1].r -= a3.i; jamp[1].i += a3.r;
    R me = R(0);
    { const R zr = R(16.0) * jamp[0].r + R(-4.0) * jamp[1].r; const R zi = R(16.0) * jamp[0].i + R(-4.0) * jamp[1].i;
      me = fma(jamp[0].r, zr, fma(jamp[0].i, zi, me)); }
    { const R zr = R(16.0) * jamp[1].r; const R zi = R(16.0) * jamp[1].i;
      me = fma(jamp[1].r, zr, fma(jamp[1].i, zi, me)); }
    return me;
#undef HEL
}

template <typename R>
__device__ __noinline__ double me2_gg_tt_impl(const double* pflat, double mt, double gs)
{
    constexpr int NEXT = Me_gg_tt::NEXT, NHEL = Me_gg_tt::NHEL, NGLUON = Me_gg_tt::NGLUON;
    constexpr double COLOUR_DEN = Me_gg_tt::COLOUR_DEN, AVG = Me_gg_tt::AVG, SYM = Me_gg_tt::SYM;
    double p[NEXT][4];
    for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];
    Me_gg_tt::Inv<R> v;
    // gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing
    const double kd1[4] = {p[0][0], p[0][1], p[0][2], p[0][3]};
    const double kd2[4] = {p[1][0], p[1][1], p[1][2], p[1][3]};
    const double kd3[4] = {kd1[0] + kd2[0], kd1[1] + kd2[1], kd1[2] + kd2[2], kd1[3] + kd2[3]};
    for (int c = 0; c < 4; ++c) v.kr[0][c] = R(kd1[c]);
    for (int c = 0; c < 4; ++c) v.kr[1][c] = R(kd2[c]);
    for (int c = 0; c < 4; ++c) v.p3r[c] = R(p[2][c]);
    v.iG[0] = R(1.0 / mdot(kd3, kd3));
    { const double q[4] = {p[2][0] - kd1[0], p[2][1] - kd1[1], p[2][2] - kd1[2], p[2][3] - kd1[3]};
      v.iQ[0] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { const double q[4] = {p[2][0] - kd2[0], p[2][1] - kd2[1], p[2][2] - kd2[2], p[2][3] - kd2[3]};
      v.iQ[1] = R(1.0 / (mdot(q, q) - mt * mt)); }
    { double a[3], b[3]; gluon_basis(p[0], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[0][j] = R(a[j]); v.e2[0][j] = R(b[j]); } }
    { double a[3], b[3]; gluon_basis(p[1], a, b);
      for (int j = 0; j < 3; ++j) { v.e1[1][j] = R(a[j]); v.e2[1][j] = R(b[j]); } }
    v.fb3 = fermion_basis<R>(p[2], mt);
    v.fb4 = fermion_basis<R>(p[3], mt);
    v.mt = R(mt);
    R acc = R(0);
#pragma unroll 1
    for (int ih = 0; ih < NHEL; ++ih) acc += hel_gg_tt<R>(v, ih);
    double gk = 1.0;
    for (int i = 0; i < NGLUON; ++i) gk *= gs * gs;
    return double(acc) / COLOUR_DEN * gk * AVG * SYM;
}

template <typename R>
__device__ double Me_gg_tt::me2(const double (&p)[NEXT][4], double mt, double gs)
{
    return me2_gg_tt_impl<R>(&p[0][0], mt, gs);
}
}  // namespace mf

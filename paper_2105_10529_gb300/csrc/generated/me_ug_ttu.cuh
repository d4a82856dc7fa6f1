// Generated by paper_2105_10529_gb300/gen/qq_processes.py -- do not edit.
#pragma once
#include "mf_helas.cuh"
namespace mf {
// u g -> t tbar u: 5 diagrams, diagram colour basis, 32 helicities, 16 allowed
struct Me_ug_ttu {
  static constexpr int NEXT = 5;
  static constexpr int NHEL = 32;
  static constexpr int NHEL_NZ = 16;   // configurations allowed by helicity conservation
  __host__ __device__ static constexpr int hel_nz(int j) { return (j & 15) | ((j & 1) << 4); }
  static constexpr int NGS = 3;   // powers of g in the amplitude
  static constexpr double AVG = 1.0 / 96.0;
  static constexpr bool TC_COLOUR = false;
  template <typename R> struct Inv { float unused; };
  template <typename R> static constexpr size_t slot_bytes() { return 0; }
  // averaged |M|^2 (S, the scalar of the momenta, carries them and the result: the FP64
  // scalar Widen<R>::type, or Df where the mixed-precision kinematics hand theirs on)
  template <typename R, bool SYNC = false, bool TC = false, typename S = typename Widen<R>::type>
  __device__ static S me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt, typename NoDeduce<S>::type gs,
                         void*, void* = nullptr, int = 0, int = 1)
  {
    // momenta of the internal lines
    const S qtt[4] = {p[2][0] + p[3][0], p[2][1] + p[3][1], p[2][2] + p[3][2], p[2][3] + p[3][3]};
    const S qu[4] = {p[0][0] - p[4][0], p[0][1] - p[4][1], p[0][2] - p[4][2], p[0][3] - p[4][3]};
    const S q1[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};
    const S q2[4] = {p[4][0] - p[1][0], p[4][1] - p[1][1], p[4][2] - p[1][2], p[4][3] - p[1][3]};
    const S q3[4] = {p[2][0] - p[1][0], p[2][1] - p[1][1], p[2][2] - p[1][2], p[2][3] - p[1][3]};
    const S q4[4] = {p[2][0] - qu[0], p[2][1] - qu[1], p[2][2] - qu[2], p[2][3] - qu[3]};
    const R iGtt = R(1.0 / mdot(qtt, qtt)), iGu = R(1.0 / mdot(qu, qu));
    const R iQ1 = R(1.0 / mdot(q1, q1)), iQ2 = R(1.0 / mdot(q2, q2));
    const R iQ3 = R(1.0 / (mdot(q3, q3) - mt * mt)), iQ4 = R(1.0 / (mdot(q4, q4) - mt * mt));
    const R Q1[4] = {R(q1[0]), R(q1[1]), R(q1[2]), R(q1[3])}, Q2[4] = {R(q2[0]), R(q2[1]), R(q2[2]), R(q2[3])};
    const R Q3[4] = {R(q3[0]), R(q3[1]), R(q3[2]), R(q3[3])}, Q4[4] = {R(q4[0]), R(q4[1]), R(q4[2]), R(q4[3])};
    const R KA[4] = {R(qu[0]), R(qu[1]), R(qu[2]), R(qu[3])};
    const R KB[4] = {R(p[1][0]), R(p[1][1]), R(p[1][2]), R(p[1][3])};
    const R KC[4] = {R(-qtt[0]), R(-qtt[1]), R(-qtt[2]), R(-qtt[3])};
    const R mtr = R(mt);
    R e1[3], e2[3];
    { S a[3], b[3]; gluon_basis(p[1], a, b); for (int j = 0; j < 3; ++j) { e1[j] = R(a[j]); e2[j] = R(b[j]); } }
    const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f5 = fermion_basis<R>(p[4], S(0.0));
    const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);
    R acc = R(0);
    // helicity filtering: only the configurations helicity conservation allows
#pragma unroll 1
    for (int jh = 0; jh < NHEL_NZ; ++jh) {
      const int ih = hel_nz(jh);
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
      const W4<R> u1 = ext_u(f1, HEL(0));
      const W4<R> g2 = ext_gluon(e1, e2, HEL(1), false);
      const W4<R> ub3 = ext_ubar(f3, HEL(2));
      const W4<R> v4 = ext_v(f4, HEL(3));
      const W4<R> ub5 = ext_ubar(f5, HEL(4));
      const W4<R> jt = ffv_cur(ub3, v4, iGtt);      // t tbar current into the u line
      const W4<R> ju = ffv_cur(ub5, u1, iGu);       // u-line current into the t line
      const cx<R> a1 = ffv_amp(ub5, ffv_col(g2, u1, Q1, R(0), iQ1), jt);
      const cx<R> a2 = ffv_amp(ffv_row(ub5, g2, Q2, R(0), iQ2), u1, jt);
      const cx<R> a3 = ffv_amp(ffv_row(ub3, g2, Q3, mtr, iQ3), v4, ju);
      const cx<R> a4 = ffv_amp(ub3, ffv_col(g2, v4, Q4, mtr, iQ4), ju);
      const cx<R> a5 = vvv_amp(ju, g2, jt, KA, KB, KC);
      R me = R(0);
      me += R(2.6666666666666665) * (a1.r * a1.r + a1.i * a1.i);
      me += R(-0.3333333333333333) * (a1.r * a2.r + a1.i * a2.i);
      me += R(2.3333333333333335) * (a1.r * a3.r + a1.i * a3.i);
      me += R(-0.6666666666666666) * (a1.r * a4.r + a1.i * a4.i);
      me += R(-3.0) * (a1.r * a5.r + a1.i * a5.i);
      me += R(-0.3333333333333333) * (a2.r * a1.r + a2.i * a1.i);
      me += R(2.6666666666666665) * (a2.r * a2.r + a2.i * a2.i);
      me += R(-0.6666666666666666) * (a2.r * a3.r + a2.i * a3.i);
      me += R(2.3333333333333335) * (a2.r * a4.r + a2.i * a4.i);
      me += R(3.0) * (a2.r * a5.r + a2.i * a5.i);
      me += R(2.3333333333333335) * (a3.r * a1.r + a3.i * a1.i);
      me += R(-0.6666666666666666) * (a3.r * a2.r + a3.i * a2.i);
      me += R(2.6666666666666665) * (a3.r * a3.r + a3.i * a3.i);
      me += R(-0.3333333333333333) * (a3.r * a4.r + a3.i * a4.i);
      me += R(-3.0) * (a3.r * a5.r + a3.i * a5.i);
      me += R(-0.6666666666666666) * (a4.r * a1.r + a4.i * a1.i);
      me += R(2.3333333333333335) * (a4.r * a2.r + a4.i * a2.i);
      me += R(-0.3333333333333333) * (a4.r * a3.r + a4.i * a3.i);
      me += R(2.6666666666666665) * (a4.r * a4.r + a4.i * a4.i);
      me += R(3.0) * (a4.r * a5.r + a4.i * a5.i);
      me += R(-3.0) * (a5.r * a1.r + a5.i * a1.i);
      me += R(3.0) * (a5.r * a2.r + a5.i * a2.i);
      me += R(-3.0) * (a5.r * a3.r + a5.i * a3.i);
      me += R(3.0) * (a5.r * a4.r + a5.i * a4.i);
      me += R(6.0) * (a5.r * a5.r + a5.i * a5.i);
      acc += me;
#undef HEL
    }
    S gk = S(1.0);
    for (int i = 0; i < NGS; ++i) gk = gk * gs;
    return S(acc) * gk * gk * AVG;
  }
  // Helicity profile: the averaged |M_h|^2 of every configuration ih (bit i: helicity of
  // external particle i, set = +1), the filtered ones included (they come out zero)
  template <typename R>
  __device__ static void hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,
                                     typename Widen<R>::type gs, double* out)
  {
    using S = typename Widen<R>::type;
    // momenta of the internal lines
    const S qtt[4] = {p[2][0] + p[3][0], p[2][1] + p[3][1], p[2][2] + p[3][2], p[2][3] + p[3][3]};
    const S qu[4] = {p[0][0] - p[4][0], p[0][1] - p[4][1], p[0][2] - p[4][2], p[0][3] - p[4][3]};
    const S q1[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};
    const S q2[4] = {p[4][0] - p[1][0], p[4][1] - p[1][1], p[4][2] - p[1][2], p[4][3] - p[1][3]};
    const S q3[4] = {p[2][0] - p[1][0], p[2][1] - p[1][1], p[2][2] - p[1][2], p[2][3] - p[1][3]};
    const S q4[4] = {p[2][0] - qu[0], p[2][1] - qu[1], p[2][2] - qu[2], p[2][3] - qu[3]};
    const R iGtt = R(1.0 / mdot(qtt, qtt)), iGu = R(1.0 / mdot(qu, qu));
    const R iQ1 = R(1.0 / mdot(q1, q1)), iQ2 = R(1.0 / mdot(q2, q2));
    const R iQ3 = R(1.0 / (mdot(q3, q3) - mt * mt)), iQ4 = R(1.0 / (mdot(q4, q4) - mt * mt));
    const R Q1[4] = {R(q1[0]), R(q1[1]), R(q1[2]), R(q1[3])}, Q2[4] = {R(q2[0]), R(q2[1]), R(q2[2]), R(q2[3])};
    const R Q3[4] = {R(q3[0]), R(q3[1]), R(q3[2]), R(q3[3])}, Q4[4] = {R(q4[0]), R(q4[1]), R(q4[2]), R(q4[3])};
    const R KA[4] = {R(qu[0]), R(qu[1]), R(qu[2]), R(qu[3])};
    const R KB[4] = {R(p[1][0]), R(p[1][1]), R(p[1][2]), R(p[1][3])};
    const R KC[4] = {R(-qtt[0]), R(-qtt[1]), R(-qtt[2]), R(-qtt[3])};
    const R mtr = R(mt);
    R e1[3], e2[3];
    { S a[3], b[3]; gluon_basis(p[1], a, b); for (int j = 0; j < 3; ++j) { e1[j] = R(a[j]); e2[j] = R(b[j]); } }
    const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f5 = fermion_basis<R>(p[4], S(0.0));
    const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);
    S gk = S(1.0);
    for (int i = 0; i < NGS; ++i) gk = gk * gs;
    for (int ih = 0; ih < NHEL; ++ih) {
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
      const W4<R> u1 = ext_u(f1, HEL(0));
      const W4<R> g2 = ext_gluon(e1, e2, HEL(1), false);
      const W4<R> ub3 = ext_ubar(f3, HEL(2));
      const W4<R> v4 = ext_v(f4, HEL(3));
      const W4<R> ub5 = ext_ubar(f5, HEL(4));
      const W4<R> jt = ffv_cur(ub3, v4, iGtt);      // t tbar current into the u line
      const W4<R> ju = ffv_cur(ub5, u1, iGu);       // u-line current into the t line
      const cx<R> a1 = ffv_amp(ub5, ffv_col(g2, u1, Q1, R(0), iQ1), jt);
      const cx<R> a2 = ffv_amp(ffv_row(ub5, g2, Q2, R(0), iQ2), u1, jt);
      const cx<R> a3 = ffv_amp(ffv_row(ub3, g2, Q3, mtr, iQ3), v4, ju);
      const cx<R> a4 = ffv_amp(ub3, ffv_col(g2, v4, Q4, mtr, iQ4), ju);
      const cx<R> a5 = vvv_amp(ju, g2, jt, KA, KB, KC);
      R me = R(0);
      me += R(2.6666666666666665) * (a1.r * a1.r + a1.i * a1.i);
      me += R(-0.3333333333333333) * (a1.r * a2.r + a1.i * a2.i);
      me += R(2.3333333333333335) * (a1.r * a3.r + a1.i * a3.i);
      me += R(-0.6666666666666666) * (a1.r * a4.r + a1.i * a4.i);
      me += R(-3.0) * (a1.r * a5.r + a1.i * a5.i);
      me += R(-0.3333333333333333) * (a2.r * a1.r + a2.i * a1.i);
      me += R(2.6666666666666665) * (a2.r * a2.r + a2.i * a2.i);
      me += R(-0.6666666666666666) * (a2.r * a3.r + a2.i * a3.i);
      me += R(2.3333333333333335) * (a2.r * a4.r + a2.i * a4.i);
      me += R(3.0) * (a2.r * a5.r + a2.i * a5.i);
      me += R(2.3333333333333335) * (a3.r * a1.r + a3.i * a1.i);
      me += R(-0.6666666666666666) * (a3.r * a2.r + a3.i * a2.i);
      me += R(2.6666666666666665) * (a3.r * a3.r + a3.i * a3.i);
      me += R(-0.3333333333333333) * (a3.r * a4.r + a3.i * a4.i);
      me += R(-3.0) * (a3.r * a5.r + a3.i * a5.i);
      me += R(-0.6666666666666666) * (a4.r * a1.r + a4.i * a1.i);
      me += R(2.3333333333333335) * (a4.r * a2.r + a4.i * a2.i);
      me += R(-0.3333333333333333) * (a4.r * a3.r + a4.i * a3.i);
      me += R(2.6666666666666665) * (a4.r * a4.r + a4.i * a4.i);
      me += R(3.0) * (a4.r * a5.r + a4.i * a5.i);
      me += R(-3.0) * (a5.r * a1.r + a5.i * a1.i);
      me += R(3.0) * (a5.r * a2.r + a5.i * a2.i);
      me += R(-3.0) * (a5.r * a3.r + a5.i * a3.i);
      me += R(3.0) * (a5.r * a4.r + a5.i * a4.i);
      me += R(6.0) * (a5.r * a5.r + a5.i * a5.i);
      out[ih] = val(S(me) * gk * gk * AVG);
#undef HEL
    }
  }
};
}  // namespace mf

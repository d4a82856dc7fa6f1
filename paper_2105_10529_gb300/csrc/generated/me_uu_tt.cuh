// Generated by paper_2105_10529_gb300/gen/qq_processes.py -- do not edit.
#pragma once
#include "mf_helas.cuh"
namespace mf {
// u ubar -> t tbar: 1 diagram, colour factor (T^c)(T^c), 16 helicities, 8 allowed
struct Me_uu_tt {
  static constexpr int NEXT = 4;
  static constexpr int NHEL = 16;
  static constexpr int NHEL_NZ = 8;   // configurations allowed by helicity conservation
  __host__ __device__ static constexpr int hel_nz(int j) { return (j & 1) | ((~j & 1) << 1) | ((j >> 1) << 2); }
  static constexpr int NGS = 2;   // powers of g in the amplitude
  static constexpr double AVG = 1.0 / 36.0;
  static constexpr bool TC_COLOUR = false;
  template <typename R> struct Inv { float unused; };
  template <typename R> static constexpr size_t slot_bytes() { return 0; }
  // averaged |M|^2 (S, the scalar of the momenta, carries them and the result: the FP64
  // scalar Widen<R>::type, or Df where the mixed-precision kinematics hand theirs on)
  template <typename R, bool SYNC = false, bool TC = false, typename S = typename Widen<R>::type>
  __device__ static S me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt, typename NoDeduce<S>::type gs,
                         void*, void* = nullptr, int = 0, int = 1)
  {
    const S q[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};
    const R iS = R(1.0 / mdot(q, q));
    const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f2 = fermion_basis<R>(p[1], S(0.0));
    const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);
    R acc = R(0);
    // helicity filtering: only the configurations helicity conservation allows
#pragma unroll 1
    for (int jh = 0; jh < NHEL_NZ; ++jh) {
      const int ih = hel_nz(jh);
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
      // vbar(p2) gamma u(p1) through the s-channel gluon into ubar(p3) gamma v(p4)
      const W4<R> ju = ffv_cur(ext_vbar(f2, HEL(1)), ext_u(f1, HEL(0)), iS);
      const cx<R> a1 = ffv_amp(ext_ubar(f3, HEL(2)), ext_v(f4, HEL(3)), ju);
      R me = R(0);
      me += R(2.0) * (a1.r * a1.r + a1.i * a1.i);
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
    const S q[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};
    const R iS = R(1.0 / mdot(q, q));
    const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f2 = fermion_basis<R>(p[1], S(0.0));
    const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);
    S gk = S(1.0);
    for (int i = 0; i < NGS; ++i) gk = gk * gs;
    for (int ih = 0; ih < NHEL; ++ih) {
#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)
      // vbar(p2) gamma u(p1) through the s-channel gluon into ubar(p3) gamma v(p4)
      const W4<R> ju = ffv_cur(ext_vbar(f2, HEL(1)), ext_u(f1, HEL(0)), iS);
      const cx<R> a1 = ffv_amp(ext_ubar(f3, HEL(2)), ext_v(f4, HEL(3)), ju);
      R me = R(0);
      me += R(2.0) * (a1.r * a1.r + a1.i * a1.i);
      out[ih] = val(S(me) * gk * gk * AVG);
#undef HEL
    }
  }
};
}  // namespace mf

"""Matrix elements with two quark lines: u ubar -> t tbar and u g -> t tbar u
(the light-quark channels of the batched p p -> t tbar + jets set).

Written from the same Feynman rules as qcd_diagrams.py (quark-gluon vertex
i g gamma^mu T^a, quark propagator i (qslash + m)/(q^2 - m^2), gluon
propagator -i g/k^2, three-gluon vertex g f^{abc} V), with the HELAS-style
routines of mf_helas.cuh.  The colour factors are kept per diagram (a
non-orthogonal basis); the colour matrix sum over all indices of
conj(X_D) X_D' comes from the Fierz identity (colour.py), with each
diagram's phase (product of the factors of i) folded into it.

u ubar -> t tbar: one s-channel gluon diagram.
u(p1) g(p2) -> t(p3) tbar(p4) u(p5): five diagrams,
  D1 the gluon absorbed on the u line before the t tbar gluon is emitted,
  D2 after it, D3 / D4 the gluon on the t / tbar side of the heavy line,
  D5 through the three-gluon vertex.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import List, Tuple

from . import colour as col

I = 1j


def _colour_matrix_ug_ttu():
    """Diagram colour factors with labels i1 (u in), a (gluon), i3 (t), j4 (tbar), i5 (u out)."""
    X = [
        [(1, [(("c", "a"), "i5", "i1"), (("c",), "i3", "j4")])],
        [(1, [(("a", "c"), "i5", "i1"), (("c",), "i3", "j4")])],
        [(1, [(("c",), "i5", "i1"), (("a", "c"), "i3", "j4")])],
        [(1, [(("c",), "i5", "i1"), (("c", "a"), "i3", "j4")])],
        # f^{cad} = -2i (Tr(T^c T^a T^d) - Tr(T^a T^c T^d))
        [(-2j, [(("c", "a", "d"), "x", "x"), (("c",), "i5", "i1"), (("d",), "i3", "j4")]),
         (2j, [(("a", "c", "d"), "y", "y"), (("c",), "i5", "i1"), (("d",), "i3", "j4")])],
    ]
    return col.colour_matrix(X, {"i1", "i3", "j4", "i5"}, {"a"})


def _colour_matrix_uu_tt():
    X = [[(1, [(("c",), "i3", "j4"), (("c",), "j2", "i1")])]]
    return col.colour_matrix(X, {"i1", "j2", "i3", "j4"}, set())


def _fold_phases(Cm, phases):
    n = len(Cm)
    return [[phases[x].conjugate() * Cm[x][y] * phases[y] for y in range(n)] for x in range(n)]


def _emit_colour_sum(C, amps: List[str]) -> List[str]:
    """|M|^2 = sum_xy Re(conj(L_x) C_xy L_y) for Hermitian C."""
    out = ["R me = R(0);"]
    n = len(amps)
    for x in range(n):
        for y in range(n):
            c = complex(C[x][y])
            if abs(c) < 1e-14:
                continue
            # Re(conj(Lx) c Ly) = Re(c) Re(conj(Lx) Ly) - Im(c) Im(conj(Lx) Ly)
            rr = f"({amps[x]}.r * {amps[y]}.r + {amps[x]}.i * {amps[y]}.i)"
            ii = f"({amps[x]}.r * {amps[y]}.i - {amps[x]}.i * {amps[y]}.r)"
            terms = []
            if abs(c.real) > 1e-14:
                terms.append(f"R({c.real!r}) * {rr}")
            if abs(c.imag) > 1e-14:
                terms.append(f"R({-c.imag!r}) * {ii}")
            out.append(f"me += {' + '.join(terms)};")
    return out


HEADER = '''// Generated by paper_2105_10529_gb300/gen/qq_processes.py -- do not edit.
#pragma once
#include "mf_helas.cuh"
namespace mf {
'''


def _struct(name: str, n_ext: int, n_hel: int, avg: str, k: int, prologue: List[str], body: List[str],
            csum: List[str], comment: str, hel_map: str, n_hel_nz: int) -> str:
    """hel_map: C expression of the j-th helicity configuration (0 <= j < n_hel_nz) that helicity
    conservation on the massless quark lines allows; the others vanish identically (exactly, with
    the massless spinors' zero components) and are skipped."""
    s = [f"// {comment}"]
    s.append(f"struct Me_{name} {{")
    s.append(f"  static constexpr int NEXT = {n_ext};")
    s.append(f"  static constexpr int NHEL = {n_hel};")
    s.append(f"  static constexpr int NHEL_NZ = {n_hel_nz};   // configurations allowed by helicity conservation")
    s.append(f"  __host__ __device__ static constexpr int hel_nz(int j) {{ return {hel_map}; }}")
    s.append(f"  static constexpr int NGS = {k};   // powers of g in the amplitude")
    s.append(f"  static constexpr double AVG = {avg};")
    s.append("  static constexpr bool TC_COLOUR = false;")
    s.append("  template <typename R> struct Inv { float unused; };")
    s.append("  template <typename R> static constexpr size_t slot_bytes() { return 0; }")
    s.append("  // averaged |M|^2 (S, the scalar of the momenta, carries them and the result: the FP64")
    s.append("  // scalar Widen<R>::type, or Df where the mixed-precision kinematics hand theirs on)")
    s.append("  template <typename R, bool SYNC = false, bool TC = false, typename S = typename Widen<R>::type>")
    s.append("  __device__ static S me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt, typename NoDeduce<S>::type gs,")
    s.append("                         void*, void* = nullptr, int = 0, int = 1)")
    s.append("  {")
    for l in prologue:
        s.append("    " + l)
    s.append("    R acc = R(0);")
    s.append("    // helicity filtering: only the configurations helicity conservation allows")
    s.append("#pragma unroll 1")
    s.append("    for (int jh = 0; jh < NHEL_NZ; ++jh) {")
    s.append("      const int ih = hel_nz(jh);")
    s.append("#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)")
    for l in body + csum:
        s.append("      " + l)
    s.append("      acc += me;")
    s.append("#undef HEL")
    s.append("    }")
    s.append("    S gk = S(1.0);")
    s.append("    for (int i = 0; i < NGS; ++i) gk = gk * gs;")
    s.append("    return S(acc) * gk * gk * AVG;")
    s.append("  }")
    s.append("  // Helicity profile: the averaged |M_h|^2 of every configuration ih (bit i: helicity of")
    s.append("  // external particle i, set = +1), the filtered ones included (they come out zero)")
    s.append("  template <typename R>")
    s.append("  __device__ static void hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,")
    s.append("                                     typename Widen<R>::type gs, double* out)")
    s.append("  {")
    s.append("    using S = typename Widen<R>::type;")
    for l in prologue:
        s.append("    " + l)
    s.append("    S gk = S(1.0);")
    s.append("    for (int i = 0; i < NGS; ++i) gk = gk * gs;")
    s.append("    for (int ih = 0; ih < NHEL; ++ih) {")
    s.append("#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)")
    for l in body + csum:
        s.append("      " + l)
    s.append("      out[ih] = val(S(me) * gk * gk * AVG);")
    s.append("#undef HEL")
    s.append("    }")
    s.append("  }")
    s.append("};")
    return "\n".join(s) + "\n"


def generate_uu_tt() -> Tuple[str, dict]:
    Cm = _colour_matrix_uu_tt()
    pro = [
        "const S q[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};",
        "const R iS = R(1.0 / mdot(q, q));",
        "const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f2 = fermion_basis<R>(p[1], S(0.0));",
        "const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);",
    ]
    body = [
        "// vbar(p2) gamma u(p1) through the s-channel gluon into ubar(p3) gamma v(p4)",
        "const W4<R> ju = ffv_cur(ext_vbar(f2, HEL(1)), ext_u(f1, HEL(0)), iS);",
        "const cx<R> a1 = ffv_amp(ext_ubar(f3, HEL(2)), ext_v(f4, HEL(3)), ju);",
    ]
    csum = _emit_colour_sum(Cm, ["a1"])
    # the massless u and ubar annihilate into a vector current only with opposite helicity bits
    # (u(+) is right-handed and pairs with vbar(-)): bit 1 = not bit 0
    hel_map = "(j & 1) | ((~j & 1) << 1) | ((j >> 1) << 2)"
    src = HEADER + _struct("uu_tt", 4, 16, "1.0 / 36.0", 2, pro, body, csum,
                           "u ubar -> t tbar: 1 diagram, colour factor (T^c)(T^c), 16 helicities, 8 allowed",
                           hel_map, 8) + "}  // namespace mf\n"
    return src, dict(n_diag=1, colour=Cm)


def generate_ug_ttu() -> Tuple[str, dict]:
    Cm = _colour_matrix_ug_ttu()
    # phases of the diagrams with the couplings g^3 taken out: fermion-line
    # diagrams (i g)^3 i (-i) = -i; the three-gluon diagram (i g)^2 g (-i)^2 = +1
    ph = [-1j, -1j, -1j, -1j, 1.0 + 0j]
    C = _fold_phases(Cm, ph)
    pro = [
        "// momenta of the internal lines",
        "const S qtt[4] = {p[2][0] + p[3][0], p[2][1] + p[3][1], p[2][2] + p[3][2], p[2][3] + p[3][3]};",
        "const S qu[4] = {p[0][0] - p[4][0], p[0][1] - p[4][1], p[0][2] - p[4][2], p[0][3] - p[4][3]};",
        "const S q1[4] = {p[0][0] + p[1][0], p[0][1] + p[1][1], p[0][2] + p[1][2], p[0][3] + p[1][3]};",
        "const S q2[4] = {p[4][0] - p[1][0], p[4][1] - p[1][1], p[4][2] - p[1][2], p[4][3] - p[1][3]};",
        "const S q3[4] = {p[2][0] - p[1][0], p[2][1] - p[1][1], p[2][2] - p[1][2], p[2][3] - p[1][3]};",
        "const S q4[4] = {p[2][0] - qu[0], p[2][1] - qu[1], p[2][2] - qu[2], p[2][3] - qu[3]};",
        "const R iGtt = R(1.0 / mdot(qtt, qtt)), iGu = R(1.0 / mdot(qu, qu));",
        "const R iQ1 = R(1.0 / mdot(q1, q1)), iQ2 = R(1.0 / mdot(q2, q2));",
        "const R iQ3 = R(1.0 / (mdot(q3, q3) - mt * mt)), iQ4 = R(1.0 / (mdot(q4, q4) - mt * mt));",
        "const R Q1[4] = {R(q1[0]), R(q1[1]), R(q1[2]), R(q1[3])}, Q2[4] = {R(q2[0]), R(q2[1]), R(q2[2]), R(q2[3])};",
        "const R Q3[4] = {R(q3[0]), R(q3[1]), R(q3[2]), R(q3[3])}, Q4[4] = {R(q4[0]), R(q4[1]), R(q4[2]), R(q4[3])};",
        "const R KA[4] = {R(qu[0]), R(qu[1]), R(qu[2]), R(qu[3])};",
        "const R KB[4] = {R(p[1][0]), R(p[1][1]), R(p[1][2]), R(p[1][3])};",
        "const R KC[4] = {R(-qtt[0]), R(-qtt[1]), R(-qtt[2]), R(-qtt[3])};",
        "const R mtr = R(mt);",
        "R e1[3], e2[3];",
        "{ S a[3], b[3]; gluon_basis(p[1], a, b); for (int j = 0; j < 3; ++j) { e1[j] = R(a[j]); e2[j] = R(b[j]); } }",
        "const FermionBasis<R> f1 = fermion_basis<R>(p[0], S(0.0)), f5 = fermion_basis<R>(p[4], S(0.0));",
        "const FermionBasis<R> f3 = fermion_basis<R>(p[2], mt), f4 = fermion_basis<R>(p[3], mt);",
    ]
    body = [
        "const W4<R> u1 = ext_u(f1, HEL(0));",
        "const W4<R> g2 = ext_gluon(e1, e2, HEL(1), false);",
        "const W4<R> ub3 = ext_ubar(f3, HEL(2));",
        "const W4<R> v4 = ext_v(f4, HEL(3));",
        "const W4<R> ub5 = ext_ubar(f5, HEL(4));",
        "const W4<R> jt = ffv_cur(ub3, v4, iGtt);      // t tbar current into the u line",
        "const W4<R> ju = ffv_cur(ub5, u1, iGu);       // u-line current into the t line",
        "const cx<R> a1 = ffv_amp(ub5, ffv_col(g2, u1, Q1, R(0), iQ1), jt);",
        "const cx<R> a2 = ffv_amp(ffv_row(ub5, g2, Q2, R(0), iQ2), u1, jt);",
        "const cx<R> a3 = ffv_amp(ffv_row(ub3, g2, Q3, mtr, iQ3), v4, ju);",
        "const cx<R> a4 = ffv_amp(ub3, ffv_col(g2, v4, Q4, mtr, iQ4), ju);",
        "const cx<R> a5 = vvv_amp(ju, g2, jt, KA, KB, KC);",
    ]
    csum = _emit_colour_sum(C, ["a1", "a2", "a3", "a4", "a5"])
    # the massless u line keeps its helicity from p1 to p5: bit 4 = bit 0
    hel_map = "(j & 15) | ((j & 1) << 4)"
    src = HEADER + _struct("ug_ttu", 5, 32, "1.0 / 96.0", 3, pro, body, csum,
                           "u g -> t tbar u: 5 diagrams, diagram colour basis, 32 helicities, 16 allowed",
                           hel_map, 16) + "}  // namespace mf\n"
    return src, dict(n_diag=5, colour=C)

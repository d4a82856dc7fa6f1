"""Tables of the Berends-Giele recursion for g g -> t tbar + (k-2) g on the GPU.

The colour-ordered partial amplitude A(t, sigma_1 .. sigma_k, tbar) of a top
line with k gluons (all momenta incoming; the outgoing gluons enter with minus
their momenta) is built from two kinds of off-shell currents:

* gluon currents J(s) of an ordered sequence s of gluons,
      J(s) = 1/P_s^2 [ - sum_{s = (L, R)} V3(J(L), P_L; J(R), P_R)
                       + sum_{s = (a, b, c)} V4(J(a), J(b), J(c)) ],
  V3 the colour-ordered three-gluon vertex and
  V4(J1, J2, J3) = 2 (J1.J3) J2 - (J1.J2) J3 - (J2.J3) J1 (couplings taken out);
  reversing s multiplies J by (-1)^(|s|+1), so only sequences whose first gluon
  is smaller than their last are stored;
* top-line row spinors U(s) after absorbing the ordered gluons s,
      U(s) = -1/((p_t - P_s)^2 - m^2) [ sum_{s = (L, R)} U(L) Jslash(R) ] (pslash_t - Pslash_s + m),
  U() = ubar(p_t); and the amplitude closes the line on v(p_tbar):
      A(sigma) = sum_{sigma = (L, R)} U(L) Jslash(R) v.
(The factors i of the vertices and propagators multiply every term of every
partial amplitude alike and are left out.)  Every current of a recursion level
has the same number of splits, so one warp can evaluate a level with its
lanes spread over the level's currents.

Output: a header with the index tables (sequence subsets as bit masks, splits
as references "id, sign") and the colour matrix C_{sigma tau} times its common
denominator, sigma and tau running over the lexicographic orderings.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Tuple

from . import colour as col


def _mask(seq) -> int:
    m = 0
    for g in seq:
        m |= 1 << g
    return m


def build(k: int) -> dict:
    gl: Dict[int, List[Tuple]] = {1: [(i,) for i in range(k)]}
    for m in range(2, k + 1):
        gl[m] = [s for s in itertools.permutations(range(k), m) if s[0] < s[-1]]
    jid: Dict[Tuple, int] = {}
    off = 0
    joff = {}
    for m in range(1, k + 1):
        joff[m] = off
        for i, s in enumerate(gl[m]):
            jid[s] = off + i
        off += len(gl[m])
    nj_total = off

    def ref(s) -> int:
        """16-bit reference of the current of any ordered sequence: id | sign bit."""
        if s in jid:
            return jid[s]
        r = tuple(reversed(s))
        neg = (len(s) + 1) % 2 == 1
        return jid[r] | (0x8000 if neg else 0)

    levels = {}
    for m in range(2, k + 1):
        v3, v3m, v4, masks = [], [], [], []
        for s in gl[m]:
            masks.append(_mask(s))
            v3.append([(ref(s[:j]), ref(s[j:])) for j in range(1, m)])
            v3m.append([(_mask(s[:j]), _mask(s[j:])) for j in range(1, m)])
            v4.append([(ref(s[:a]), ref(s[a:b]), ref(s[b:])) for a in range(1, m) for b in range(a + 1, m)])
        levels[m] = dict(n=len(gl[m]), mask=masks, v3=v3, v3m=v3m, v4=v4)

    # top-line currents: prefixes of orderings of length 1 .. k-1; id 0 is ubar itself
    ul: Dict[int, List[Tuple]] = {0: [()]}
    uid: Dict[Tuple, int] = {(): 0}
    uoff = {0: 0}
    off = 1
    for m in range(1, k):
        uoff[m] = off
        ul[m] = list(itertools.permutations(range(k), m))
        for i, s in enumerate(ul[m]):
            uid[s] = off + i
        off += len(ul[m])
    nu_total = off
    ulev = {}
    for m in range(1, k):
        ulev[m] = dict(n=len(ul[m]), mask=[_mask(s) for s in ul[m]],
                       terms=[[(uid[s[:j]], ref(s[j:])) for j in range(m)] for s in ul[m]])
    perms = list(itertools.permutations(range(k)))
    closure = [[(uid[p[:j]], ref(p[j:])) for j in range(k)] for p in perms]

    Cm = col.colour_matrix_words(perms)
    den = 1
    for row in Cm:
        for v in row:
            den = den * v.denominator // math.gcd(den, v.denominator)
    CI = [[int(v * den) for v in row] for row in Cm]
    return dict(k=k, gl=gl, jid=jid, joff=joff, nj_total=nj_total, levels=levels, uoff=uoff, nu_total=nu_total,
                ulev=ulev, closure=closure, perms=perms, colour=CI, colour_den=den)


def _arr(name: str, ctype: str, dims: List[int], flat: List[int]) -> str:
    assert len(flat) == math.prod(dims), (name, len(flat), dims)
    d = "".join(f"[{x}]" for x in dims)
    body = ", ".join(str(v) for v in flat)
    return f"__device__ const {ctype} {name}{d} = {{{body}}};"


def _flat(x):
    if isinstance(x, (list, tuple)):
        out = []
        for y in x:
            out.extend(_flat(y))
        return out
    return [x]


def generate(k: int, name: str) -> Tuple[str, dict]:
    t = build(k)
    L = []
    L.append("// Generated by paper_2105_10529_gb300/gen/bg_tables.py -- do not edit.")
    L.append(f"// Berends-Giele tables of {name}: {k} gluons on a top line, {len(t['perms'])} colour orderings,")
    L.append(f"// {t['nj_total']} stored gluon currents, {t['nu_total']} top-line currents.")
    L.append("#pragma once")
    L.append("#include <cstdint>")
    L.append('#include "mf_bg.cuh"')
    L.append("namespace mf {")
    L.append(f"namespace bg_{name} {{")
    L.append(f"constexpr int K = {k};")
    L.append(f"constexpr int NPERM = {len(t['perms'])};")
    L.append(f"constexpr int NJ = {t['nj_total']};     // stored gluon currents (ids: level by level)")
    L.append(f"constexpr int NU = {t['nu_total']};     // top-line currents (id 0: ubar)")
    L.append(f"constexpr double COLOUR_DEN = {t['colour_den']}.0;")
    for m in range(1, k + 1):
        L.append(f"constexpr int JOFF{m} = {t['joff'][m]}, NJ{m} = {len(t['gl'][m])};")
    for m in range(1, k):
        L.append(f"constexpr int UOFF{m} = {t['uoff'][m]}, NU{m} = {t['ulev'][m]['n']};")
    for m in range(2, k + 1):
        lv = t["levels"][m]
        n = lv["n"]
        L.append(_arr(f"j{m}_mask", "uint8_t", [n], lv["mask"]))
        L.append(_arr(f"j{m}_v3", "uint16_t", [n, m - 1, 2], _flat(lv["v3"])))
        L.append(_arr(f"j{m}_v3m", "uint8_t", [n, m - 1, 2], _flat(lv["v3m"])))
        nv4 = (m - 1) * (m - 2) // 2
        if nv4:
            L.append(_arr(f"j{m}_v4", "uint16_t", [n, nv4, 3], _flat(lv["v4"])))
    for m in range(1, k):
        u = t["ulev"][m]
        L.append(_arr(f"u{m}_mask", "uint8_t", [u["n"]], u["mask"]))
        L.append(_arr(f"u{m}_terms", "uint16_t", [u["n"], m, 2], _flat(u["terms"])))
    L.append(_arr("closure", "uint16_t", [len(t["perms"]), k, 2], _flat(t["closure"])))
    n = len(t["perms"])
    L.append(f"// C_{{sigma tau}} times COLOUR_DEN (integers), orderings lexicographic")
    L.append(_arr("colour", "float", [n * n], _flat(t["colour"])))
    L.append(f"}}  // namespace bg_{name}")
    L.append("")
    # the level drivers: one warp, lanes over the currents of a level (gluon level m with
    # top-line level m - 1), __syncwarp between levels
    def gl(m):
        nv4 = (m - 1) * (m - 2) // 2
        v4 = f"&T::j{m}_v4[0][0][0]" if nv4 else "nullptr"
        return (f"bg_gluon_current<R, {m}, {nv4}>(w, t, T::JOFF{m}, T::j{m}_mask, &T::j{m}_v3[0][0][0], "
                f"&T::j{m}_v3m[0][0][0], {v4})")

    def gl_adj(m):
        nv4 = (m - 1) * (m - 2) // 2
        v4 = f"&T::j{m}_v4[0][0][0]" if nv4 else "nullptr"
        return (f"bg_gluon_current_adj<R, {m}, {nv4}>(w, a, gi, t, T::JOFF{m}, T::j{m}_mask, &T::j{m}_v3[0][0][0], "
                f"&T::j{m}_v3m[0][0][0], {v4})")

    def tl(m, adj=False):
        f = "bg_top_current_adj" if adj else "bg_top_current"
        extra = "a, " if adj else ""
        return f"{f}<R, {m}>(w, {extra}t - T::NJ{m + 1 if not adj else m + 1}, T::UOFF{m}, T::u{m}_mask, &T::u{m}_terms[0][0][0])"

    L.append(f"// level drivers of the recursion of {name} (see mf_bg.cuh)")
    L.append(f"struct BgGen_{name} {{")
    L.append(f"    static constexpr int K = {k}, NPERM = {n}, NJ = {t['nj_total']}, NU = {t['nu_total']};")
    L.append(f"    static constexpr double COLOUR_DEN = {t['colour_den']}.0;")
    L.append(f"    __device__ static const float* colour() {{ return bg_{name}::colour; }}")
    L.append(f"    __device__ static const uint16_t* closure() {{ return &bg_{name}::closure[0][0][0]; }}")
    L.append("    // gluon currents of 2 .. K gluons and top-line currents of 1 .. K-1 gluons from the")
    L.append("    // external states in w.J[0 .. K-1] and w.U[0]")
    L.append("    template <typename R, class W> __device__ static void forward(W& w, int lane)")
    L.append("    {")
    L.append(f"        namespace T = bg_{name};")
    for m in range(2, k + 1):
        # gluon level m with top-line level m - 1
        L.append(f"        for (int t = lane; t < T::NJ{m} + T::NU{m - 1}; t += 32) {{")
        L.append(f"            if (t < T::NJ{m}) {gl(m)};")
        L.append(f"            else {tl(m - 1).replace(f't - T::NJ{m}', f't - T::NJ{m}')};")
        L.append("        }")
        L.append("        __syncwarp();")
    L.append("    }")
    L.append("    // the reverse sweep: adjoints of the currents (a.Jb, a.Ub, a.Vb from the closures)")
    L.append("    // and of the per-event invariants (into the lane's registers gi), level by level")
    L.append("    // downwards: top-line level m with gluon level m + 1 (each pushes only to lower levels)")
    L.append("    template <typename R, class W, class A, class I>")
    L.append("    __device__ static void reverse(const W& w, A& a, I& gi, int lane)")
    L.append("    {")
    L.append(f"        namespace T = bg_{name};")
    for m in range(k - 1, 0, -1):
        L.append(f"        for (int t = lane; t < T::NJ{m + 1} + T::NU{m}; t += 32) {{")
        L.append(f"            if (t < T::NJ{m + 1}) {gl_adj(m + 1)};")
        L.append(f"            else bg_top_current_adj<R, {m}>(w, a, gi, t - T::NJ{m + 1}, T::UOFF{m}, T::u{m}_mask, "
                 f"&T::u{m}_terms[0][0][0]);")
        L.append("        }")
        L.append("        __syncwarp();")
    L.append("    }")
    L.append("};")
    L.append("}  // namespace mf")
    return "\n".join(L) + "\n", t


# Floating-point operations of the routines the recursion calls (add, sub, mul = 1,
# fused multiply-add = 2), read off mf_helas.cuh and mf_bg.cuh as written.
BG_FLOPS = dict(
    v3=166,        # vvv_cur (158) and its accumulation into the current (8)
    v4=192,        # three complex Minkowski products (3 x 30), their scales (6), three complex axpy (96)
    scale=8,       # the current times its inverse propagator denominator
    top_term=96,   # row spinor times Jslash (Sigma, Sigmabar: 24; two 2x2 row products: 56) and its axpy (16)
    top_prop=75,   # (qslash + m) on the row spinor (two real 2x2 halves: 50; mass terms and scale: 24; sign: 1)
    closure=106,   # ffv_amp (102) and its signed accumulation (4)
)


def helicity_flops(k: int) -> dict:
    """Algorithmic FLOPs of one helicity configuration of the recursion: the
    gluon currents, the top line, the closures and the colour sum
    sum_{sigma tau} A*_sigma C_{sigma tau} A_tau (two real quadratic forms of the
    symmetric C, counted over its upper triangle: one multiply-add per pair and form)."""
    t = build(k)
    n_v3 = sum(lv["n"] * (m - 1) for m, lv in t["levels"].items())
    n_v4 = sum(lv["n"] * (m - 1) * (m - 2) // 2 for m, lv in t["levels"].items())
    n_cur = sum(lv["n"] for lv in t["levels"].values())
    n_top = sum(u["n"] * m for m, u in t["ulev"].items())
    n_prop = sum(u["n"] for u in t["ulev"].values())
    n_clo = len(t["closure"]) * k
    n = len(t["perms"])
    f = dict(v3=n_v3 * BG_FLOPS["v3"], v4=n_v4 * BG_FLOPS["v4"], scale=n_cur * BG_FLOPS["scale"],
             top=n_top * BG_FLOPS["top_term"] + n_prop * BG_FLOPS["top_prop"], closure=n_clo * BG_FLOPS["closure"],
             colour=n * (n + 1) * 2 + n * 4)
    f["total"] = sum(f.values())
    f["counts"] = dict(v3=n_v3, v4=n_v4, currents=n_cur, top_terms=n_top, top_props=n_prop, closure_terms=n_clo)
    return f

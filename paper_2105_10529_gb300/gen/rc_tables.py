"""Tables of the helicity-recycled Berends-Giele evaluation of g g -> t tbar g g.

The colour-ordered partial amplitudes A(t, sigma, tbar) of four gluons on a top
line (the recursion of bg_tables.py: gluon currents J(s), top-line row spinors
U(s), all momenta incoming) are evaluated for the 32 helicity configurations of
the parity-halved sum of one event at once, with two observations:

* Helicity recycling.  An off-shell current depends only on the helicities of
  the external particles it contains.  A current of the gluons s has
  2^|s| values over all configurations (fewer when it contains the gluon whose
  helicity the parity halving fixes), not 32; each distinct value is computed
  once and stored in a slot of the event's store.  A "task" is one
  (object, helicity combination) pair; a step runs 32 tasks of one routine,
  one per lane.
* A meet-in-the-middle closure.  Every composition of the ordering
  sigma = (a, b, c, d) into blocks either has a block boundary between b and c,
  or a block that straddles it.  With U2(a b) the top line after absorbing a, b
  (propagator included), W2(c d) the line from v(p_tbar) after absorbing c, d
  (no propagator at its left end), Vr1(d) = P Jslash(d) v and U1(a) = ubar
  Jslash(a) P:
      A(sigma) = U2(a b) W2(c d)
               + ubar Jslash(J(a b c)) Vr1(d)    + ubar Jslash(J(a b c d)) v
               + U1(a) Jslash(J(b c)) Vr1(d)     + U1(a) Jslash(J(b c d)) v,
  so the three-gluon top-line level U(a b c) of the plain recursion (24
  currents, up to 16 helicity combinations each) is never formed.  Each of the
  four straddling terms is row Jslash(J) col = X . J with the bilinear
  X^mu = row gamma^mu col (a current of its own, recycled like the others), so
  the per-configuration work is five complex contractions per ordering.

Helicity bits follow the matrix-element code: configuration ih, bit i the
helicity of external particle i (g g t tbar g g), set = +1; the parity-halved
sum takes ih = 1 + 2 l for lane l (gluon 0 at +1).  The free bits 1..5 of ih are
the lane's bits 0..4, and the slot of an object for lane l is
base + pext(l, lane mask of the object).
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Tuple

from . import colour as col

K = 4
GLUON_BIT = [0, 1, 4, 5]      # helicity bit of gluon i (particle order g g t tbar g g)
T_BIT, TB_BIT = 2, 3
FULL = (1 << K) - 1


class Obj:
    def __init__(self, name: str, kind: str, hmask: int):
        self.name, self.kind, self.hmask = name, kind, hmask
        self.free = sorted(b for b in range(6) if (hmask >> b) & 1 and b != 0)
        self.n = 1 << len(self.free)
        self.base = -1

    @property
    def lane_mask(self) -> int:
        return sum(1 << (b - 1) for b in self.free)

    def combo(self, assign: Dict[int, int]) -> int:
        """Combination index for the helicity bits assign[bit] in {0, 1}."""
        return sum(assign[b] << j for j, b in enumerate(self.free))

    def slot(self, assign: Dict[int, int]) -> int:
        return self.base + self.combo(assign)

    def assignments(self):
        for c in range(self.n):
            yield c, {b: (c >> j) & 1 for j, b in enumerate(self.free)}


def _gmask(seq) -> int:
    m = 0
    for g in seq:
        m |= 1 << g
    return m


def _hmask_gluons(seq) -> int:
    m = 0
    for g in seq:
        m |= 1 << GLUON_BIT[g]
    return m


def build() -> dict:
    objs: Dict[str, Obj] = {}
    order: List[str] = []

    def add(name, kind, hmask):
        o = Obj(name, kind, hmask)
        objs[name] = o
        order.append(name)
        return o

    # external states
    for i in range(K):
        add(f"G{i}", "ext", 1 << GLUON_BIT[i])
    add("UB", "ext", 1 << T_BIT)
    add("V", "ext", 1 << TB_BIT)
    # gluon currents of ordered sequences, one of each reflection pair
    seqs = {m: [s for s in itertools.permutations(range(K), m) if s[0] < s[-1]] for m in (2, 3, 4)}
    for m in (2, 3, 4):
        for s in seqs[m]:
            add("J" + "".join(map(str, s)), f"J{m}", _hmask_gluons(s))

    def J(s) -> Tuple[str, int]:
        """(object, sign) of the current of any ordered gluon sequence s."""
        if len(s) == 1:
            return f"G{s[0]}", 1
        if s[0] < s[-1]:
            return "J" + "".join(map(str, s)), 1
        r = tuple(reversed(s))
        return "J" + "".join(map(str, r)), (-1) ** (len(s) + 1)

    # top line from ubar and from v
    for a in range(K):
        add(f"U1_{a}", "U1", (1 << T_BIT) | (1 << GLUON_BIT[a]))
    for a, b in itertools.permutations(range(K), 2):
        add(f"U2_{a}{b}", "U2", (1 << T_BIT) | _hmask_gluons((a, b)))
    for d in range(K):
        add(f"VR1_{d}", "VR1", (1 << TB_BIT) | (1 << GLUON_BIT[d]))
    for c, d in itertools.permutations(range(K), 2):
        add(f"W2_{c}{d}", "W2", (1 << TB_BIT) | _hmask_gluons((c, d)))
    # bilinears row gamma^mu col of the straddling terms
    for d in range(K):
        add(f"XUV1_{d}", "X", (1 << T_BIT) | (1 << TB_BIT) | (1 << GLUON_BIT[d]))
    for a, d in itertools.permutations(range(K), 2):
        add(f"XU1V1_{a}{d}", "X", (1 << T_BIT) | (1 << TB_BIT) | _hmask_gluons((a, d)))
    for a in range(K):
        add(f"XU1V_{a}", "X", (1 << T_BIT) | (1 << TB_BIT) | (1 << GLUON_BIT[a]))
    add("JQ", "X", (1 << T_BIT) | (1 << TB_BIT))

    base = 0
    for name in order:
        objs[name].base = base
        base += objs[name].n
    nslot = base

    def S(name, assign):
        return objs[name].slot(assign)

    tasks: Dict[str, List[List[int]]] = {t: [] for t in ("EXT", "J2", "J3", "J4", "U1", "VR1", "U2", "W2", "X")}
    for name in order:
        o = objs[name]
        for c, asg in o.assignments():
            full = dict(asg)
            full[0] = 1                      # gluon 0 at +1
            out = o.base + c
            if o.kind == "ext":
                if name.startswith("G"):
                    i = int(name[1])
                    code, hel = i, full[GLUON_BIT[i]]
                elif name == "UB":
                    code, hel = 4, full[T_BIT]
                else:
                    code, hel = 5, full[TB_BIT]
                tasks["EXT"].append([out, code, hel])
            elif o.kind == "J2":
                s = tuple(int(ch) for ch in name[1:])
                a, b = J(s[:1]), J(s[1:])
                tasks["J2"].append([out, S(a[0], full), S(b[0], full), 0, _gmask(s[:1]), _gmask(s[1:]), _gmask(s)])
            elif o.kind == "J3":
                s = tuple(int(ch) for ch in name[1:])
                x, y, z = (J(s[i:i + 1]) for i in range(3))
                xy, yz = J(s[:2]), J(s[1:])
                sgn = (1 if yz[1] < 0 else 0) | (2 if xy[1] < 0 else 0)
                tasks["J3"].append([out, S(x[0], full), S(y[0], full), S(z[0], full), S(xy[0], full), S(yz[0], full),
                                    sgn, _gmask(s[:1]), _gmask(s[1:]), _gmask(s[:2]), _gmask(s[2:]), _gmask(s)])
            elif o.kind == "J4":
                s = tuple(int(ch) for ch in name[1:])
                w_, x, y, z = (J(s[i:i + 1]) for i in range(4))
                wx, xy, yz = J(s[:2]), J(s[1:3]), J(s[2:])
                wxy, xyz = J(s[:3]), J(s[1:])
                sgn = ((1 if xyz[1] < 0 else 0) | (2 if wx[1] * yz[1] < 0 else 0) | (4 if wxy[1] < 0 else 0)
                       | (8 if yz[1] < 0 else 0) | (16 if xy[1] < 0 else 0) | (32 if wx[1] < 0 else 0))
                tasks["J4"].append([out] + [S(t[0], full) for t in (w_, x, y, z, wx, xy, yz, wxy, xyz)] +
                                   [sgn, _gmask(s[:1]), _gmask(s[1:]), _gmask(s[:2]), _gmask(s[2:]), _gmask(s[:3]),
                                    _gmask(s[3:]), _gmask(s)])
            elif o.kind == "U1":
                a = int(name[3:])
                tasks["U1"].append([out, S("UB", full), S(f"G{a}", full), _gmask((a,))])
            elif o.kind == "U2":
                a, b = int(name[3]), int(name[4])
                jab = J((a, b))
                tasks["U2"].append([out, S("UB", full), S(jab[0], full), 1 if jab[1] < 0 else 0, S(f"U1_{a}", full),
                                    S(f"G{b}", full), _gmask((a, b))])
            elif o.kind == "VR1":
                d = int(name[4:])
                tasks["VR1"].append([out, S(f"G{d}", full), S("V", full), FULL ^ (1 << d)])
            elif o.kind == "W2":
                c_, d = int(name[3]), int(name[4])
                jcd = J((c_, d))
                tasks["W2"].append([out, S(jcd[0], full), 1 if jcd[1] < 0 else 0, S("V", full), S(f"G{c_}", full),
                                    S(f"VR1_{d}", full)])
            elif o.kind == "X":
                if name.startswith("XUV1_"):
                    row, colm = "UB", f"VR1_{name[5:]}"
                elif name.startswith("XU1V1_"):
                    row, colm = f"U1_{name[6]}", f"VR1_{name[7]}"
                elif name.startswith("XU1V_"):
                    row, colm = f"U1_{name[5]}", "V"
                else:
                    row, colm = "UB", "V"
                tasks["X"].append([out, S(row, full), S(colm, full)])

    # phase 2: five contractions per ordering (lexicographic orderings = colour-flow order)
    # the orderings in pairs (sigma, reverse sigma), the flows of the colour basis in that order:
    # the third terms X(ubar, v) . J(sigma) of a pair contract the same two slots (J of the reversed
    # sequence is the stored current with its sign), so the pair computes the product once (bit 25
    # of the second's word: reuse the first's value, with the second's sign)
    perms = []
    for s_ in itertools.permutations(range(K)):
        if s_ not in perms:
            perms += [s_, tuple(reversed(s_))]
    terms = []
    lane_words = []   # [ordering][term][lane]: slot of operand A | slot of B << 12 | sign << 24 | reuse << 25
    for (a, b, c_, d) in perms:
        j3a, j4, j2, j3b = J((a, b, c_)), J((a, b, c_, d)), J((b, c_)), J((b, c_, d))
        row = []
        for kind, x, (y, sg) in ((0, f"U2_{a}{b}", (f"W2_{c_}{d}", 1)), (1, f"XUV1_{d}", j3a), (1, "JQ", j4),
                                 (1, f"XU1V1_{a}{d}", j2), (1, f"XU1V_{a}", j3b)):
            ox, oy = objs[x], objs[y]
            row.append([kind, ox.base, ox.lane_mask, oy.base, oy.lane_mask, 1 if sg < 0 else 0])
        terms.append(row)
        second = len(terms) % 2 == 0          # the second ordering of its pair
        if second:
            prev = terms[-2][2]
            assert (prev[1], prev[2], prev[3], prev[4]) == tuple(row[2][1:5]), "a pair shares its J4 term"
        lw = []
        for k, (kind, ba, ma, bb, mb, neg) in enumerate(row):
            words = []
            for lane in range(32):
                sa, sb = ba + _pext(lane, ma), bb + _pext(lane, mb)
                assert sa < 4096 and sb < 4096
                words.append(sa | (sb << 12) | (neg << 24) | ((1 << 25) if (second and k == 2) else 0))
            lw.append(words)
        lane_words.append(lw)

    Cm = col.colour_matrix_words(perms)
    den = 1
    for r in Cm:
        for v in r:
            den = den * v.denominator // math.gcd(den, v.denominator)
    CI = [[int(v * den) for v in r] for r in Cm]
    return dict(objs=objs, order=order, nslot=nslot, tasks=tasks, terms=terms, lane_words=lane_words, perms=perms,
                colour=CI, colour_den=den)


def _pext(lane: int, mask: int) -> int:
    r, j = 0, 0
    for b in range(5):
        if (mask >> b) & 1:
            r |= ((lane >> b) & 1) << j
            j += 1
    return r


# fields per task of each routine (uint16 each), and the order of the steps
TASK_FIELDS = dict(EXT=3, J2=7, J3=12, J4=18, U1=4, VR1=4, U2=7, W2=6, X=3)
STAGES = [("EXT",), ("J2",), ("J3", "U1", "VR1"), ("J4", "U2", "W2", "X")]

# FLOPs of the routines as written (add, sub, mul = 1, fused multiply-add = 2)
RC_FLOPS = dict(
    EXT=6,           # a polarisation or spinor from its basis (scalings)
    J2=166 + 8,      # one three-gluon current and the scale by 1/P^2
    J3=2 * 166 + 192 + 8,
    J4=3 * 166 + 3 * 192 + 8,
    U1=56 + 75,      # row times Jslash, then (qslash + m) and the scale
    VR1=56 + 75,
    U2=2 * 56 + 16 + 75,
    W2=2 * 56 + 16,
    X=80,            # psibar gamma^mu psi
    TERM=30,         # one complex contraction of four components, accumulated
)


def flops_per_event(t: dict) -> dict:
    """Algorithmic FLOPs per event passing the cuts: every task once, the
    contractions of every ordering for each of the 32 configurations, and the
    colour sum of each configuration counted as the diagram code counts it (the
    two real quadratic forms of the symmetric colour matrix over its upper
    triangle, one multiply-add per nonzero entry and form, and the final products)."""
    f = {k: len(v) * RC_FLOPS[k] for k, v in t["tasks"].items()}
    n = len(t["perms"])
    # five contractions per ordering, the third shared by an ordering and its reverse
    f["terms"] = 32 * (n * 5 - n // 2) * RC_FLOPS["TERM"]
    nz = sum(1 for i in range(n) for j in range(i, n) if t["colour"][i][j] != 0)
    f["colour"] = 32 * (2 * 2 * nz + 4 * n)
    f["total"] = sum(f.values())
    return f


def _arr(name: str, ctype: str, dims: List[int], flat: List[int], space: str = "__device__") -> str:
    assert len(flat) == math.prod(dims), (name, len(flat), dims)
    d = "".join(f"[{x}]" for x in dims)
    body = ", ".join(str(v) for v in flat)
    return f"{space} const {ctype} {name}{d} = {{{body}}};"


def generate(name: str = "gg_ttgg") -> Tuple[str, dict]:
    t = build()
    L = []
    L.append("// Generated by paper_2105_10529_gb300/gen/rc_tables.py -- do not edit.")
    L.append(f"// Helicity-recycled Berends-Giele tables of {name}: {len(t['order'])} objects in {t['nslot']} slots,")
    L.append(f"// tasks per routine {({k: len(v) for k, v in t['tasks'].items()})}.")
    L.append("#pragma once")
    L.append("#include <cstdint>")
    L.append("namespace mf {")
    L.append(f"namespace rc_{name} {{")
    L.append(f"constexpr int NSLOT = {t['nslot']};")
    L.append(f"constexpr int NPERM = {len(t['perms'])};")
    L.append(f"constexpr double COLOUR_DEN = {t['colour_den']}.0;")
    L.append("// the tasks of a routine: [step][q][lane] 16-byte words, word q holding fields 8q .. 8q + 7 of")
    L.append("// the lane's task (uint16 each, low half first); field 0 = 0xFFFF: no task")
    for k, v in t["tasks"].items():
        nf = TASK_FIELDS[k]
        nq = (nf + 7) // 8
        steps = (len(v) + 31) // 32
        flat = []
        for s in range(steps):
            rows = []
            for lane in range(32):
                i = s * 32 + lane
                row = v[i] if i < len(v) else [0xFFFF] + [0] * (nf - 1)
                assert len(row) == nf, (k, row)
                rows.append(row + [0] * (8 * nq - nf))
            for q in range(nq):
                for lane in range(32):
                    f = rows[lane][8 * q: 8 * q + 8]
                    flat.extend(f[2 * i] | (f[2 * i + 1] << 16) for i in range(4))
        L.append(f"constexpr int N_{k} = {len(v)}, STEPS_{k} = {steps}, NF_{k} = {nf}, NQ_{k} = {nq};")
        L.append(_arr(f"task_{k}", "uint32_t", [steps, nq, 32, 4], flat))
    flat = []
    for lw in t["lane_words"]:
        for words in lw:
            flat.extend(words)
    L.append("// per ordering (in pairs sigma, reverse sigma), its five contractions (the first a row . col")
    L.append("// product, the others Minkowski products) for every lane: slot of operand A | slot of B << 12 |")
    L.append("// sign << 24 (1: minus) | reuse << 25 (the pair's second: the third term's value is the first's)")
    L.append(f"constexpr int TERM_WORDS = {len(flat)};")
    L.append(_arr("lane_terms", "uint32_t", [len(t["lane_words"]), 5, 32], flat))
    L.append("// the lane masks of the two operands of every contraction (mask A | mask B << 5): the lanes")
    L.append("// whose bits agree on a mask read the same slot (the reverse sweep sums over them)")
    L.append(_arr("term_masks", "uint16_t", [len(t["terms"]), 5],
                  [row[k][2] | (row[k][4] << 5) for row in t["terms"] for k in range(5)], space="__constant__"))
    n = len(t["perms"])
    L.append("// the colour matrix C_{sigma tau} times COLOUR_DEN, the orderings in the pairs above (the per-lane")
    L.append("// colour sum of the derivative pass reads it as constant operands, the tensor cores as shorts)")
    L.append(_arr("colour", "float", [n * n], [t["colour"][i][j] for i in range(n) for j in range(n)],
                  space="__constant__"))
    assert t["colour_den"] == 54
    L.append(_arr("colour54", "short", [n * n], [t["colour"][i][j] for i in range(n) for j in range(n)],
                  space="__constant__"))
    L.append(f"}}  // namespace rc_{name}")
    L.append("}  // namespace mf")
    return "\n".join(L) + "\n", t


if __name__ == "__main__":
    t = build()
    print("slots", t["nslot"], {k: len(v) for k, v in t["tasks"].items()})
    print(flops_per_event(t))

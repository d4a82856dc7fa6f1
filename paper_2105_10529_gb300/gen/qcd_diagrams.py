"""Tree-level Feynman diagrams for g g -> t tbar + (k-2) gluons and emission
of a straight-line CUDA matrix element (Sec. 2.1-2.2 of arXiv:2105.10529:
process-specific code built from external wavefunctions, vertices and
propagators, looped over helicities and summed with the colour matrix).

Diagrams.  All gluons are treated with incoming momenta K_i (outgoing
gluons get K = -p).  A diagram attaches an ordered sequence of blocks
B_1..B_m to the heavy-quark line ubar(p3) ... v(p4); each block is a gluon
tree built from three- and four-gluon vertices (one leaf = an external
gluon).  With m = 1 the single tree meets the quark pair's own current
J_q at its top vertex.  For k = 2, 3, 4 this gives 3, 16 and 123 diagrams,
the four-gluon vertex counted once (its three colour structures are three
amplitudes).

Colour.  Every amplitude's colour factor is expanded on the colour-flow
basis (T^{s_1} ... T^{s_k})_{i3 j4}, s a permutation of the gluons, using
f^{abc} T^c = -i [T^a, T^b]; the overall phases of the vertex and propagator
factors are folded into those coefficients, so the Lorentz routines only
carry real factors.  The colour matrix comes from the Fierz identity
(colour.py).  Couplings: every diagram has k powers of g, applied at the end.

Feynman rules (Feynman gauge; D = d - i g A^a T^a): quark-gluon vertex
i g gamma^mu T^a, quark propagator i (qslash + m)/(q^2 - m^2), gluon
propagator -i g_{mu nu}/k^2, three-gluon vertex g f^{abc} V_{mu nu rho},
four-gluon vertex -i g^2 (f f)(g g - g g) in three colour structures.
"""
from __future__ import annotations

import itertools
import re
import math
from fractions import Fraction
from functools import reduce
from typing import Dict, List, Tuple

from . import colour as col

I = 1j


# ---------------------------------------------------------------- gluon trees

def _subsets_with_min(S):
    """Proper non-empty subsets of S that contain min(S)."""
    s = sorted(S)
    first, rest = s[0], s[1:]
    for r in range(0, len(rest) + 1):
        for c in itertools.combinations(rest, r):
            sub = frozenset((first,) + c)
            if sub != frozenset(S):
                yield sub


def trees(S) -> List[Tuple]:
    """All gluon trees over the leaf set S (canonical child order)."""
    S = frozenset(S)
    if len(S) == 1:
        return [("L", next(iter(S)))]
    out = []
    for S1 in _subsets_with_min(S):
        S2 = S - S1
        for A in trees(S1):
            for B in trees(S2):
                out.append(("V3", A, B))
    if len(S) >= 3:
        for S1 in _subsets_with_min(S):
            R = S - S1
            if len(R) < 2:
                continue
            for S2 in _subsets_with_min(R):
                S3 = R - S2
                for A in trees(S1):
                    for B in trees(S2):
                        for C in trees(S3):
                            for t in (1, 2, 3):
                                out.append(("V4", A, B, C, t))
    return out


def leaves(T) -> frozenset:
    if T[0] == "L":
        return frozenset([T[1]])
    return reduce(frozenset.union, (leaves(c) for c in T[1:4] if isinstance(c, tuple)))


def tree_poly(T) -> col.Poly:
    """Colour polynomial of a tree current with its phases folded in:
    leaf 1; three-gluon current -[W_A, W_B]; four-gluon currents
    +[[W_A,W_B],W_C], +[[W_A,W_C],W_B], +[[W_B,W_C],W_A]."""
    if T[0] == "L":
        return {(T[1],): 1}
    if T[0] == "V3":
        return col.pscale(col.comm(tree_poly(T[1]), tree_poly(T[2])), -1)
    A, B, C = (tree_poly(x) for x in T[1:4])
    t = T[4]
    if t == 1:
        return col.comm(col.comm(A, B), C)
    if t == 2:
        return col.comm(col.comm(A, C), B)
    return col.comm(col.comm(B, C), A)


def ordered_partitions(items):
    """Ordered set partitions of items into non-empty blocks."""
    items = list(items)
    if not items:
        yield []
        return
    n = len(items)
    # choose the first block as any non-empty subset, recurse on the rest
    for r in range(1, n + 1):
        for first in itertools.combinations(items, r):
            rest = [x for x in items if x not in first]
            for tail in ordered_partitions(rest):
                yield [frozenset(first)] + tail


def diagrams(k: int):
    """List of (kind, data, colour poly).  kind 'Q': blocks on the quark line;
    'T3'/'T4': a single tree meeting the quark current at its top vertex."""
    out = []
    G = frozenset(range(k))
    for part in ordered_partitions(range(k)):
        m = len(part)
        if m < 2:
            continue
        for combo in itertools.product(*[trees(B) for B in part]):
            poly = reduce(col.pmul, [tree_poly(T) for T in combo])
            phase = I * (-1) ** (m - 1)
            out.append(("Q", tuple(combo), col.pscale(poly, phase)))
    for S1 in _subsets_with_min(G):
        S2 = G - S1
        for A in trees(S1):
            for B in trees(S2):
                poly = col.pscale(col.comm(tree_poly(A), tree_poly(B)), -I)
                out.append(("T3", (A, B), poly))
    if k >= 3:
        for S1 in _subsets_with_min(G):
            R = G - S1
            if len(R) < 2:
                continue
            for S2 in _subsets_with_min(R):
                S3 = R - S2
                for A in trees(S1):
                    for B in trees(S2):
                        for C in trees(S3):
                            Pa, Pb, Pc = tree_poly(A), tree_poly(B), tree_poly(C)
                            polys = [col.comm(col.comm(Pa, Pb), Pc), col.comm(col.comm(Pa, Pc), Pb),
                                     col.comm(col.comm(Pb, Pc), Pa)]
                            for t in (1, 2, 3):
                                out.append(("T4", (A, B, C, t), col.pscale(polys[t - 1], I)))
    return out


def count_feynman_diagrams(k: int) -> int:
    """Diagrams with the four-gluon vertex counted once."""
    n = 0
    for kind, data, _ in diagrams(k):
        if kind == "Q":
            if all(_v4_term(T) in (0, 1) for T in data):
                n += 1
        elif kind == "T3":
            if all(_v4_term(T) in (0, 1) for T in data):
                n += 1
        else:
            if data[3] == 1 and all(_v4_term(T) in (0, 1) for T in data[:3]):
                n += 1
    return n


def _v4_term(T) -> int:
    """0 if T has no four-gluon vertex, 1 if every one has term 1, else 2."""
    if T[0] == "L":
        return 0
    if T[0] == "V3":
        a, b = _v4_term(T[1]), _v4_term(T[2])
        return max(a, b)
    inner = max(_v4_term(x) for x in T[1:4])
    return max(inner, 1 if T[4] == 1 else 2)


# ---------------------------------------------------------------- code emission

class Emitter:
    """Builds the straight-line helicity body with memoised wavefunctions."""

    def __init__(self, k: int):
        self.k = k
        self.lines: List[str] = []
        self.tree_var: Dict[Tuple, str] = {}
        self.L: Dict[Tuple, str] = {(): "ub3"}
        self.R: Dict[Tuple, str] = {(): "v4"}
        self.n_w = 0
        self.n_amp = 0
        self.kvars = set()       # gluon subsets whose momentum (R) is needed
        self.gden = set()        # gluon subsets whose 1/K^2 is needed
        self.qsub = set()        # quark propagator subsets (absorbed from the ubar side)
        self.kmasks = set()      # gluon subsets whose momentum is read in the body
        self.counts = dict(vvv=0, vvvv=0, ffv_row=0, ffv_col=0, ffv_amp=0, vvv_amp=0, vvvv_amp=0, ffv_cur=0)

    @staticmethod
    def mask(S) -> int:
        return sum(1 << i for i in S)

    def new_w(self) -> str:
        self.n_w += 1
        return f"w{self.n_w}"

    def mom(self, m: int) -> str:
        """R-typed momentum of the gluons in mask m, loaded from the per-event
        slot at its point of use (a volatile load, so it is not kept live)."""
        self.n_w += 1
        self.kmasks.add(m)
        v = f"k{m}_{self.n_w}"
        comps = ", ".join(f"ldv(v.K[@K{m}@][{c}])" for c in range(4))
        self.lines.append(f"const R {v}[4] = {{{comps}}};")
        return v

    def qmom(self, m: int) -> str:
        """R-typed quark propagator momentum p3 - K(mask m) at its point of use."""
        self.n_w += 1
        self.kmasks.add(m)
        v = f"q{m}_{self.n_w}"
        comps = ", ".join(f"ldv(v.p3[{c}]) - ldv(v.K[@K{m}@][{c}])" for c in range(4))
        self.lines.append(f"const R {v}[4] = {{{comps}}};")
        return v

    def tree(self, T) -> str:
        if T in self.tree_var:
            return self.tree_var[T]
        if T[0] == "L":
            v = f"g{T[1]}"
            self.tree_var[T] = v
            return v
        if T[0] == "V3":
            a, b = self.tree(T[1]), self.tree(T[2])
            ma, mb = self.mask(leaves(T[1])), self.mask(leaves(T[2]))
            m = ma | mb
            self.gden.add(m)
            ka, kb = self.mom(ma), self.mom(mb)
            v = self.new_w()
            self.lines.append(f"const W4<R> {v} = vvv_cur({a}, {b}, {ka}, {kb}, iG{m});")
            self.counts["vvv"] += 1
            self.tree_var[T] = v
            return v
        # V4: emit all three structures at once
        base = T[:4]
        keys = [base + (t,) for t in (1, 2, 3)]
        a, b, c = (self.tree(x) for x in T[1:4])
        m = self.mask(leaves(T))
        self.gden.add(m)
        vs = [self.new_w() for _ in range(3)]
        self.lines.append(f"W4<R> {vs[0]}, {vs[1]}, {vs[2]};")
        self.lines.append(f"vvvv_cur({a}, {b}, {c}, iG{m}, {vs[0]}, {vs[1]}, {vs[2]});")
        self.counts["vvvv"] += 1
        for kk, v in zip(keys, vs):
            self.tree_var[kk] = v
        return self.tree_var[T]

    def left(self, seq: Tuple) -> str:
        """ubar(p3) with the blocks of seq absorbed (with propagator)."""
        if seq in self.L:
            return self.L[seq]
        prev = self.left(seq[:-1])
        J = self.tree(seq[-1])
        S = frozenset().union(*[leaves(T) for T in seq])
        m = self.mask(S)
        self.qsub.add(m)
        q = self.qmom(m)
        v = self.new_w()
        self.lines.append(f"const W4<R> {v} = ffv_row({prev}, {J}, {q}, mt, iQ{m});")
        self.counts["ffv_row"] += 1
        self.L[seq] = v
        return v

    def right(self, seq: Tuple) -> str:
        """v(p4) with the blocks of seq absorbed (with propagator)."""
        if seq in self.R:
            return self.R[seq]
        nxt = self.right(seq[1:])
        J = self.tree(seq[0])
        full = frozenset(range(self.k))
        S = full - frozenset().union(*[leaves(T) for T in seq])    # absorbed on the ubar side
        m = self.mask(S)
        self.qsub.add(m)
        q = self.qmom(m)
        v = self.new_w()
        self.lines.append(f"const W4<R> {v} = ffv_col({J}, {nxt}, {q}, mt, iQ{m});")
        self.counts["ffv_col"] += 1
        self.R[seq] = v
        return v

    def new_amp(self) -> str:
        self.n_amp += 1
        return f"a{self.n_amp}"


def _split_cost(em: Emitter, blocks: Tuple, j: int) -> int:
    c = 0
    for l in range(1, j + 1):
        if blocks[:l] not in em.L:
            c += 1
    m = len(blocks)
    for l in range(j + 2, m):
        if blocks[l:] not in em.R:
            c += 1
    return c


def _jadd(jv: str, a: str, c: complex) -> str:
    c = complex(c)
    re, im = c.real, c.imag
    if (re, im) == (1, 0):
        return f"jadd_p({jv}, {a});"
    if (re, im) == (-1, 0):
        return f"jadd_m({jv}, {a});"
    if (re, im) == (0, 1):
        return f"jadd_pi({jv}, {a});"
    if (re, im) == (0, -1):
        return f"jadd_mi({jv}, {a});"
    return f"jadd_c({jv}, {a}, R({re!r}), R({im!r}));"


def _block_size(T) -> int:
    return len(leaves(T))


def _emit_amp_jamps(em: "Emitter", a: str, poly, widx):
    for w, c in sorted(poly.items()):
        em.lines.append(_jadd(f"jamp[{widx[w]}]", a, c))


def _r1(em: "Emitter", leaf: int, tag: str) -> str:
    """v(p4) with one external gluon absorbed: (qslash + m) gslash v4 / (q^2 - m^2)."""
    key = ("R1", leaf, tag)
    if key in em.tree_var:
        return em.tree_var[key]
    v = em.new_w()
    m = full_mask = (1 << em.k) - 1
    S = full_mask & ~(1 << leaf)
    em.qsub.add(S)
    q = em.qmom(S)
    em.lines.append(f"const W4<R> {v} = ffv_col(g{leaf}, v4, {q}, mt, iQ{S});")
    em.counts["ffv_col"] += 1
    em.tree_var[key] = v
    return v


def _ffv_amp(em: "Emitter", L: str, R_: str, J: str) -> str:
    a = em.new_amp()
    em.lines.append(f"const cx<R> {a} = ffv_amp({L}, {R_}, {J});")
    em.counts["ffv_amp"] += 1
    return a


def _schedule(em: "Emitter", diags, k: int, widx):
    """Emission order chosen for short live ranges:
    A. quark-line diagrams whose blocks are single gluons or pair currents,
       walked depth-first over their ubar-side chains; a diagram ending in a
       single gluon closes on v(p4) with that gluon absorbed (R1), any other
       closes on v(p4) directly;
    B. for every three-gluon subset (k = 4): its tree currents, the
       quark-line diagrams (S, c) and (c, S) and the single-tree diagram with
       top vertex (S, c), c the remaining gluon; then the currents die;
    C. the remaining single-tree diagrams (top vertex meets the quark
       current J_q)."""
    full = (1 << k) - 1
    # pair currents first (live throughout)
    for T in sorted({T for kind, data, _ in diags if kind == "Q" for T in data if _block_size(T) == 2}, key=str):
        em.tree(T)
    # A
    qa = [d for d in diags if d[0] == "Q" and max(_block_size(T) for T in d[1]) <= 2]
    qa.sort(key=lambda d: [(_block_size(T), str(T)) for T in d[1]])
    for kind, blocks, poly in qa:
        m = len(blocks)
        last = blocks[-1]
        if last[0] == "L":
            Lv = em.left(blocks[:m - 2])
            J = em.tree(blocks[m - 2])
            Rv = _r1(em, last[1], "A")
        else:
            Lv = em.left(blocks[:m - 1])
            J = em.tree(last)
            Rv = "v4"
        a = _ffv_amp(em, Lv, Rv, J)
        _emit_amp_jamps(em, a, poly, widx)
    # quark current for the single-tree diagrams
    em.gden.add(full)
    em.kvars.add(full)
    em.lines.append(f"const W4<R> jq = ffv_cur(ub3, v4, iG{full});")
    em.counts["ffv_cur"] += 1
    single = [d for d in diags if d[0] != "Q"]
    done_single = set()
    # B
    if k >= 4:
        # chains of phase A end here; single-gluon chains are recomputed inside each block
        em.L = {(): "ub3"}
        for S in itertools.combinations(range(k), 3):
            S = frozenset(S)
            c = next(iter(frozenset(range(k)) - S))
            em.lines.append("{")
            Rc = _r1(em, c, "B%d" % c)
            Lc = em.left((("L", c),))
            uses = {}
            for kind, blocks, poly in diags:
                if kind != "Q" or len(blocks) != 2:
                    continue
                sizes = [_block_size(T) for T in blocks]
                if sizes == [3, 1] and leaves(blocks[0]) == S:
                    uses.setdefault(blocks[0], []).append(("QR", poly))
                elif sizes == [1, 3] and leaves(blocks[1]) == S:
                    uses.setdefault(blocks[1], []).append(("QL", poly))
            for i, (kind, data, poly) in enumerate(single):
                if kind == "T3" and (leaves(data[0]) == S or leaves(data[1]) == S):
                    T = data[0] if leaves(data[0]) == S else data[1]
                    uses.setdefault(T, []).append(("T3", i))
                    done_single.add(i)
            # one tree (or one four-gluon vertex with its three structures) at a time
            groups = []
            for T in trees(S):
                if T[0] == "V4":
                    key = T[:4]
                    if groups and groups[-1][0] == key:
                        groups[-1][1].append(T)
                        continue
                    groups.append((key, [T]))
                else:
                    groups.append((T, [T]))
            for _, group in groups:
                em.lines.append("{")
                for T in group:
                    Jv = em.tree(T)
                    for use in uses.get(T, []):
                        if use[0] == "QR":
                            a_ = _ffv_amp(em, "ub3", Rc, Jv)
                            _emit_amp_jamps(em, a_, use[1], widx)
                        elif use[0] == "QL":
                            a_ = _ffv_amp(em, Lc, "v4", Jv)
                            _emit_amp_jamps(em, a_, use[1], widx)
                        else:
                            kind, data, poly = single[use[1]]
                            _emit_single(em, kind, data, poly, widx, full)
                em.lines.append("}")
                for T in group:
                    em.tree_var.pop(T, None)
            em.lines.append("}")
            em.L.pop((("L", c),), None)
    # C
    for i, (kind, data, poly) in enumerate(single):
        if i not in done_single:
            _emit_single(em, kind, data, poly, widx, full)


def _emit_single(em: "Emitter", kind, data, poly, widx, full):
    if kind == "T3":
        A, B = data
        va, vb = em.tree(A), em.tree(B)
        ma, mb = em.mask(leaves(A)), em.mask(leaves(B))
        ka, kb = em.mom(ma), em.mom(mb)
        kq = em.mom(full)
        em.lines.append(f"const R nk{kq}[4] = {{-{kq}[0], -{kq}[1], -{kq}[2], -{kq}[3]}};")
        a = em.new_amp()
        em.lines.append(f"const cx<R> {a} = vvv_amp({va}, {vb}, jq, {ka}, {kb}, nk{kq});")
        em.counts["vvv_amp"] += 1
        _emit_amp_jamps(em, a, poly, widx)
        return
    A, B, C, t = data
    key = ("AMP4", A, B, C)
    if key not in em.tree_var:
        va, vb, vc = em.tree(A), em.tree(B), em.tree(C)
        names = [em.new_amp() for _ in range(3)]
        em.lines.append(f"cx<R> {names[0]}, {names[1]}, {names[2]};")
        em.lines.append(f"vvvv_amp({va}, {vb}, {vc}, jq, {names[0]}, {names[1]}, {names[2]});")
        em.counts["vvvv_amp"] += 1
        em.tree_var[key] = names
    _emit_amp_jamps(em, em.tree_var[key][t - 1], poly, widx)


_K4 = re.compile(r"const R (\w+)\[4\] = \{ldv\(v\.K\[(\d+)\]\[0\]\), ldv\(v\.K\[\2\]\[1\]\), "
                 r"ldv\(v\.K\[\2\]\[2\]\), ldv\(v\.K\[\2\]\[3\]\)\};")
_Q4 = re.compile(r"const R (\w+)\[4\] = \{ldv\(v\.p3\[0\]\) - ldv\(v\.K\[(\d+)\]\[0\]\), "
                 r"ldv\(v\.p3\[1\]\) - ldv\(v\.K\[\2\]\[1\]\), ldv\(v\.p3\[2\]\) - ldv\(v\.K\[\2\]\[2\]\), "
                 r"ldv\(v\.p3\[3\]\) - ldv\(v\.K\[\2\]\[3\]\)\};")


def _wide_access(line: str) -> str:
    """One line of the warp-per-event helicity body with its shared-memory
    accesses widened: momentum 4-vectors of the record in one 16-byte load,
    colour-flow updates as one 8-byte load and store (same arithmetic)."""
    line = _K4.sub(lambda m: f"R {m.group(1)}[4]; ldv4(v.K[{m.group(2)}], {m.group(1)});", line)
    line = _Q4.sub(lambda m: f"R {m.group(1)}[4]; ldv4_diff(v.p3, v.K[{m.group(2)}], {m.group(1)});", line)
    line = line.replace("{ vset(jamp[c].r, R(0)); vset(jamp[c].i, R(0)); }", "jzero64(jamp[c]);")
    for f in ("jadd_mi(", "jadd_pi(", "jadd_p(", "jadd_m("):
        line = line.replace(f, f.replace("jadd_", "jadd64_"))
    assert "jadd_" not in line and "ldv(v.K" not in line, line
    return line


def generate_gluon_process(k: int, name: str, sym: Fraction) -> Tuple[str, dict]:
    """CUDA source for the averaged |M|^2 of g g -> t tbar + (k-2) g."""
    words = list(itertools.permutations(range(k)))
    widx = {w: i for i, w in enumerate(words)}
    ncol = len(words)
    diags = diagrams(k)
    em = Emitter(k)
    full = (1 << k) - 1
    _schedule(em, diags, k, widx)
    need_jq = True

    # colour matrix
    Cm = col.colour_matrix_words(words)
    den = 1
    for row in Cm:
        for v in row:
            den = den * v.denominator // math.gcd(den, v.denominator)
    CI = [[int(v * den) for v in row] for row in Cm]

    n_in = 2
    n_ext = k + 2
    gl_ext = [0, 1] + list(range(4, 2 + k))
    gden = sorted(em.gden)
    qsub = sorted(em.qsub)
    gidx = {m: i for i, m in enumerate(gden)}
    qidx = {m: i for i, m in enumerate(qsub)}

    kmasks = sorted(em.kmasks)
    kidx = {m: i for i, m in enumerate(kmasks)}
    # prologue: helicity-independent pieces, FP64 arithmetic, stored as R in the slot
    pro: List[str] = []
    pro.append("// gluon momenta, incoming convention: gluons 0,1 incoming, the rest outgoing")
    for i, e in enumerate(gl_ext):
        sgn = "" if i < n_in else "-"
        pro.append(f"const S kd{1 << i}[4] = {{{sgn}p[{e}][0], {sgn}p[{e}][1], {sgn}p[{e}][2], {sgn}p[{e}][3]}};")
    needed_sums = {m for m in set(gden) | set(qsub) | set(kmasks) if bin(m).count("1") > 1}
    for m in sorted(needed_sums, key=lambda x: (bin(x).count("1"), x)):
        bits = [1 << i for i in range(k) if m >> i & 1]
        comps = ", ".join(" + ".join(f"kd{b}[{c}]" for b in bits) for c in range(4))
        pro.append(f"const S kd{m}[4] = {{{comps}}};")
    for m in kmasks:
        pro.append(f"for (int c = 0; c < 4; ++c) v.K[{kidx[m]}][c] = R(kd{m}[c]);")
    pro.append("for (int c = 0; c < 4; ++c) v.p3[c] = R(p[2][c]);")
    for m in gden:
        pro.append(f"v.iG[{gidx[m]}] = R(1.0 / mdot(kd{m}, kd{m}));")
    for m in qsub:
        pro.append(f"{{ const S q[4] = {{p[2][0] - kd{m}[0], p[2][1] - kd{m}[1], p[2][2] - kd{m}[2], p[2][3] - kd{m}[3]}};")
        pro.append(f"  v.iQ[{qidx[m]}] = R(1.0 / (mdot(q, q) - mt * mt)); }}")
    for i, e in enumerate(gl_ext):
        pro.append(f"{{ S a[3], b[3]; gluon_basis(p[{e}], a, b);")
        pro.append(f"  for (int j = 0; j < 3; ++j) {{ v.e1[{i}][j] = R(a[j]); v.e2[{i}][j] = R(b[j]); }} }}")
    pro.append("v.fb3 = fermion_basis<R>(p[2], mt);")
    pro.append("v.fb4 = fermion_basis<R>(p[3], mt);")
    pro.append("v.mt = R(mt);")

    import re as _re

    def subst(line: str) -> str:
        line = _re.sub(r"\biG(\d+)\b", lambda mm: f"ldv(v.iG[{gidx[int(mm.group(1))]}])", line)
        line = _re.sub(r"\biQ(\d+)\b", lambda mm: f"ldv(v.iQ[{qidx[int(mm.group(1))]}])", line)
        line = _re.sub(r"@K(\d+)@", lambda mm: str(kidx[int(mm.group(1))]), line)
        line = line.replace(", mt, ", ", ldv(v.mt), ")
        return line

    body: List[str] = []
    body.append("// colour-flow amplitudes accumulate in the slot (shared memory), not in registers")
    body.append("volatile cx<R>* jamp = reinterpret_cast<volatile cx<R>*>(const_cast<cx<R>*>(v.jamp));")
    body.append("#pragma unroll")
    body.append("for (int c = 0; c < NCOL; ++c) { vset(jamp[c].r, R(0)); vset(jamp[c].i, R(0)); }")
    for i, e in enumerate(gl_ext):
        out = "false" if i < n_in else "true"
        body.append(f"W4<R> g{i}; {{ R a[3], b[3]; for (int j = 0; j < 3; ++j) {{ a[j] = ldv(v.e1[{i}][j]); b[j] = ldv(v.e2[{i}][j]); }}")
        body.append(f"  g{i} = ext_gluon(a, b, HEL({e}), {out}); }}")
    body.append("const W4<R> ub3 = ext_ubar(load_basis(v.fb3), HEL(2));")
    body.append("const W4<R> v4 = ext_v(load_basis(v.fb4), HEL(3));")
    body.extend(subst(l) for l in em.lines)

    # colour sum, symmetric form: sum_ij C_ij J_i J_j = sum_i J_i (C_ii J_i + 2 sum_{j>i} C_ij J_j)
    cs: List[str] = []
    cs.append("cx<R> J[NCOL];")
    cs.append("#pragma unroll")
    cs.append("for (int c = 0; c < NCOL; ++c) J[c] = mkc(vget(jamp[c].r), vget(jamp[c].i));")
    cs.append("R me = R(0);")
    for i in range(ncol):
        tr = [f"R({float(CI[i][i])!r}) * J[{i}].r"]
        ti = [f"R({float(CI[i][i])!r}) * J[{i}].i"]
        for j in range(i + 1, ncol):
            if CI[i][j] != 0:
                tr.append(f"R({float(2 * CI[i][j])!r}) * J[{j}].r")
                ti.append(f"R({float(2 * CI[i][j])!r}) * J[{j}].i")
        cs.append(f"{{ const R zr = {' + '.join(tr)}; const R zi = {' + '.join(ti)};")
        cs.append(f"  me = fma(J[{i}].r, zr, fma(J[{i}].i, zi, me)); }}")
    cs.append("return me;")

    n_diag = count_feynman_diagrams(k)
    src = []
    src.append(f"// Generated by paper_2105_10529_gb300/gen/qcd_diagrams.py -- do not edit.")
    src.append(f"// {name}: {n_diag} Feynman diagrams ({len(diags)} amplitudes with the four-gluon")
    src.append(f"// colour structures counted apart), {ncol} colour flows, {1 << n_ext} helicities.")
    src.append(f"// Wavefunction/vertex calls per helicity: {em.counts}")
    tc = ncol >= 24
    src.append("#pragma once")
    src.append('#include "mf_helas.cuh"')
    src.append('#include "mf_tc.cuh"')
    src.append("namespace mf {")
    if tc:
        src.append(f"// 54 C: the colour matrix times its common denominator, for the tensor-core colour sum")
        vals = ", ".join(str(int(CI[i][j])) for i in range(ncol) for j in range(ncol))
        src.append(f"static __constant__ short colour54_{name}[{ncol * ncol}] = {{{vals}}};")
        assert den == 54
    src.append(f"struct Me_{name} {{")
    src.append(f"  static constexpr int NEXT = {n_ext};")
    src.append(f"  static constexpr int NCOL = {ncol};")
    src.append(f"  static constexpr int NHEL = {1 << n_ext};")
    src.append(f"  static constexpr int NGLUON = {k};")
    src.append(f"  static constexpr int NDIAG = {n_diag};")
    src.append(f"  static constexpr double COLOUR_DEN = {den}.0;")
    src.append(f"  static constexpr double AVG = 1.0 / 256.0;")
    src.append(f"  static constexpr double SYM = {float(sym)!r};")
    src.append(f"  // colour sum on the tensor cores available (a dense 24 x 24 contraction)")
    src.append(f"  static constexpr bool TC_COLOUR = {'true' if tc else 'false'};")
    if tc:
        src.append(f"  __device__ static const short* colour54() {{ return colour54_{name}; }}")
    src.append("  // helicity-independent per-event pieces")
    n_words = 4 * len(kmasks) + 4 + max(1, len(gden)) + max(1, len(qsub)) + 6 * k + 20 + 1 + 2 * ncol
    pad = 1 if n_words % 2 == 0 else 2   # odd number of 32-bit words per slot: conflict-free in shared memory
    src.append("  // per-thread slot: internal momenta, FP64-computed inverse denominators,")
    src.append("  // polarisation bases and spinor pieces of the event (kept in shared memory)")
    src.append("  template <typename R> struct Inv {")
    src.append(f"    R K[{len(kmasks)}][4]; R p3[4]; R iG[{max(1, len(gden))}]; R iQ[{max(1, len(qsub))}];")
    src.append(f"    R e1[{k}][3]; R e2[{k}][3]; FermionBasis<R> fb3, fb4; R mt;")
    src.append(f"    cx<R> jamp[{ncol}];   // colour-flow amplitudes of the helicity being summed")
    src.append(f"    float pad[{pad}];")
    src.append("  };")
    src.append("  // averaged |M|^2 (spin/colour average and identical-particle factor included);")
    src.append("  // p: momenta (E,px,py,pz) incoming first: g, g, t, tbar, g...")
    src.append("  // slot: this thread's Inv<R> in shared memory, or null for a private local copy")
    src.append("  // SYNC: a CTA barrier after every helicity (every thread of the CTA must call)")
    src.append("  // R: float or double (or Dual of them for derivatives); the momenta, masses and")
    src.append("  // the result use the scalar S of the momenta: the matching FP64 scalar Widen<R>::type,")
    src.append("  // or Df (double-float) where the mixed-precision kinematics hand theirs on")
    src.append("  // TC: colour sum on the tensor cores (float, SYNC, CTAs of 128 or 256 threads; cta: the CTA's TcCta)")
    src.append("  // hpart, hparts: helicity split, this call sums every hparts-th evaluated helicity")
    src.append("  // from the hpart-th on (the caller adds the hparts partial sums)")
    src.append("  template <typename R, bool SYNC = false, bool TC = false, typename S = typename Widen<R>::type>")
    src.append("  __device__ static S me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt, typename NoDeduce<S>::type gs,")
    src.append("                         void* slot, void* cta = nullptr, int hpart = 0, int hparts = 1);")
    src.append("  template <typename R> static constexpr size_t slot_bytes() { return sizeof(Inv<R>); }")
    src.append("  // per-helicity averaged |M_h|^2 of all NHEL configurations into out[NHEL] (diagnostic)")
    src.append("  template <typename R>")
    src.append("  __device__ static void hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,")
    src.append("                                     typename Widen<R>::type gs, double* out);")
    if tc:
        src.append("  // warp-per-event schedule: the helicity-independent words of Inv (everything before jamp),")
        src.append("  // filled for one event by one thread (inv), then read by the 32 lanes of a warp, each")
        src.append("  // evaluating one of the 32 helicities of the parity-halved sum (hel_j, colour flows in")
        src.append("  // caller storage, no colour sum)")
        src.append(f"  static constexpr int INV_WORDS = {n_words - 2 * ncol};")
        src.append("  template <typename R>")
        src.append("  __device__ static void inv(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt, Inv<R>& v);")
        src.append("  // hel_j reads the warp's record at REC_OFF + (threadIdx.x / 32) REC_STRIDE bytes and keeps the")
        src.append("  // thread's colour flows at threadIdx.x JROW words, both from the start of dynamic shared memory")
        src.append("  template <typename R, int JROW, int REC_OFF, int REC_STRIDE>")
        src.append("  __device__ static void hel_j(int ih);")
    src.append("};")
    src.append("")
    src.append("// one helicity configuration: amplitudes, colour flows and (CSUM) the colour sum;")
    src.append("// out of line so that its register allocation sees only one helicity")
    src.append("template <typename R, bool CSUM = true>")
    src.append(f"__device__ __noinline__ R hel_{name}(const Me_{name}::Inv<R>& v, int ih)")
    src.append("{")
    src.append(f"    constexpr int NCOL = Me_{name}::NCOL;")
    src.append("#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)")
    for l in body:
        src.append("    " + l)
    src.append("    if constexpr (!CSUM) return R(0);   // the caller sums the colour flows left in the slot")
    for l in cs:
        src.append("    " + l)
    src.append("#undef HEL")
    src.append("}")
    src.append("")
    src.append("template <typename R, bool SYNC, bool TC, typename S>")
    src.append(f"__device__ __noinline__ S me2_{name}_impl(const S* pflat, S mt, S gs, void* slot, void* cta, int hpart,")
    src.append("                                       int hparts)")
    src.append("{")
    src.append(f"    constexpr int NEXT = Me_{name}::NEXT, NHEL = Me_{name}::NHEL, NGLUON = Me_{name}::NGLUON;")
    src.append(f"    constexpr double COLOUR_DEN = Me_{name}::COLOUR_DEN, AVG = Me_{name}::AVG, SYM = Me_{name}::SYM;")
    src.append("    S p[NEXT][4];")
    src.append("    for (int i = 0; i < NEXT; ++i)")
    src.append("        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];")
    src.append(f"    Me_{name}::Inv<R> local;   // used when the caller has no shared-memory slot")
    src.append(f"    Me_{name}::Inv<R>& v = slot ? *static_cast<Me_{name}::Inv<R>*>(slot) : local;")
    for l in pro:
        src.append("    " + l)
    src.append("    // Parity: flipping every helicity leaves the colour-summed |M_h|^2 of these")
    src.append("    // tree amplitudes unchanged, so the sum over all helicities is twice the")
    src.append("    // sum over the configurations with the first gluon at helicity +1.")
    src.append("    R acc = R(0);")
    src.append("#pragma unroll 1")
    src.append("    for (int ih = 1 + 2 * hpart; ih < NHEL; ih += 2 * hparts) {")
    if tc:
        src.append("        if constexpr (TC) {")
        src.append("            // the colour sum synchronises the CTA itself (its barriers replace SYNC's)")
        src.append("            static_assert(SYNC && sizeof(R) == 4, \"tensor-core colour sum: float, whole-CTA calls\");")
        src.append("            hel_" + name + "<R, false>(v, ih);")
        src.append(f"            acc += tc_colour_sum<Me_{name}::NCOL>(static_cast<TcCta*>(cta),")
        src.append("                                                  reinterpret_cast<const volatile float*>(v.jamp));")
        src.append("        } else {")
        src.append("            acc += hel_" + name + "<R>(v, ih);")
        src.append("            if (SYNC) __syncthreads();")
        src.append("        }")
    else:
        src.append("        static_assert(!TC, \"no tensor-core colour sum for this colour basis\");")
        src.append("        acc += hel_" + name + "<R>(v, ih);")
        src.append("        if (SYNC) __syncthreads();")
    src.append("    }")
    src.append("    acc *= R(2);")
    src.append("    S gk = S(1.0);")
    src.append("    for (int i = 0; i < NGLUON; ++i) gk = gk * (gs * gs);")
    src.append("    return S(acc) / COLOUR_DEN * gk * AVG * SYM;")
    src.append("}")
    src.append("")
    src.append("template <typename R, bool SYNC, bool TC, typename S>")
    src.append(f"__device__ S Me_{name}::me2(const S (&p)[NEXT][4], typename NoDeduce<S>::type mt,")
    src.append("    typename NoDeduce<S>::type gs, void* slot, void* cta, int hpart, int hparts)")
    src.append("{")
    src.append(f"    return me2_{name}_impl<R, SYNC, TC, S>(&p[0][0], mt, gs, slot, cta, hpart, hparts);")
    src.append("}")
    src.append("")
    src.append("// the prologue of me2 alone: the event's helicity-independent pieces into v")
    src.append("template <typename R>")
    src.append(f"__device__ __forceinline__ void inv_{name}(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,")
    src.append(f"                                       Me_{name}::Inv<R>& v)")
    src.append("{")
    src.append("    using S = typename Widen<R>::type;")
    src.append(f"    constexpr int NEXT = Me_{name}::NEXT;")
    src.append("    S p[NEXT][4];")
    src.append("    for (int i = 0; i < NEXT; ++i)")
    src.append("        for (int c = 0; c < 4; ++c) p[i][c] = pflat[4 * i + c];")
    for l in pro:
        src.append("    " + l)
    src.append("}")
    src.append("")
    src.append("// Helicity profile: the averaged |M_h|^2 of every one of the NHEL helicity configurations")
    src.append("// (ih bit i: helicity of external particle i, set = +1), parity mirrors included, so that")
    src.append("// out[ih] sums to me2 and out[ih] = out[ih ^ (NHEL - 1)] tests the parity halving of me2")
    src.append("template <typename R>")
    src.append(f"__device__ void hel_profile_{name}(const typename Widen<R>::type* pflat, typename Widen<R>::type mt,")
    src.append(f"                                   typename Widen<R>::type gs, Me_{name}::Inv<R>& v, double* out)")
    src.append("{")
    src.append("    using S = typename Widen<R>::type;")
    src.append(f"    inv_{name}<R>(pflat, mt, v);")
    src.append("    S gk = S(1.0);")
    src.append(f"    for (int i = 0; i < Me_{name}::NGLUON; ++i) gk = gk * (gs * gs);")
    src.append(f"    for (int ih = 0; ih < Me_{name}::NHEL; ++ih)")
    src.append(f"        out[ih] = val(S(hel_{name}<R>(v, ih)) / Me_{name}::COLOUR_DEN * gk * Me_{name}::AVG * Me_{name}::SYM);")
    src.append("}")
    src.append("template <typename R>")
    src.append(f"__device__ void Me_{name}::hel_profile(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt,")
    src.append("                                  typename Widen<R>::type gs, double* out)")
    src.append("{")
    src.append(f"    Me_{name}::Inv<R> v;")
    src.append(f"    hel_profile_{name}<R>(&p[0][0], mt, gs, v, out);")
    src.append("}")
    if tc:
        src.append("")
        src.append("// one helicity's colour-flow amplitudes (the same as hel_" + name + ", without the colour sum);")
        src.append("// the record and the colour-flow row sit at fixed offsets of dynamic shared memory, so that")
        src.append("// both addresses are shared-space offsets derived from threadIdx.x")
        src.append("// (R = float: the record's momenta are read 16 bytes and the colour flows")
        src.append("// updated 8 bytes at a time; REC_STRIDE and JROW keep them aligned)")
        src.append("template <typename R, int JROW, int REC_OFF, int REC_STRIDE>")
        src.append(f"__device__ __noinline__ void hel_{name}_j(int ih)")
        src.append("{")
        src.append(f"    constexpr int NCOL = Me_{name}::NCOL;")
        src.append("    static_assert(sizeof(R) == 4 && REC_OFF % 16 == 0 && REC_STRIDE % 16 == 0 && JROW % 2 == 0,")
        src.append("                  \"aligned float records and colour-flow rows\");")
        src.append("    extern __shared__ __align__(128) unsigned char mf_lh_smem[];")
        src.append(f"    const Me_{name}::Inv<R>& v = *reinterpret_cast<const Me_{name}::Inv<R>*>(")
        src.append("        mf_lh_smem + REC_OFF + (threadIdx.x >> 5) * REC_STRIDE);")
        src.append("    volatile cx<R>* jamp = reinterpret_cast<volatile cx<R>*>(mf_lh_smem + threadIdx.x * (JROW * sizeof(R)));")
        src.append("#define HEL(i) ((ih >> (i)) & 1 ? 1 : -1)")
        assert body[1].startswith("volatile cx<R>* jamp =")
        for l in body[2:]:
            src.append("    " + _wide_access(l))
        src.append("#undef HEL")
        src.append("}")
        src.append("")
        src.append("template <typename R>")
        src.append(f"__device__ void Me_{name}::inv(const typename Widen<R>::type (&p)[NEXT][4], typename Widen<R>::type mt, Inv<R>& v)")
        src.append("{")
        src.append(f"    inv_{name}<R>(&p[0][0], mt, v);")
        src.append("}")
        src.append("template <typename R, int JROW, int REC_OFF, int REC_STRIDE>")
        src.append(f"__device__ void Me_{name}::hel_j(int ih)")
        src.append("{")
        src.append(f"    hel_{name}_j<R, JROW, REC_OFF, REC_STRIDE>(ih);")
        src.append("}")
    src.append("}  // namespace mf")
    stats = dict(n_diag=n_diag, n_amp=len(diags), ncol=ncol, counts=dict(em.counts), colour_den=den)
    stats["flops_per_helicity"] = helicity_flops(em, ncol, CI)
    stats["n_hel"] = 1 << n_ext
    # parity halves the helicity configurations evaluated
    stats["flops_me"] = stats["flops_per_helicity"] * stats["n_hel"] // 2
    stats["flops_me_all_helicities"] = stats["flops_per_helicity"] * stats["n_hel"]
    return "\n".join(src) + "\n", stats


# Floating-point operations of each routine of mf_helas.cuh as written
# (add, sub, mul = 1; fused multiply-add = 2), read off the routine bodies.
ROUTINE_FLOPS = dict(
    vvv=158,        # vvv_cur: 3 momentum combinations, J1.J2, 2 momentum dots, 4 components
    vvvv=264,       # vvvv_cur: 3 dots + 3 two-term combinations per component
    ffv_row=152,    # ffv_row: Sigma/Sigmabar of J, two 2x2 products, two (q-slash + m) halves
    ffv_col=152,    # ffv_col: same structure on a column spinor
    ffv_amp=102,    # ffv_amp: Sigma/Sigmabar of J and two spinor contractions
    vvv_amp=166,    # vvv_amp: 3 dots, 3 momentum dots, 3 products
    vvvv_amp=222,   # vvvv_amp: 6 dots and 3 two-term differences
    ffv_cur=80,     # ffv_cur: 8 complex products and the 4 components
)


def helicity_flops(em: "Emitter", ncol: int, CI) -> int:
    """Algorithmic FLOPs of one helicity configuration of the generated body:
    vertex routines, external states, momentum sums, colour-flow
    accumulation and the colour sum."""
    f = sum(ROUTINE_FLOPS[k] * v for k, v in em.counts.items())
    f += 6 * em.k + 2 * 10                     # external gluon and fermion states
    for line in em.lines:
        if line.startswith("const R k") or line.startswith("const R q"):
            f += line.count("+") + line.count(" - ")
        if line.startswith("jamp[") or ".r +=" in line or ".r -=" in line or "fma(R(" in line:
            f += 2
    nz = sum(1 for i in range(ncol) for j in range(i, ncol) if CI[i][j] != 0)
    f += 2 * 2 * nz + 4 * ncol                  # symmetric colour sum (re and im) and the final products
    return f


if __name__ == "__main__":
    for k in (2, 3, 4):
        print(k, count_feynman_diagrams(k), len(diagrams(k)))

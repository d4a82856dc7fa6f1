"""Exact SU(N) colour algebra for the code generator (N = 3).

Colour factors of tree diagrams are written as products of strings of
generators (T^{a1} ... T^{an})_{ij}; the colour matrix of a set of such
factors, C_{xy} = sum over every colour index of conj(X_x) X_y, closes every
fundamental index into traces, which the Fierz identity

    T^a_{ij} T^a_{kl} = 1/2 (delta_il delta_kj - 1/N delta_ij delta_kl)

reduces to powers of N = Tr(1).  All arithmetic is in exact fractions.
This is the generator's own route to the colour matrix (no explicit
matrices); it shares nothing with the oracle, which sums Gell-Mann matrices
numerically.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from typing import Dict, List, Sequence, Tuple

NC = 3
HALF = Fraction(1, 2)
INV_N = Fraction(1, NC)


def _canon_trace(t: Tuple) -> Tuple:
    """Cyclic canonical form of a trace (smallest rotation)."""
    if not t:
        return t
    return min((tuple(t[i:] + t[:i]) for i in range(len(t))), key=repr)


@lru_cache(maxsize=None)
def _traces_value(traces: Tuple[Tuple, ...]) -> Fraction:
    """Value of a product of traces Tr(w1) Tr(w2) ... in which every adjoint
    label occurs exactly twice (summed)."""
    traces = tuple(t for t in traces)
    # empty traces are N each
    val = Fraction(1)
    rest = []
    for t in traces:
        if len(t) == 0:
            val *= NC
        elif len(t) == 1:
            return Fraction(0)         # Tr(T^a) = 0
        else:
            rest.append(t)
    if not rest:
        return val
    # pick the first label of the first trace and find its partner
    t0 = rest[0]
    a = t0[0]
    # partner in the same trace?
    pos = [i for i, x in enumerate(t0) if x == a]
    if len(pos) == 2:
        i, j = pos
        A = t0[i + 1:j]
        B = t0[j + 1:] + t0[:i]
        # Tr(T^a A T^a B) = 1/2 (Tr A Tr B - 1/N Tr(A B))
        others = tuple(rest[1:])
        v1 = _traces_value(_sorted_traces(others + (A, B)))
        v2 = _traces_value(_sorted_traces(others + (A + B,)))
        return val * HALF * (v1 - INV_N * v2)
    # partner in another trace
    for k in range(1, len(rest)):
        if a in rest[k]:
            t1 = rest[k]
            i = t0.index(a)
            j = t1.index(a)
            A = t0[i + 1:] + t0[:i]          # Tr(T^a A)
            B = t1[j + 1:] + t1[:j]          # Tr(T^a B)
            others = tuple(r for m, r in enumerate(rest) if m not in (0, k))
            # Tr(T^a A) Tr(T^a B) = 1/2 (Tr(A B) - 1/N Tr A Tr B)
            v1 = _traces_value(_sorted_traces(others + (A + B,)))
            v2 = _traces_value(_sorted_traces(others + (A, B)))
            return val * HALF * (v1 - INV_N * v2)
    raise ValueError("unpaired adjoint label %r" % (a,))


def _sorted_traces(ts: Sequence[Tuple]) -> Tuple[Tuple, ...]:
    return tuple(sorted((_canon_trace(tuple(t)) for t in ts), key=repr))


def trace_value(traces: Sequence[Sequence]) -> Fraction:
    return _traces_value(_sorted_traces([tuple(t) for t in traces]))


# A colour factor is a product of open strings: list of (word, i, j) with
# fundamental index labels i (row) and j (column); labels that appear twice
# across strings are contracted.  A colour factor may also be a linear
# combination (list of (coefficient, product)).

String = Tuple[Tuple, str, str]


def close_strings(strings: List[String]) -> List[Tuple]:
    """Contract fundamental indices of a product of strings into traces.
    Each index label must occur once as a row and once as a column index."""
    by_row = {s[1]: s for s in strings}
    used = set()
    traces = []
    for s in strings:
        if id(s) in used:
            continue
        word = []
        cur = s
        while True:
            used.add(id(cur))
            word.extend(cur[0])
            nxt = by_row.get(cur[2])
            if nxt is None:
                raise ValueError("dangling index %s" % cur[2])
            if id(nxt) in used:
                break
            cur = nxt
        traces.append(tuple(word))
    return traces


def conj_strings(strings: List[String], ext_fund, ext_adj) -> List[String]:
    """conj((T^w)_{ij}) = (T^{reverse w})_{ji}.  Summed (internal) labels of
    the conjugated factor are renamed so that they stay distinct from the
    other factor's; external labels are kept (they are summed across both)."""
    def fl(l):
        return l if l in ext_fund else l + "'"

    def al(a):
        return a if a in ext_adj else (a, "'")
    return [(tuple(al(a) for a in reversed(w)), fl(j), fl(i)) for (w, i, j) in strings]


def colour_matrix(factors, ext_fund, ext_adj) -> List[List[complex]]:
    """C[x][y] = sum over all indices of conj(X_x) X_y, where X_x is a linear
    combination sum_k c_k (product of strings)_k.  ext_fund / ext_adj name the
    external quark and gluon colour labels shared by x and y."""
    n = len(factors)
    out = [[0j] * n for _ in range(n)]
    for x in range(n):
        for y in range(n):
            tot = 0j
            for cx, sx in factors[x]:
                for cy, sy in factors[y]:
                    tr = close_strings(conj_strings(sx, ext_fund, ext_adj) + list(sy))
                    v = trace_value(tr)
                    tot += complex(cx).conjugate() * complex(cy) * float(v)
            out[x][y] = tot
    return out


def colour_matrix_words(words: List[Tuple]) -> List[List[Fraction]]:
    """Colour matrix for single strings (T^{w})_{i j} on one open quark line:
    C[x][y] = Tr(T^{reverse w_x} T^{w_y}) as exact fractions."""
    n = len(words)
    return [[trace_value([tuple(reversed(words[x])) + tuple(words[y])]) for y in range(n)] for x in range(n)]


# ---------------------------------------------------------------- word polynomials

Poly = Dict[Tuple, complex]


def pmul(a: Poly, b: Poly) -> Poly:
    out: Poly = {}
    for wa, ca in a.items():
        for wb, cb in b.items():
            w = wa + wb
            out[w] = out.get(w, 0) + ca * cb
    return {w: c for w, c in out.items() if c != 0}


def padd(*ps: Poly, coeffs=None) -> Poly:
    out: Poly = {}
    coeffs = coeffs or [1] * len(ps)
    for p, k in zip(ps, coeffs):
        for w, c in p.items():
            out[w] = out.get(w, 0) + k * c
    return {w: c for w, c in out.items() if c != 0}


def pscale(p: Poly, k: complex) -> Poly:
    return {w: c * k for w, c in p.items() if c * k != 0}


def comm(a: Poly, b: Poly) -> Poly:
    return padd(pmul(a, b), pmul(b, a), coeffs=[1, -1])

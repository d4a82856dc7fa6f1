"""Helpers shared by the GPU parity tests: oracle per-event references and
cut-threshold distances.  Inputs come from paper_2105_10529_gb300.inputs;
expected values come only from the oracle."""
import math

import numpy as np

import oracle as O
from paper_2105_10529_gb300 import inputs as IN

PHYS = {
    IN.EE_MUMU: IN.Physics(sqrt_s=91.19, seed=0),
    IN.GG_TT: IN.Physics(seed=1),
    IN.GG_TTG: IN.Physics(seed=2),
    IN.GG_TTGG: IN.Physics(seed=3),
    IN.UU_TT: IN.Physics(seed=4, channel=1),
    IN.UG_TTU: IN.Physics(seed=5, channel=3),
    IN.GG_TTGGG: IN.Physics(seed=6),
}


def random_grid(dim, nb=50, seed=0):
    """A non-uniform VEGAS grid: sorted random edges with fixed ends."""
    rng = np.random.default_rng(seed)
    g = np.empty((dim, nb + 1))
    for d in range(dim):
        w = rng.uniform(0.2, 1.8, nb)
        e = np.concatenate([[0.0], np.cumsum(w)])
        g[d] = e / e[-1]
        g[d, 0], g[d, -1] = 0.0, 1.0
    return g


def oracle_events(proc, phys, pdf, grid, n, iteration=0, first=0, events=None):
    """Oracle per-event outputs for events first..first+n-1 (or the given list)."""
    idx = list(range(first, first + n)) if events is None else list(events)
    out = dict(u=[], x=[], bins=[], w=[], mask=[], me2=[], p=[], plab=[], x12=[])
    dim = IN.DIM[proc]
    n_ext = IN.N_EXT[proc]
    for o in O.events(proc, phys, pdf, grid, idx, iteration):
        out["u"].append(np.array(o.u[:dim]))
        out["x"].append(np.array(o.x[:dim]))
        out["bins"].append(np.array(o.bins[:dim], dtype=np.uint8))
        out["w"].append(o.w)
        out["mask"].append(o.mask)
        out["me2"].append(o.me2)
        out["p"].append(np.array(o.p[:4 * n_ext]).reshape(n_ext, 4))
        out["plab"].append(np.array(o.plab[:4 * n_ext]).reshape(n_ext, 4))
        out["x12"].append((o.x1, o.x2))
    return {k: np.array(v) for k, v in out.items()}


def cut_margin(proc, phys, plab):
    """Smallest relative distance of a cut variable to its threshold."""
    if proc not in (IN.GG_TTG, IN.GG_TTGG, IN.UG_TTU):
        return math.inf
    light = [4] if proc != IN.GG_TTGG else [4, 5]
    sh = math.sinh(phys.eta_max)
    m = math.inf
    for j in light:
        p = plab[j]
        pt2 = p[1] ** 2 + p[2] ** 2
        m = min(m, abs(pt2 / phys.pt_min ** 2 - 1.0))
        m = min(m, abs(abs(p[3]) / (math.sqrt(pt2) * sh) - 1.0))
    if proc == IN.GG_TTGG:
        a, b = plab[4], plab[5]
        ea = math.asinh(a[3] / math.hypot(a[1], a[2]))
        eb = math.asinh(b[3] / math.hypot(b[1], b[2]))
        dphi = math.atan2(a[2], a[1]) - math.atan2(b[2], b[1])
        dphi = (dphi + math.pi) % (2 * math.pi) - math.pi
        m = min(m, abs(((ea - eb) ** 2 + dphi ** 2) / phys.dr_min ** 2 - 1.0))
    return m


def rambo_gamma(x, n_final):
    """Boost factor Q0/M of RAMBO's conformal map for each event, from the
    VEGAS-mapped points x [n, D] (dimensions 2.. hold 4 uniforms per final
    particle: cos theta = 2u1 - 1, phi = 2 pi u2, E = -ln(u3 u4))."""
    x = np.asarray(x, float)
    Q = np.zeros((x.shape[0], 4))
    for i in range(n_final):
        u = x[:, 2 + 4 * i: 6 + 4 * i]
        c = 2.0 * u[:, 0] - 1.0
        s = np.sqrt(1.0 - c * c)
        f = 2.0 * np.pi * u[:, 1]
        e = -np.log(u[:, 2] * u[:, 3])
        Q += np.stack([e, e * s * np.cos(f), e * s * np.sin(f), e * c], axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - Q[:, 1] ** 2 - Q[:, 2] ** 2 - Q[:, 3] ** 2)
    return Q[:, 0] / M


def rel_err(a, b):
    a = np.asarray(a, float); b = np.asarray(b, float)
    den = np.maximum(np.abs(b), 1e-300)
    return np.where((a == 0) & (b == 0), 0.0, np.abs(a - b) / den)


def assert_fp_parity(err, prec, what="", bound=None):
    """Per-event floating-point parity.  Mixed path: every event within 1e-5.
    FP64 path: every event within its own bound (default 1e-12; the callers pass
    fp64_event_bounds, which exceed 1e-12 only where the event is
    ill-conditioned: a final particle along a beam, a PDF value near x = 1,
    a large RAMBO boost), and the median below 1e-14."""
    err = np.asarray(err, float)
    if err.size == 0:
        return
    if prec == 1:
        assert err.max() < 1e-5, (what, err.max(), int(np.argmax(err)))
        return
    assert_fp64_bounded(err, np.full(err.shape, 1e-12) if bound is None else bound, what)


def check_events_against_oracle(proc, phys, opdf, grid, ev, iteration, prec, first=0, events=None, what=""):
    """Per-event parity of a pass's outputs (a dict of device tensors with
    some of bins, mask, w, me2) against the oracle's events: bins bit-exact,
    masks bit-exact away from a cut threshold, w and |M|^2 within the
    precision's per-event bound.  events: the indices of the pass to check
    (default: all); first: the pass's event offset."""
    n = int(next(iter(ev.values())).shape[0])
    idx = np.arange(n) if events is None else np.asarray(events)
    ref = oracle_events(proc, phys, opdf, grid, 0, iteration=iteration, events=[first + int(i) for i in idx])
    if "bins" in ev:
        assert np.array_equal(ev["bins"].cpu().numpy()[idx], ref["bins"]), what
    same = np.ones(len(idx), dtype=bool)
    if "mask" in ev:
        mk = ev["mask"].cpu().numpy()[idx].astype(int)
        for i in np.nonzero(mk != ref["mask"])[0]:
            assert cut_margin(proc, phys, ref["plab"][i]) < 1e-9, (what, "mask flip far from a threshold", int(idx[i]))
        same = mk == ref["mask"]
    bounds = dict(zip(("me2", "w"), fp64_event_bounds(proc, phys, opdf, ref))) if prec == 0 else {}
    for f in ("w", "me2"):
        if f in ev:
            v = ev[f].cpu().numpy()[idx]
            assert_fp_parity(rel_err(v[same], ref[f][same]), prec, f"{what} {f}",
                             bounds[f][same] if prec == 0 else None)
    return ref


EPS = np.finfo(float).eps
# process -> (PDF flavours of the two incoming partons, masses of the final particles)
_FLAV = {IN.GG_TT: (0, 0), IN.GG_TTG: (0, 0), IN.GG_TTGG: (0, 0), IN.GG_TTGGG: (0, 0), IN.UU_TT: (1, 2),
         IN.UG_TTU: (1, 0)}


def me_condition(proc, phys, p):
    """Condition number of |M|^2 at momenta p [n_ext, 4] (partonic frame): the
    matrix element depends on the momenta through Minkowski products p_i . p_j,
    which cancel for two nearly collinear momenta (a final particle along a
    beam, a gluon along a top); the relative rounding of the momenta reaches
    p_i . p_j amplified by (E_i E_j + |p_i| |p_j|) / |p_i . p_j|.  The largest such
    factor over all pairs (at least 1)."""
    k = 1.0
    n = p.shape[0]
    for i in range(n):
        for j in range(i + 1, n):
            a, b = p[i], p[j]
            dot = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]
            mag = a[0] * b[0] + math.sqrt(a[1] ** 2 + a[2] ** 2 + a[3] ** 2) * math.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2)
            k = max(k, mag / max(abs(dot), 1e-300))
    return k


def pdf_condition(opdf, flav, x, q2):
    """|d ln(x f) / d ln x| + 1 of the interpolated PDF (central difference in
    ln x): how much a relative rounding of ln x (the two paths form it
    differently) grows in the PDF value.  Large where the interpolant nears a
    zero, in the last x cell toward x = 1."""
    if x >= 1.0 or x <= 0.0:
        return 1.0
    h = 1e-6
    lx = math.log(x)
    f0 = opdf.xf(flav, x, q2)
    fp = opdf.xf(flav, min(math.exp(lx + h), 1.0), q2)
    fm = opdf.xf(flav, math.exp(lx - h), q2)
    if f0 == 0.0:
        return 1e300
    return abs((fp - fm) / (2 * h) / f0) + 1.0


def momentum_inconsistency(proc, phys, p):
    """How far momenta p [n_ext, 4] (partonic frame) are from the constraints every
    |M|^2 formula assumes: the largest mass-shell residual |p_i^2 - m_i^2| / E_i^2 and
    the momentum-conservation residual relative to sqrt(shat).  Both sides' RAMBO
    momenta carry these at rounding level, amplified where the conformal map is
    ill-conditioned, and different formulas for |M|^2 (closed form, recursion,
    diagrams) respond to them differently."""
    n_ext = p.shape[0]
    masses = [0.0] * n_ext
    if proc != IN.EE_MUMU:
        masses[2] = masses[3] = phys.mt
    sh = max(abs(p[i][0] ** 2 - p[i][1] ** 2 - p[i][2] ** 2 - p[i][3] ** 2 - masses[i] ** 2) / p[i][0] ** 2
             for i in range(n_ext))
    cons = np.abs(p[0] + p[1] - p[2:].sum(0)).max() / (p[0][0] + p[1][0])
    return max(sh, cons)


def fp64_event_bounds(proc, phys, opdf, ref, p_gpu=None):
    """Per-event bounds for the FP64 path against the oracle, from the
    conditioning of each event (64 eps times the condition numbers, and never
    below 1e-12):
      |M|^2 : 64 eps me_condition, plus 16 me_condition times the inputs'
              disagreement: the larger momentum_inconsistency of the two sides'
              momenta (the oracle's, and the GPU's p_gpu [n, n_ext, 4] where
              given) and their largest difference relative to the largest component;
      w     : that, plus the weight factor's 64 eps sum_i pdf_condition(x_i) (1 + |ln tau|)
              (ln x_i = v ln tau carries an absolute rounding of order eps |ln tau|,
              tau = x1 x2) and the RAMBO map's 8 gamma^2 eps.
    Returns (bound_me2 [n], bound_w [n])."""
    n = len(ref["w"])
    b_me = np.empty(n); b_w = np.empty(n)
    gam = np.ones(n) if proc == IN.EE_MUMU else rambo_gamma(ref["x"], IN.N_EXT[proc] - 2)
    for e in range(n):
        km = me_condition(proc, phys, ref["p"][e])
        inc = momentum_inconsistency(proc, phys, ref["p"][e])
        if p_gpu is not None:
            inc = max(inc, momentum_inconsistency(proc, phys, p_gpu[e]))
            inc += float(np.abs(p_gpu[e] - ref["p"][e]).max() / np.abs(ref["p"][e]).max())
        b_me[e] = max(1e-12, 64 * EPS * km) + 16 * km * inc
        bw = b_me[e] + 8 * gam[e] ** 2 * EPS
        if proc in _FLAV:
            x1, x2 = ref["x12"][e]
            p = ref["p"][e]
            if proc in (IN.GG_TT, IN.UU_TT):
                q2 = phys.mt ** 2
            else:
                ht = sum(math.sqrt((phys.mt ** 2 if i in (2, 3) else 0.0) + p[i][1] ** 2 + p[i][2] ** 2)
                         for i in range(2, p.shape[0]))
                q2 = 0.25 * ht * ht
            f1, f2 = _FLAV[proc]
            ltau = 1 + abs(math.log(x1 * x2))
            bw += 64 * EPS * ltau * (pdf_condition(opdf, f1, x1, q2) + pdf_condition(opdf, f2, x2, q2))
        b_w[e] = max(1e-12, bw)
    return b_me, b_w


def assert_fp64_bounded(err, bound, what=""):
    """FP64 per-event parity: every event within its own conditioning bound,
    and the bulk far below 1e-12 (median under 1e-14 for 100 events or more)."""
    err = np.asarray(err, float); bound = np.asarray(bound, float)
    if err.size == 0:
        return
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (what, [(int(i), float(err[i]), float(bound[i])) for i in bad[:5]])
    if err.size >= 100:
        assert np.median(err) < 1e-14, (what, np.median(err))
